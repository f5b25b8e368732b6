// Upward pass, far-field translations, downward pass and the per-leaf
// evaluation (near field + local expansion) of the kernel-independent FMM
// (paper Section 2.4: Eq. nearfar, Eq. s2l and the recursive hierarchy).
//
// Surface vectors (check potentials, equivalent densities) are rows of 160
// floats (152 used) per box.  Matrices are stored transposed ([col][row]) so a
// CTA with one thread per output row reads each column coalesced.
//
//   k_upward     level l, boxes with sources:
//                  leaf  -> P2M: upward check potential by direct kernel sums
//                           over the box's sources, then UC2E;
//                  other -> M2M: sum over children of (UC2E M2M-kernel) ueq_child.
//   k_m2l_simt   level l, target boxes with a V list: dchk += M2L_o ueq_A (FP32 SIMT).
//   k_p2l        X list: dchk += kernel sums from the sources of coarser leaves.
//   k_down       level l: deq = DC2E dchk + (DC2E L2L-kernel) deq_parent.
//   k_leaf       leaves with targets: S(t) = L2P(deq) + M2P over W + P2P over U
//                (+ the self term), written to the dense output.
#include "sph_kernels.cuh"

namespace sph {

constexpr int PPAD = SPH_PP;
constexpr int P = SPH_P;
constexpr int NSLOT = 316;

// Position of cell (i,j,k) relative to the centre of box (level l, coords bx,by,bz), in cm.
// Box centre in half-cell units: 2*b*size + size; cell centre: 2*i + 1.
__device__ __forceinline__ void rel_cell(int i, int j, int k, int bx, int by, int bz, int size, float hh,
                                         float &x, float &y, float &z) {
    x = (float)(2 * i + 1 - (2 * bx * size + size)) * hh;
    y = (float)(2 * j + 1 - (2 * by * size + size)) * hh;
    z = (float)(2 * k + 1 - (2 * bz * size + size)) * hh;
}

__device__ __forceinline__ void box_coords(const TreeDev &T, int b, int &x, int &y, int &z) {
    uint32_t ux, uy, uz;
    demorton3(T.b_key[b], ux, uy, uz);
    x = (int)ux; y = (int)uy; z = (int)uz;
}

// ------------------------------------------------------------------ upward
// blockDim = 320: thread t handles surface point t % 160 and half (t / 160) of the sources.
__global__ void __launch_bounds__(320) k_upward(FmmDev F, int level, int box_begin, int box_count) {
    int b = box_begin + blockIdx.x;
    if (blockIdx.x >= box_count) return;
    const TreeDev &T = F.T;
    int sb = T.b_sb[b], se = T.b_se[b];
    if (se <= sb) return;
    __shared__ float vec[PPAD];
    __shared__ float part[2][PPAD];
    __shared__ uint32_t spc[256];
    __shared__ float sw[256];
    const int tid = threadIdx.x, pt = tid % PPAD, half = tid / PPAD;
    const int size = 1 << (F.D - level);
    const float w = F.kp.h * size * 0.5f;
    float *ueq = F.ueq + (size_t)b * PPAD;
    if (T.b_leaf[b]) {
        int bx, by, bz;
        box_coords(T, b, bx, by, bz);
        float sx = 0, sy = 0, sz = 0;
        if (pt < P) {
            sx = (float)R_UC * w * F.O.surf[4 * pt + 0];
            sy = (float)R_UC * w * F.O.surf[4 * pt + 1];
            sz = (float)R_UC * w * F.O.surf[4 * pt + 2];
        }
        float acc = 0.f;
        const float hh = 0.5f * F.kp.h;
        for (int s0 = sb; s0 < se; s0 += 256) {
            int m = min(256, se - s0);
            __syncthreads();
            for (int u = tid; u < m; u += blockDim.x) {
                spc[u] = F.src_pc[s0 + u];
                sw[u] = F.src_q[s0 + u] * F.wscale;
            }
            __syncthreads();
            if (pt < P) {
                for (int u = half; u < m; u += 2) {
                    uint32_t p = spc[u];
                    float x, y, z;
                    rel_cell(pc_i(p), pc_j(p), pc_k(p), bx, by, bz, size, hh, x, y, z);
                    float dx = sx - x, dy = sy - y, dz = sz - z;
                    acc = fmaf(g_of_r2(dx * dx + dy * dy + dz * dz, F.kp), sw[u], acc);
                }
            }
        }
        part[half][pt] = acc;
        __syncthreads();
        if (tid < PPAD) vec[tid] = tid < P ? part[0][tid] + part[1][tid] : 0.f;
        __syncthreads();
        // ueq = UC2E * check
        const float *M = F.O.uc2e_t + (size_t)level * PPAD * PPAD;
        float a0 = 0.f;
        for (int j = half; j < P; j += 2) a0 = fmaf(M[j * PPAD + pt], vec[j], a0);
        part[half][pt] = a0;
        __syncthreads();
        if (tid < PPAD) ueq[tid] = tid < P ? part[0][tid] + part[1][tid] : 0.f;
    } else {
        // M2M from the children (level + 1)
        float acc = 0.f;
        uint32_t ck = T.b_key[b] << 3;
        const int *bat = T.box_at + dense_off(level + 1);
        for (int c = 0; c < 8; ++c) {
            int C = bat[ck + c];
            if (C < 0 || T.b_se[C] <= T.b_sb[C]) continue;   // uniform across the CTA
            __syncthreads();
            if (tid < PPAD) vec[tid] = F.ueq[(size_t)C * PPAD + tid];
            __syncthreads();
            const float *M = F.O.m2m_t + ((size_t)level * 8 + c) * PPAD * PPAD;
            for (int j = half; j < P; j += 2) acc = fmaf(M[j * PPAD + pt], vec[j], acc);
        }
        part[half][pt] = acc;
        __syncthreads();
        if (tid < PPAD) ueq[tid] = tid < P ? part[0][tid] + part[1][tid] : 0.f;
    }
}

void fmm_upward_level(const FmmDev &F, int level, int box_begin, int box_count, cudaStream_t st) {
    if (box_count <= 0 || level < 2) return;
    k_upward<<<box_count, 320, 0, st>>>(F, level, box_begin, box_count);
}

// ------------------------------------------------------------------ M2L (FP32 SIMT)
__global__ void __launch_bounds__(320) k_m2l_simt(FmmDev F, int level, int box_begin, int box_count) {
    int b = box_begin + blockIdx.x;
    if (blockIdx.x >= box_count) return;
    int v0 = F.L.v_off[b], v1 = F.L.v_off[b + 1];
    if (v1 <= v0) return;
    __shared__ float vec[PPAD];
    __shared__ float part[2][PPAD];
    const int tid = threadIdx.x, pt = tid % PPAD, half = tid / PPAD;
    const float *Mlev = F.O.m2l_t + (size_t)level * NSLOT * PPAD * PPAD;
    float acc = 0.f;
    for (int v = v0; v < v1; ++v) {
        int A = F.L.v_src[v];
        int slot = F.O.slot_of_code[F.L.v_oc[v]];
        __syncthreads();
        if (tid < PPAD) vec[tid] = F.ueq[(size_t)A * PPAD + tid];
        __syncthreads();
        const float *M = Mlev + (size_t)slot * PPAD * PPAD;
        for (int j = half; j < P; j += 2) acc = fmaf(M[j * PPAD + pt], vec[j], acc);
    }
    part[half][pt] = acc;
    __syncthreads();
    if (tid < P) F.dchk[(size_t)b * PPAD + tid] += part[0][tid] + part[1][tid];
}

void fmm_m2l_level(const FmmDev &F, int level, int box_begin, int box_count, int m2l_prec, cudaStream_t st) {
    if (box_count <= 0 || level < 2) return;
    (void)m2l_prec;
    k_m2l_simt<<<box_count, 320, 0, st>>>(F, level, box_begin, box_count);
}

// ------------------------------------------------------------------ P2L (X list)
__global__ void __launch_bounds__(320) k_p2l(FmmDev F, int level, int box_begin, int box_count) {
    int b = box_begin + blockIdx.x;
    if (blockIdx.x >= box_count) return;
    int x0 = F.L.x_off[b], x1 = F.L.x_off[b + 1];
    if (x1 <= x0) return;
    __shared__ uint32_t spc[256];
    __shared__ float sw[256];
    __shared__ float part[2][PPAD];
    const int tid = threadIdx.x, pt = tid % PPAD, half = tid / PPAD;
    const int size = 1 << (F.D - level);
    const float w = F.kp.h * size * 0.5f;
    const float hh = 0.5f * F.kp.h;
    int bx, by, bz;
    box_coords(F.T, b, bx, by, bz);
    float cx = 0, cy = 0, cz = 0;
    if (pt < P) {
        cx = (float)R_DC * w * F.O.surf[4 * pt + 0];
        cy = (float)R_DC * w * F.O.surf[4 * pt + 1];
        cz = (float)R_DC * w * F.O.surf[4 * pt + 2];
    }
    float acc = 0.f;
    for (int x = x0; x < x1; ++x) {
        int A = F.L.x_src[x];
        int sb = F.T.b_sb[A], se = F.T.b_se[A];
        for (int s0 = sb; s0 < se; s0 += 256) {
            int m = min(256, se - s0);
            __syncthreads();
            for (int u = tid; u < m; u += blockDim.x) {
                spc[u] = F.src_pc[s0 + u];
                sw[u] = F.src_q[s0 + u] * F.wscale;
            }
            __syncthreads();
            if (pt < P) {
                for (int u = half; u < m; u += 2) {
                    uint32_t p = spc[u];
                    float sx, sy, sz;
                    rel_cell(pc_i(p), pc_j(p), pc_k(p), bx, by, bz, size, hh, sx, sy, sz);
                    float dx = cx - sx, dy = cy - sy, dz = cz - sz;
                    acc = fmaf(g_of_r2(dx * dx + dy * dy + dz * dz, F.kp), sw[u], acc);
                }
            }
        }
    }
    part[half][pt] = acc;
    __syncthreads();
    if (tid < P) F.dchk[(size_t)b * PPAD + tid] += part[0][tid] + part[1][tid];
}

void fmm_p2l_level(const FmmDev &F, int level, int box_begin, int box_count, cudaStream_t st) {
    if (box_count <= 0 || level < 2) return;
    k_p2l<<<box_count, 320, 0, st>>>(F, level, box_begin, box_count);
}

// ------------------------------------------------------------------ downward: DC2E + L2L
__global__ void __launch_bounds__(320) k_down(FmmDev F, int level, int box_begin, int box_count) {
    int b = box_begin + blockIdx.x;
    if (blockIdx.x >= box_count) return;
    const TreeDev &T = F.T;
    if (T.b_te[b] <= T.b_tb[b]) return;
    __shared__ float vchk[PPAD], vpar[PPAD];
    __shared__ float part[2][PPAD];
    const int tid = threadIdx.x, pt = tid % PPAD, half = tid / PPAD;
    int parent = T.b_parent[b];
    bool has_parent = level >= 3 && parent >= 0;
    if (tid < PPAD) {
        vchk[tid] = F.dchk[(size_t)b * PPAD + tid];
        vpar[tid] = has_parent ? F.deq[(size_t)parent * PPAD + tid] : 0.f;
    }
    __syncthreads();
    const float *Md = F.O.dc2e_t + (size_t)level * PPAD * PPAD;
    float acc = 0.f;
    for (int j = half; j < P; j += 2) acc = fmaf(Md[j * PPAD + pt], vchk[j], acc);
    if (has_parent) {
        int c = (int)(T.b_key[b] & 7u);
        const float *Ml = F.O.l2l_t + ((size_t)level * 8 + c) * PPAD * PPAD;
        for (int j = half; j < P; j += 2) acc = fmaf(Ml[j * PPAD + pt], vpar[j], acc);
    }
    part[half][pt] = acc;
    __syncthreads();
    if (tid < PPAD) F.deq[(size_t)b * PPAD + tid] = tid < P ? part[0][tid] + part[1][tid] : 0.f;
}

void fmm_down_level(const FmmDev &F, int level, int box_begin, int box_count, cudaStream_t st) {
    if (box_count <= 0 || level < 2) return;
    k_down<<<box_count, 320, 0, st>>>(F, level, box_begin, box_count);
}

// ------------------------------------------------------------------ leaves
// One CTA (128 threads) per box; thread t handles targets t, t+128, ... of the box.
constexpr int LT = 128;
constexpr int LS = 512;   // sources per shared tile

__global__ void __launch_bounds__(LT) k_leaf(FmmDev F, int nboxes, float *__restrict__ out) {
    int b = blockIdx.x;
    const TreeDev &T = F.T;
    if (!T.b_leaf[b]) return;
    int tb = T.b_tb[b], te = T.b_te[b];
    if (te <= tb) return;
    const int level = T.b_level[b];
    const int size = 1 << (F.D - level);
    const float hh = 0.5f * F.kp.h;
    int bx, by, bz;
    box_coords(T, b, bx, by, bz);
    __shared__ float4 sv[PPAD];          // equivalent points (x, y, z, density)
    __shared__ uint32_t spc[LS];
    __shared__ float sw[LS];

    for (int t0 = tb; t0 < te; t0 += LT) {
        int t = t0 + threadIdx.x;
        bool act = t < te;
        uint32_t tp = act ? F.trg_pc[t] : 0u;
        int ti = pc_i(tp), tj = pc_j(tp), tk = pc_k(tp);
        float tx, ty, tz;
        rel_cell(ti, tj, tk, bx, by, bz, size, hh, tx, ty, tz);
        float acc = 0.f;
        // L2P: downward equivalent density of this box (levels >= 2)
        if (level >= 2) {
            const float w = F.kp.h * size * 0.5f;
            __syncthreads();
            for (int j = threadIdx.x; j < P; j += LT) {
                sv[j] = make_float4((float)R_DE * w * F.O.surf[4 * j + 0], (float)R_DE * w * F.O.surf[4 * j + 1],
                                    (float)R_DE * w * F.O.surf[4 * j + 2], F.deq[(size_t)b * PPAD + j]);
            }
            __syncthreads();
            if (act) {
                for (int j = 0; j < P; ++j) {
                    float4 e = sv[j];
                    float dx = tx - e.x, dy = ty - e.y, dz = tz - e.z;
                    acc = fmaf(g_of_r2(dx * dx + dy * dy + dz * dz, F.kp), e.w, acc);
                }
            }
        }
        // M2P over the W list: upward equivalent densities of finer boxes
        for (int wv = F.L.w_off[b]; wv < F.L.w_off[b + 1]; ++wv) {
            int A = F.L.w_src[wv];
            int al = T.b_level[A];
            int asz = 1 << (F.D - al);
            int ax, ay, az;
            box_coords(T, A, ax, ay, az);
            const float aw = F.kp.h * asz * 0.5f;
            // target position relative to A's centre
            float rx, ry, rz;
            rel_cell(ti, tj, tk, ax, ay, az, asz, hh, rx, ry, rz);
            __syncthreads();
            for (int j = threadIdx.x; j < P; j += LT) {
                sv[j] = make_float4((float)R_UE * aw * F.O.surf[4 * j + 0], (float)R_UE * aw * F.O.surf[4 * j + 1],
                                    (float)R_UE * aw * F.O.surf[4 * j + 2], F.ueq[(size_t)A * PPAD + j]);
            }
            __syncthreads();
            if (act) {
                for (int j = 0; j < P; ++j) {
                    float4 e = sv[j];
                    float dx = rx - e.x, dy = ry - e.y, dz = rz - e.z;
                    acc = fmaf(g_of_r2(dx * dx + dy * dy + dz * dz, F.kp), e.w, acc);
                }
            }
        }
        // P2P over the U list (near field, Eq. nearfar), with the self term
        for (int uv = F.L.u_off[b]; uv < F.L.u_off[b + 1]; ++uv) {
            int A = F.L.u_src[uv];
            int sb = T.b_sb[A], se = T.b_se[A];
            for (int s0 = sb; s0 < se; s0 += LS) {
                int m = min(LS, se - s0);
                __syncthreads();
                for (int u = threadIdx.x; u < m; u += LT) {
                    spc[u] = F.src_pc[s0 + u];
                    sw[u] = F.src_q[s0 + u] * F.wscale;
                }
                __syncthreads();
                if (act) {
                    for (int u = 0; u < m; ++u) {
                        uint32_t p = spc[u];
                        int di = ti - pc_i(p), dj = tj - pc_j(p), dk = tk - pc_k(p);
                        int d2 = di * di + dj * dj + dk * dk;
                        float g = d2 ? g_of_cells(d2, F.kp) : (F.self_mode ? F.kp.gself : 0.f);
                        acc = fmaf(g, sw[u], acc);
                    }
                }
            }
        }
        if (act) out[(int64_t)ti + (int64_t)F.nx * ((int64_t)tj + (int64_t)F.ny * tk)] = acc;
    }
}

void fmm_leaf(const FmmDev &F, int nboxes, int leaf_cap, float *out_dense, cudaStream_t st) {
    if (nboxes <= 0) return;
    (void)leaf_cap;
    k_leaf<<<nboxes, LT, 0, st>>>(F, nboxes, out_dense);
}

}  // namespace sph
