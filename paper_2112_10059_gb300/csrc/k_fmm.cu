// Upward pass, far-field translations, downward pass and the per-leaf
// evaluation (near field + far field) of the kernel-independent FMM
// (paper Section 2.4: Eq. nearfar, Eq. s2l and the recursive hierarchy).
//
// Every box carries two state vectors of n values (rows padded to npad): u_B
// from the sources inside B and d_B from the sources far from B (see OpsDev for
// their meaning under FAR_CHEB / FAR_SURFACE).
//   k_upward     level l, boxes with sources:
//                  leaf  -> P2M: FAR_CHEB    u_B[m] = sum_s S_m(y_s) w_s  (anterpolation)
//                                FAR_SURFACE u_B[i] = sum_s G(|x_i - y_s|) w_s (check potential)
//                  other -> M2M: u_B = sum over children c of M2M_c u_c.
//   k_m2l_simt   level l, target boxes with a V list: d_B += M2L_o u_A (FP32 SIMT).
//   k_p2l        X list: d_B[i] += sum over the coarser leaf's sources of G(|x_i - y_s|) w_s.
//   k_down       level l >= 3: d_B += L2L_c d_parent.
//   k_leaf       leaves with targets: S(t) = L2P + M2P over W + P2P over U (+ self term),
//                written to the dense output.
//                  L2P: FAR_CHEB    sum_m S_m(x_t) d_B[m] (interpolation);
//                       FAR_SURFACE E_l[cell of t] . d_B, or FP64 for leaves too coarse for a table.
//                  M2P: FAR_CHEB    sum_m G(|x_t - y_m^A|) u_A[m];
//                       FAR_SURFACE FP64 equivalent density of A, then FP64 kernel sums.
// CTAs of the box kernels have 2 * npad threads: thread t owns state row t % npad
// and half (t / npad) of the reduction, so each matrix column is read coalesced.
#include "sph_kernels.cuh"

namespace sph {

// Position of cell (i,j,k) relative to the centre of box (coords bx,by,bz, edge size cells), in cm.
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

// 1D Chebyshev Lagrange basis values S_k(x), k < p, of the nodes t[] (FP32).
__device__ __forceinline__ void cheb_basis(int p, const float *t, float x, float *S) {
    for (int k = 0; k < p; ++k) {
        float v = 1.f;
        for (int j = 0; j < p; ++j)
            if (j != k) v *= (x - t[j]) / (t[k] - t[j]);
        S[k] = v;
    }
}

// ------------------------------------------------------------------ upward
constexpr int UT = 256;   // sources per shared tile

__device__ __forceinline__ void upward_box(const FmmDev &F, int level, int b) {
    const TreeDev &T = F.T;
    int sb = T.b_sb[b], se = T.b_se[b];
    if (se <= sb) return;
    const int n = F.O.n, np = F.O.npad;
    __shared__ float vec[MAXPAD];
    __shared__ float part[2][MAXPAD];
    __shared__ uint32_t spc[UT];
    __shared__ float sw[UT];
    __shared__ float bas[UT][3][8];
    __shared__ float tcheb[8];
    const int tid = threadIdx.x, pt = tid % np, half = tid / np;
    const int size = 1 << (F.D - level);
    const float w = F.kp.h * size * 0.5f;
    const float hh = 0.5f * F.kp.h;
    float *u = F.ueq + (size_t)b * np;
    if (T.b_leaf[b]) {
        int bx, by, bz;
        box_coords(T, b, bx, by, bz);
        const bool cheb = F.O.method == FAR_CHEB;
        const int p = F.O.order;
        if (cheb && tid < p) tcheb[tid] = F.O.cheb_t[tid];
        float sx = 0, sy = 0, sz = 0;
        int ia = 0, ib = 0, ic = 0;
        if (pt < n) {
            if (cheb) {
                ia = pt % p; ib = (pt / p) % p; ic = pt / (p * p);
            } else {
                sx = (float)F.O.r.uc * w * F.O.nodes[4 * pt + 0];
                sy = (float)F.O.r.uc * w * F.O.nodes[4 * pt + 1];
                sz = (float)F.O.r.uc * w * F.O.nodes[4 * pt + 2];
            }
        }
        float acc = 0.f;
        const float iw = 1.0f / w;
        for (int s0 = sb; s0 < se; s0 += UT) {
            int m = min(UT, se - s0);
            __syncthreads();
            for (int v = tid; v < m; v += blockDim.x) {
                uint32_t pc = F.src_pc[s0 + v];
                spc[v] = pc;
                sw[v] = F.src_q[s0 + v] * F.wscale;
                if (cheb) {
                    float x, y, z;
                    rel_cell(pc_i(pc), pc_j(pc), pc_k(pc), bx, by, bz, size, hh, x, y, z);
                    cheb_basis(p, tcheb, x * iw, bas[v][0]);
                    cheb_basis(p, tcheb, y * iw, bas[v][1]);
                    cheb_basis(p, tcheb, z * iw, bas[v][2]);
                }
            }
            __syncthreads();
            if (pt < n) {
                if (cheb) {
                    for (int v = half; v < m; v += 2)
                        acc = fmaf(bas[v][0][ia] * bas[v][1][ib] * bas[v][2][ic], sw[v], acc);
                } else {
                    for (int v = half; v < m; v += 2) {
                        uint32_t pc = spc[v];
                        float x, y, z;
                        rel_cell(pc_i(pc), pc_j(pc), pc_k(pc), bx, by, bz, size, hh, x, y, z);
                        float dx = sx - x, dy = sy - y, dz = sz - z;
                        acc = fmaf(g_of_r2(dx * dx + dy * dy + dz * dz, F.kp), sw[v], acc);
                    }
                }
            }
        }
        part[half][pt] = acc;
        __syncthreads();
        if (tid < np) u[tid] = tid < n ? part[0][tid] + part[1][tid] : 0.f;
    } else {
        // M2M from the children (level + 1)
        float acc = 0.f;
        uint32_t ck = T.b_key[b] << 3;
        const int *bat = T.box_at + dense_off(level + 1);
        for (int c = 0; c < 8; ++c) {
            int C = bat[ck + c];
            if (C < 0 || T.b_se[C] <= T.b_sb[C]) continue;   // uniform across the CTA
            __syncthreads();
            if (tid < np) vec[tid] = F.ueq[(size_t)C * np + tid];
            __syncthreads();
            const float *M = F.O.m2m_t + ((size_t)level * 8 + c) * np * np;
            for (int j = half; j < n; j += 2) acc = fmaf(M[(size_t)j * np + pt], vec[j], acc);
        }
        part[half][pt] = acc;
        __syncthreads();
        if (tid < np) u[tid] = tid < n ? part[0][tid] + part[1][tid] : 0.f;
    }
}

// CTAs walk the compact list of this level's boxes that hold sources.
__global__ void __launch_bounds__(2 * MAXPAD) k_upward(FmmDev F, int level, const int *__restrict__ list,
                                                       const int *__restrict__ count) {
    const int cnt = *count;
    for (int i = blockIdx.x; i < cnt; i += gridDim.x) {
        upward_box(F, level, list[i]);
        __syncthreads();
    }
}

void fmm_upward_level(const FmmDev &F, int level, int box_count, const int *list, const int *count,
                      cudaStream_t st) {
    if (box_count <= 0 || level < 2) return;
    int grid = box_count < 152 * 8 ? box_count : 152 * 8;
    k_upward<<<grid, 2 * F.O.npad, 0, st>>>(F, level, list, count);
}

// Compact work lists: per level the boxes with sources (stored in the level's box range),
// and the leaves that the leaf kernel has to visit (any without a table L2P, or with a
// U or W list).
__global__ void k_work_lists(FmmDev F, int nboxes, int *__restrict__ src_list, int *__restrict__ src_cnt,
                             int *__restrict__ leaf_list, int *__restrict__ leaf_cnt) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nboxes) return;
    const TreeDev &T = F.T;
    int l = T.b_level[b];
    if (l >= 2 && T.b_se[b] > T.b_sb[b]) {
        int i = atomicAdd(src_cnt + l, 1);
        src_list[T.lvl_base[l] + i] = b;
    }
    if (T.b_leaf[b] && T.b_te[b] > T.b_tb[b]) {
        bool l2p_done = F.leaf_l2p_done && F.O.method == FAR_CHEB && l >= 2 && F.O.e_off[l] >= 0;
        bool need = !l2p_done || F.L.u_off[b] != F.L.u_off[b + 1] || F.L.w_off[b] != F.L.w_off[b + 1];
        if (need) leaf_list[atomicAdd(leaf_cnt, 1)] = b;
    }
}

void fmm_work_lists(const FmmDev &F, int nboxes, int *src_list, int *src_cnt, int *leaf_list, int *leaf_cnt,
                    cudaStream_t st) {
    if (nboxes <= 0) return;
    k_work_lists<<<(nboxes + 255) / 256, 256, 0, st>>>(F, nboxes, src_list, src_cnt, leaf_list, leaf_cnt);
}

// ------------------------------------------------------------------ M2L (FP32 SIMT)
__global__ void __launch_bounds__(2 * MAXPAD) k_m2l_simt(FmmDev F, int level, int box_begin, int box_count) {
    int b = box_begin + blockIdx.x;
    if (blockIdx.x >= box_count) return;
    int v0 = F.L.v_off[b], v1 = F.L.v_off[b + 1];
    if (v1 <= v0) return;
    const int n = F.O.n, np = F.O.npad;
    __shared__ float vec[MAXPAD];
    __shared__ float part[2][MAXPAD];
    const int tid = threadIdx.x, pt = tid % np, half = tid / np;
    const float *Mlev = F.O.m2l_t + (size_t)level * NSLOT * np * np;
    float acc = 0.f;
    for (int v = v0; v < v1; ++v) {
        int A = F.L.v_src[v];
        int slot = F.O.slot_of_code[F.L.v_oc[v]];
        __syncthreads();
        if (tid < np) vec[tid] = F.ueq[(size_t)A * np + tid];
        __syncthreads();
        const float *M = Mlev + (size_t)slot * np * np;
        for (int j = half; j < n; j += 2) acc = fmaf(M[(size_t)j * np + pt], vec[j], acc);
    }
    part[half][pt] = acc;
    __syncthreads();
    if (tid < n) F.dchk[(size_t)b * np + tid] += part[0][tid] + part[1][tid];
}

void fmm_m2l_level(const FmmDev &F, int level, int box_begin, int box_count, int m2l_prec, cudaStream_t st) {
    if (box_count <= 0 || level < 2) return;
    (void)m2l_prec;
    k_m2l_simt<<<box_count, 2 * F.O.npad, 0, st>>>(F, level, box_begin, box_count);
}

// ------------------------------------------------------------------ P2L (X list)
__global__ void __launch_bounds__(2 * MAXPAD) k_p2l(FmmDev F, int level, int box_begin, int box_count) {
    int b = box_begin + blockIdx.x;
    if (blockIdx.x >= box_count) return;
    int x0 = F.L.x_off[b], x1 = F.L.x_off[b + 1];
    if (x1 <= x0) return;
    const int n = F.O.n, np = F.O.npad;
    __shared__ uint32_t spc[UT];
    __shared__ float sw[UT];
    __shared__ float part[2][MAXPAD];
    const int tid = threadIdx.x, pt = tid % np, half = tid / np;
    const int size = 1 << (F.D - level);
    const float w = F.kp.h * size * 0.5f;
    const float hh = 0.5f * F.kp.h;
    const float rad = F.O.method == FAR_CHEB ? w : (float)F.O.r.dc * w;
    int bx, by, bz;
    box_coords(F.T, b, bx, by, bz);
    float cx = 0, cy = 0, cz = 0;
    if (pt < n) {
        cx = rad * F.O.nodes[4 * pt + 0];
        cy = rad * F.O.nodes[4 * pt + 1];
        cz = rad * F.O.nodes[4 * pt + 2];
    }
    float acc = 0.f;
    for (int x = x0; x < x1; ++x) {
        int A = F.L.x_src[x];
        int sb = F.T.b_sb[A], se = F.T.b_se[A];
        for (int s0 = sb; s0 < se; s0 += UT) {
            int m = min(UT, se - s0);
            __syncthreads();
            for (int v = tid; v < m; v += blockDim.x) {
                spc[v] = F.src_pc[s0 + v];
                sw[v] = F.src_q[s0 + v] * F.wscale;
            }
            __syncthreads();
            if (pt < n) {
                for (int v = half; v < m; v += 2) {
                    uint32_t pc = spc[v];
                    float sx, sy, sz;
                    rel_cell(pc_i(pc), pc_j(pc), pc_k(pc), bx, by, bz, size, hh, sx, sy, sz);
                    float dx = cx - sx, dy = cy - sy, dz = cz - sz;
                    acc = fmaf(g_of_r2(dx * dx + dy * dy + dz * dz, F.kp), sw[v], acc);
                }
            }
        }
    }
    part[half][pt] = acc;
    __syncthreads();
    if (tid < n) F.dchk[(size_t)b * np + tid] += part[0][tid] + part[1][tid];
}

void fmm_p2l_level(const FmmDev &F, int level, int box_begin, int box_count, cudaStream_t st) {
    if (box_count <= 0 || level < 2) return;
    k_p2l<<<box_count, 2 * F.O.npad, 0, st>>>(F, level, box_begin, box_count);
}

// ------------------------------------------------------------------ downward: L2L
__global__ void __launch_bounds__(2 * MAXPAD) k_down(FmmDev F, int level, int box_begin, int box_count) {
    int b = box_begin + blockIdx.x;
    if (blockIdx.x >= box_count) return;
    const TreeDev &T = F.T;
    if (T.b_te[b] <= T.b_tb[b]) return;
    int parent = T.b_parent[b];
    if (level < 3 || parent < 0) return;
    const int n = F.O.n, np = F.O.npad;
    __shared__ float vpar[MAXPAD];
    __shared__ float part[2][MAXPAD];
    const int tid = threadIdx.x, pt = tid % np, half = tid / np;
    if (tid < np) vpar[tid] = F.dchk[(size_t)parent * np + tid];
    __syncthreads();
    int c = (int)(T.b_key[b] & 7u);
    const float *Ml = F.O.l2l_t + ((size_t)level * 8 + c) * np * np;
    float acc = 0.f;
    for (int j = half; j < n; j += 2) acc = fmaf(Ml[(size_t)j * np + pt], vpar[j], acc);
    part[half][pt] = acc;
    __syncthreads();
    if (tid < n) F.dchk[(size_t)b * np + tid] += part[0][tid] + part[1][tid];
}

void fmm_down_level(const FmmDev &F, int level, int box_begin, int box_count, cudaStream_t st) {
    if (box_count <= 0 || level < 3) return;
    k_down<<<box_count, 2 * F.O.npad, 0, st>>>(F, level, box_begin, box_count);
}

// ------------------------------------------------------------------ leaves
constexpr int LT = 128;   // threads per leaf CTA
constexpr int LS = 512;   // sources per shared tile

// eq[i] = sum_k pinv[i][k] chk[k] in FP64 (pinv row-major n x n); all LT threads, ends synchronised.
__device__ __forceinline__ void equiv64(const double *__restrict__ pinv, const float *__restrict__ chk, int n,
                                        double *eq) {
    for (int i = threadIdx.x; i < n; i += LT) {
        double a = 0.0;
        for (int k = 0; k < n; ++k) a = fma(pinv[(size_t)i * n + k], (double)chk[k], a);
        eq[i] = a;
    }
    __syncthreads();
}

// sum_j G(|x - r u_j|) eq[j] in FP64, x relative to the surface centre.
__device__ __forceinline__ double eval64(const double *eq, int n, float r, float x, float y, float z, const FmmDev &F,
                                         const float4 *sv) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) {
        double dx = (double)x - (double)r * sv[j].x;
        double dy = (double)y - (double)r * sv[j].y;
        double dz = (double)z - (double)r * sv[j].z;
        double R = sqrt(dx * dx + dy * dy + dz * dz);
        s = fma(g64(R, F.alpha, F.beta, F.C64), eq[j], s);
    }
    return s;
}

__device__ __forceinline__ void leaf_box(const FmmDev &F, int b, float *__restrict__ out) {
    const TreeDev &T = F.T;
    if (!T.b_leaf[b]) return;
    int tb = T.b_tb[b], te = T.b_te[b];
    if (te <= tb) return;
    const int n = F.O.n, np = F.O.npad;
    const bool cheb = F.O.method == FAR_CHEB;
    const int p = F.O.order;
    const int level = T.b_level[b];
    const int size = 1 << (F.D - level);
    // a table L2P (k_l2p_gemm) already wrote S for this leaf: add the near field only
    const bool l2p_done = F.leaf_l2p_done && cheb && level >= 2 && F.O.e_off[level] >= 0;
    if (l2p_done && F.L.u_off[b] == F.L.u_off[b + 1] && F.L.w_off[b] == F.L.w_off[b + 1]) return;
    const float hh = 0.5f * F.kp.h;
    int bx, by, bz;
    box_coords(T, b, bx, by, bz);
    __shared__ float4 sv[MAXPAD];                  // unit node positions
    __shared__ __align__(16) float sd[MAXPAD];     // a state vector
    __shared__ double sd64[MAXPAD];
    __shared__ uint32_t spc[LS];
    __shared__ float sw[LS];
    __shared__ float tcheb[8];
    __shared__ float ctab[16][8];                  // Chebyshev basis at the cell positions of one axis
    for (int j = threadIdx.x; j < np; j += LT)
        sv[j] = make_float4(F.O.nodes[4 * j], F.O.nodes[4 * j + 1], F.O.nodes[4 * j + 2], 0.f);
    if (cheb && threadIdx.x < p) tcheb[threadIdx.x] = F.O.cheb_t[threadIdx.x];
    if (cheb && level >= 2 && size <= 16) {
        __syncthreads();
        // unit coordinate of cell l along an axis: (2 l + 1 - size) / size
        for (int e = threadIdx.x; e < size * p; e += LT) {
            int l = e / p, a = e % p;
            float x = (float)(2 * l + 1 - size) / (float)size;
            float v = 1.f;
            for (int j = 0; j < p; ++j)
                if (j != a) v *= (x - tcheb[j]) / (tcheb[a] - tcheb[j]);
            ctab[l][a] = v;
        }
    }

    for (int t0 = tb; t0 < te; t0 += LT) {
        int t = t0 + threadIdx.x;
        bool act = t < te;
        uint32_t tp = act ? F.trg_pc[t] : 0u;
        int ti = pc_i(tp), tj = pc_j(tp), tk = pc_k(tp);
        float tx, ty, tz;
        rel_cell(ti, tj, tk, bx, by, bz, size, hh, tx, ty, tz);
        float acc = 0.f;
        // ---- L2P (levels >= 2)
        if (level >= 2 && !l2p_done) {
            const float w = F.kp.h * size * 0.5f;
            __syncthreads();
            if (cheb) {
                for (int j = threadIdx.x; j < np; j += LT) sd[j] = F.dchk[(size_t)b * np + j];
                __syncthreads();
                if (act) {
                    float Sx[8], Sy[8], Sz[8];
                    if (size <= 16) {   // cell centres sit at size fixed positions per axis: table
                        const int lx = ti - bx * size, ly = tj - by * size, lz = tk - bz * size;
                        for (int a = 0; a < p; ++a) {
                            Sx[a] = ctab[lx][a];
                            Sy[a] = ctab[ly][a];
                            Sz[a] = ctab[lz][a];
                        }
                    } else {
                        const float iw = 1.0f / w;
                        cheb_basis(p, tcheb, tx * iw, Sx);
                        cheb_basis(p, tcheb, ty * iw, Sy);
                        cheb_basis(p, tcheb, tz * iw, Sz);
                    }
                    for (int c = 0; c < p; ++c) {
                        float zc = 0.f;
                        for (int bb = 0; bb < p; ++bb) {
                            const float *row = sd + p * (bb + p * c);
                            float r = 0.f;
                            for (int a = 0; a < p; ++a) r = fmaf(Sx[a], row[a], r);
                            zc = fmaf(Sy[bb], r, zc);
                        }
                        acc = fmaf(Sz[c], zc, acc);
                    }
                }
            } else {
                const long long eo = F.O.e_off[level];
                if (eo >= 0) {
                    for (int j = threadIdx.x; j < np; j += LT) sd[j] = F.dchk[(size_t)b * np + j];
                    __syncthreads();
                    if (act) {
                        int lx = ti - bx * size, ly = tj - by * size, lz = tk - bz * size;
                        const float4 *row =
                            (const float4 *)(F.O.e_tab + eo + (size_t)(lx + size * (ly + size * lz)) * np);
                        const float4 *d4 = (const float4 *)sd;
                        for (int j = 0; j < np / 4; ++j) {
                            float4 a = __ldg(row + j), v = d4[j];
                            acc = fmaf(a.x, v.x, fmaf(a.y, v.y, fmaf(a.z, v.z, fmaf(a.w, v.w, acc))));
                        }
                    }
                } else {
                    equiv64(F.O.dc64 + (size_t)level * F.O.pinv_stride, F.dchk + (size_t)b * np, n, sd64);
                    if (act) acc += (float)eval64(sd64, n, (float)F.O.r.de * w, tx, ty, tz, F, sv);
                }
            }
        }
        // ---- M2P over the W list (finer boxes A not adjacent to this leaf)
        for (int wv = F.L.w_off[b]; wv < F.L.w_off[b + 1]; ++wv) {
            int A = F.L.w_src[wv];
            int al = T.b_level[A];
            int asz = 1 << (F.D - al);
            int ax, ay, az;
            box_coords(T, A, ax, ay, az);
            const float aw = F.kp.h * asz * 0.5f;
            float rx, ry, rz;
            rel_cell(ti, tj, tk, ax, ay, az, asz, hh, rx, ry, rz);
            __syncthreads();
            if (cheb) {
                for (int j = threadIdx.x; j < np; j += LT) sd[j] = F.ueq[(size_t)A * np + j];
                __syncthreads();
                if (act) {
                    for (int j = 0; j < n; ++j) {
                        float dx = rx - aw * sv[j].x, dy = ry - aw * sv[j].y, dz = rz - aw * sv[j].z;
                        acc = fmaf(g_of_r2(dx * dx + dy * dy + dz * dz, F.kp), sd[j], acc);
                    }
                }
            } else {
                equiv64(F.O.uc64 + (size_t)al * F.O.pinv_stride, F.ueq + (size_t)A * np, n, sd64);
                if (act) acc += (float)eval64(sd64, n, (float)F.O.r.ue * aw, rx, ry, rz, F, sv);
            }
        }
        // ---- P2P over the U list (near field, Eq. nearfar), with the self term
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
                        uint32_t pc = spc[u];
                        int di = ti - pc_i(pc), dj = tj - pc_j(pc), dk = tk - pc_k(pc);
                        int d2 = di * di + dj * dj + dk * dk;
                        float g = d2 ? g_of_cells(d2, F.kp) : (F.self_mode ? F.kp.gself : 0.f);
                        acc = fmaf(g, sw[u], acc);
                    }
                }
            }
        }
        if (act) {
            float *o = out + (int64_t)ti + (int64_t)F.nx * ((int64_t)tj + (int64_t)F.ny * tk);
            *o = l2p_done ? *o + acc : acc;
        }
    }
}

// CTAs walk the compact list of leaves that need this kernel.
__global__ void __launch_bounds__(LT) k_leaf(FmmDev F, const int *__restrict__ list, const int *__restrict__ count,
                                             float *__restrict__ out) {
    const int cnt = *count;
    for (int i = blockIdx.x; i < cnt; i += gridDim.x) {
        leaf_box(F, list[i], out);
        __syncthreads();
    }
}

void fmm_leaf(const FmmDev &F, int nboxes, const int *list, const int *count, float *out_dense, cudaStream_t st) {
    if (nboxes <= 0) return;
    int grid = nboxes < 152 * 16 ? nboxes : 152 * 16;
    k_leaf<<<grid, LT, 0, st>>>(F, list, count, out_dense);
}

}  // namespace sph
