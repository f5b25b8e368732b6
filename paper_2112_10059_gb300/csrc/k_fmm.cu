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
#include <algorithm>

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

// The same basis from the barycentric weights w_k = 1 / prod_{j != k} (t_k - t_j):
// S_k(x) = w_k prod_{j < k} (x - t_j) prod_{j > k} (x - t_j), by prefix and suffix products
// (no division per evaluation).
__device__ __forceinline__ void cheb_basis_w(int p, const float *t, const float *w, float x, float *S) {
    float d[8], pre[8];
    float acc = 1.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {          // fixed trip counts: the arrays stay in registers
        d[k] = k < p ? x - t[k] : 1.f;
        pre[k] = acc;
        acc *= d[k];
    }
    float suf = 1.f;
#pragma unroll
    for (int k = 7; k >= 0; --k) {
        if (k < p) S[k] = w[k] * pre[k] * suf;
        suf *= d[k];
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
    __shared__ float tcheb[8], wcheb[8];
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
        if (cheb && tid < p) {
            const float tk = F.O.cheb_t[tid];
            float w = 1.f;
            for (int j = 0; j < p; ++j)
                if (j != tid) w *= tk - F.O.cheb_t[j];
            tcheb[tid] = tk;
            wcheb[tid] = 1.f / w;
        }
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
                    cheb_basis_w(p, tcheb, wcheb, x * iw, bas[v][0]);
                    cheb_basis_w(p, tcheb, wcheb, y * iw, bas[v][1]);
                    cheb_basis_w(p, tcheb, wcheb, z * iw, bas[v][2]);
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
// leaves_only: the split boxes' M2M runs on the tensor cores (k_m2m_tc)
__global__ void __launch_bounds__(2 * MAXPAD) k_upward(FmmDev F, int level, const int *__restrict__ list,
                                                       const int *__restrict__ count, int leaves_only) {
    pdl_enter();
    const int cnt = *count;
    for (int i = blockIdx.x; i < cnt; i += gridDim.x) {
        const int b = list[i];
        if (leaves_only && !F.T.b_leaf[b]) continue;   // uniform across the CTA
        upward_box(F, level, b);
        __syncthreads();
    }
}

int fmm_upward_level(const FmmDev &F, int level, int box_count, const int *list, const int *count, bool leaves_only,
                     cudaStream_t st) {
    if (box_count <= 0 || level < 2) return 0;
    int grid = box_count < 152 * 8 ? box_count : 152 * 8;
    launch_pdl(k_upward, grid, 2 * F.O.npad, 0, st, F, level, list, count, leaves_only ? 1 : 0);
    return 1;
}

// Compact work lists: per level the boxes with sources (stored in the level's box range),
// and the leaves that the leaf kernel has to visit (any without a table L2P, or with a
// U or W list).
// Append with one atomic per (warp, counter): lanes with `pred` that share a counter get
// consecutive slots from the group's leader.  Every lane of `act` must call it.
__device__ __forceinline__ int warp_append(unsigned act, bool pred, int *counter) {
    const int lane = threadIdx.x & 31;
    const unsigned long long key = pred ? reinterpret_cast<unsigned long long>(counter) : 0ull;
    const unsigned grp = __match_any_sync(act, key);
    const int leader = __ffs(grp) - 1;
    int base = 0;
    if (pred && lane == leader) base = atomicAdd(counter, __popc(grp));
    base = __shfl_sync(grp, base, leader);
    return base + __popc(grp & ((1u << lane) - 1u));
}

__global__ void k_work_lists(FmmDev F, int nboxes, int *__restrict__ src_list, int *__restrict__ src_cnt,
                             int *__restrict__ leaf_list, int *__restrict__ leaf_cnt, int *__restrict__ p2p_list,
                             int *__restrict__ p2p_cnt, int p2p_stride, int *__restrict__ own_list,
                             int *__restrict__ own_cnt, int *__restrict__ w_list, int *__restrict__ w_cnt) {
    pdl_enter();
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nboxes) return;
    const unsigned act = __activemask();
    const TreeDev &T = F.T;
    const int l = T.b_level[b];
    const bool has_src = l >= 2 && T.b_se[b] > T.b_sb[b];
    const bool leaf_t = T.b_leaf[b] && T.b_te[b] > T.b_tb[b];
    bool need = false, p2p = false, has_w = false;
    if (leaf_t) {
        bool l2p_done = F.leaf_l2p_done && F.O.method == FAR_CHEB && l >= 2 && (F.O.e_off[l] >= 0 || F.l2p_sep);
        bool has_u = F.L.u_off[b] != F.L.u_off[b + 1];
        has_w = F.L.w_off[b] != F.L.w_off[b + 1];
        // the separate near-field kernel takes U and (Chebyshev far field) W lists
        bool w_sep = F.p2p_separate && F.O.method == FAR_CHEB;
        need = !l2p_done || ((has_u || has_w) && !F.p2p_separate) || (has_w && !w_sep);
        p2p = F.p2p_separate && (has_u || (has_w && w_sep));
    }
    int i = warp_append(act, has_src, src_cnt + l);
    if (has_src) src_list[T.lvl_base[l] + i] = b;
    // split boxes with sources: the tensor-core M2M adds its children's terms into a zeroed row
    if (has_src && !T.b_leaf[b] && F.O.m2m_img != nullptr) {
        float4 *u = reinterpret_cast<float4 *>(F.ueq + (size_t)b * F.O.npad);
        for (int j = 0; j < F.O.npad / 4; ++j) u[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    // deepest level under the fused L2L + L2P: only the rows that M2L / P2L add into are
    // cleared, and those leaves (with targets) listed for the L2P of their own local terms
    const bool own = F.d_sparse_from >= 0 && b >= F.d_sparse_from &&
                     (F.L.v_off[b + 1] != F.L.v_off[b] || F.L.x_off[b + 1] != F.L.x_off[b]);
    if (own) {
        float4 *d = reinterpret_cast<float4 *>(F.dchk + (size_t)b * F.O.npad);
        for (int j = 0; j < F.O.npad / 4; ++j) d[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    i = warp_append(act, own && leaf_t, own_cnt);
    if (own && leaf_t) own_list[i] = b;
    // per level, the leaves with targets (the separable L2P walks these only; the fused deepest
    // level, whose boxes start at d_sparse_from, needs no list)
    const bool l2p = leaf_t && l >= 2 && F.l2p_list != nullptr && !(F.d_sparse_from >= 0 && b >= F.d_sparse_from);
    i = warp_append(act, l2p, F.l2p_cnt + l);
    if (l2p) F.l2p_list[T.lvl_base[l] + i] = b;
    i = warp_append(act, need, leaf_cnt);
    if (need) leaf_list[i] = b;
    // near-field leaves by their number of kernel evaluations (targets x U-list sources and
    // W-list nodes), in classes of halving size, so that the near field can start the heaviest
    // first and end on light ones
    int cls = P2P_CLASSES - 1;
    if (p2p) {
        int64_t ns = 0;
        for (int u = F.L.u_off[b]; u < F.L.u_off[b + 1]; ++u) {
            const int A = F.L.u_src[u];
            ns += T.b_se[A] - T.b_sb[A];
        }
        if (F.O.method == FAR_CHEB) ns += (int64_t)(F.L.w_off[b + 1] - F.L.w_off[b]) * F.O.n;   // W nodes
        const int64_t w = ns * (T.b_te[b] - T.b_tb[b]);
        cls = 0;
        while (cls < P2P_CLASSES - 1 && w < (P2P_CLASS0 >> cls)) ++cls;
    }
    int my_idx = 0;
    for (int c = 0; c < P2P_CLASSES; ++c) {
        const bool in = p2p && cls == c;
        i = warp_append(act, in, p2p_cnt + c);
        if (in) {
            p2p_list[(size_t)c * p2p_stride + i] = b;
            my_idx = i;
        }
    }
    if (w_list) {
        const bool wl = p2p && has_w && F.O.method == FAR_CHEB;
        i = warp_append(act, wl, w_cnt);
        if (wl) w_list[i] = cls * p2p_stride + my_idx;   // the leaf's slot in p2p_list
    }
}

void fmm_work_lists(const FmmDev &F, int nboxes, int *src_list, int *src_cnt, int *leaf_list, int *leaf_cnt,
                    int *p2p_list, int *p2p_cnt, int p2p_stride, int *own_list, int *own_cnt, cudaStream_t st,
                    int *w_list, int *w_cnt) {
    if (nboxes <= 0) return;
    launch_pdl(k_work_lists, (nboxes + 255) / 256, 256, 0, st, F, nboxes, src_list, src_cnt, leaf_list, leaf_cnt, p2p_list,
                                                       p2p_cnt, p2p_stride, own_list, own_cnt, w_list, w_cnt);
}

// ------------------------------------------------------------------ M2L (FP32 SIMT)
__global__ void __launch_bounds__(2 * MAXPAD) k_m2l_simt(FmmDev F, int level, int box_begin, int box_count) {
    pdl_enter();
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
    launch_pdl(k_m2l_simt, box_count, 2 * F.O.npad, 0, st, F, level, box_begin, box_count);
}

// ------------------------------------------------------------------ P2L (X list)
__global__ void __launch_bounds__(2 * MAXPAD) k_p2l(FmmDev F, int level, int box_begin, int box_count) {
    pdl_enter();
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
    launch_pdl(k_p2l, box_count, 2 * F.O.npad, 0, st, F, level, box_begin, box_count);
}

// ------------------------------------------------------------------ downward: L2L
__global__ void __launch_bounds__(2 * MAXPAD) k_down(FmmDev F, int level, int box_begin, int box_count) {
    pdl_enter();
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
    launch_pdl(k_down, box_count, 2 * F.O.npad, 0, st, F, level, box_begin, box_count);
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
    const bool l2p_done = F.leaf_l2p_done && cheb && level >= 2 && (F.O.e_off[level] >= 0 || F.l2p_sep);
    const bool do_u = !F.p2p_separate;
    const bool do_w = !(F.p2p_separate && cheb);     // the near-field kernel takes Chebyshev M2P
    if (l2p_done && (!do_u || F.L.u_off[b] == F.L.u_off[b + 1]) && (!do_w || F.L.w_off[b] == F.L.w_off[b + 1]))
        return;
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
        uint32_t tp = act ? key_pc(F.trg_key[t]) : 0u;
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
        for (int wv = F.L.w_off[b]; do_w && wv < F.L.w_off[b + 1]; ++wv) {
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
        for (int uv = F.L.u_off[b]; do_u && uv < F.L.u_off[b + 1]; ++uv) {
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
    pdl_enter();
    const int cnt = *count;
    for (int i = blockIdx.x; i < cnt; i += gridDim.x) {
        leaf_box(F, list[i], out);
        __syncthreads();
    }
}

// ---------------------------------------------------------------- L2P by tensor-product stages
// Chebyshev far field, leaves without an interpolation table (edge e > 16 cells): with the
// 1D Lagrange basis S_a(x) of the box's cell centres along each axis,
//     S(x, y, z) = sum_c S_c(z) sum_b S_b(y) sum_a S_a(x) d[a + p (b + p c)]
// is evaluated in three contractions held in shared memory: T1[c][b][x] (p^2 e), T2 for a
// band of Y rows, T2[c][y][x] (p Y e), then 5 (= p) multiply-adds per cell, written in
// coalesced x rows.  A box is split over CTAs by z slabs (grid.y).  Cells outside the
// grid are skipped; a partly selected box writes only where the target mask is set.
constexpr int SEP_SLAB = 16;
constexpr int SEP_T2_FLOATS = 16384;   // 64 KiB band of T2

__host__ int sep_band_rows(int p, int e) {
    int Y = SEP_T2_FLOATS / (p * e);
    return Y < 1 ? 1 : (Y > e ? e : Y);
}
size_t sep_smem_bytes(int p, int np, int e) {
    return sizeof(float) * ((size_t)np + (size_t)p * e + (size_t)p * p * e + (size_t)p * sep_band_rows(p, e) * e);
}

__global__ void __launch_bounds__(256) k_l2p_sep(FmmDev F, int level, const int *__restrict__ list,
                                                 const int *__restrict__ count, int band, float *__restrict__ out) {
    pdl_enter();
    const int box_count = *count;
    if ((int)blockIdx.x >= box_count) return;   // a CTA without a box of the list (see k_l2p_sep_small)
    extern __shared__ float sm[];
    const int p = F.O.order, n = F.O.n, np = F.O.npad;
    const int e = 1 << (F.D - level);
    float *sd = sm;                         // [np]
    float *Sb = sd + np;                    // [p][e]
    float *T1 = Sb + p * e;                 // [p*p][e]: (c, b) x
    float *T2 = T1 + p * p * e;             // [p][band][e]
    __shared__ float tch[8];
    const int tid = threadIdx.x;
    const int z0 = blockIdx.y * SEP_SLAB, z1 = min(e, z0 + SEP_SLAB);
    if (tid < p) tch[tid] = F.O.cheb_t[tid];
    for (int i = blockIdx.x; i < box_count; i += gridDim.x) {
        const int b = list[i];
        const TreeDev &T = F.T;
        if (!T.b_leaf[b] || T.b_te[b] <= T.b_tb[b] || z0 >= e) continue;   // uniform over the CTA
        const bool full = T.b_te[b] - T.b_tb[b] == e * e * e;
        uint32_t ux, uy, uz;
        demorton3(T.b_key[b], ux, uy, uz);
        const int bx = (int)ux * e, by = (int)uy * e, bz = (int)uz * e;
        __syncthreads();
        for (int j = tid; j < n; j += blockDim.x) sd[j] = F.dchk[(size_t)b * np + j];
        for (int j = tid; j < p * e; j += blockDim.x) {
            const int a = j / e, x = j % e;
            const float u = (float)(2 * x + 1 - e) / (float)e;
            float v = 1.f;
            for (int k = 0; k < p; ++k)
                if (k != a) v *= (u - tch[k]) / (tch[a] - tch[k]);
            Sb[j] = v;
        }
        __syncthreads();
        for (int j = tid; j < p * p * e; j += blockDim.x) {
            const int x = j % e, cb = j / e;
            const float *row = sd + p * cb;
            float acc = 0.f;
            for (int a = 0; a < p; ++a) acc = fmaf(row[a], Sb[a * e + x], acc);
            T1[j] = acc;
        }
        for (int y0 = 0; y0 < e; y0 += band) {
            const int ny = min(band, e - y0);
            __syncthreads();
            for (int j = tid; j < p * ny * e; j += blockDim.x) {
                const int x = j % e, yy = (j / e) % ny, c = j / (e * ny);
                float acc = 0.f;
                for (int bb = 0; bb < p; ++bb) acc = fmaf(T1[(c * p + bb) * e + x], Sb[bb * e + y0 + yy], acc);
                T2[(c * band + yy) * e + x] = acc;
            }
            __syncthreads();
            const int cells = (z1 - z0) * ny * e;
            for (int j = tid; j < cells; j += blockDim.x) {
                const int x = j % e, yy = (j / e) % ny, z = z0 + j / (e * ny);
                const int gx = bx + x, gy = by + y0 + yy, gz = bz + z;
                if (gx >= F.nx || gy >= F.ny || gz >= F.nz) continue;
                const int64_t o = (int64_t)gx + (int64_t)F.nx * ((int64_t)gy + (int64_t)F.ny * gz);
                if (!full && !F.tmask[o]) continue;
                float acc = 0.f;
                for (int c = 0; c < p; ++c) acc = fmaf(T2[(c * band + yy) * e + x], Sb[c * e + z], acc);
                out[o] = acc;
            }
        }
    }
}

// Small leaves (edge e <= 8): one warp per box, the same three contractions in the warp's own
// shared slots, outputs as float4 runs along x for whole boxes (e a multiple of 4 and x rows
// 16-byte aligned), per cell otherwise.
constexpr int SEPW_WARPS = 8;
constexpr int SEPW_MAXE = 8;
constexpr int SEPW_MAXP = 6;           // orders up to 6 (n <= 216, npad <= 224)
constexpr int SEPW_NP = 224;

__global__ void __launch_bounds__(SEPW_WARPS * 32) k_l2p_sep_small(FmmDev F, int level, const int *__restrict__ list,
                                                                   const int *__restrict__ count,
                                                                   float *__restrict__ out) {
    pdl_enter();
    const int box_count = *count;
    // the launch is sized by the level's box count; the leaves with targets are often far fewer
    // (none at all on a level above a fused deepest one): CTAs without a box leave before the
    // basis set-up
    if ((int)blockIdx.x * SEPW_WARPS >= box_count) return;
    __shared__ float Sb[SEPW_MAXP * SEPW_MAXE];                                  // [p][e]
    __shared__ __align__(16) float sd[SEPW_WARPS][SEPW_NP];
    __shared__ float T1[SEPW_WARPS][SEPW_MAXP * SEPW_MAXP * SEPW_MAXE];          // [p*p][e]
    __shared__ float T2[SEPW_WARPS][SEPW_MAXP * SEPW_MAXE * SEPW_MAXE];          // [p][e][e]
    __shared__ float tch[8];
    const int p = F.O.order, n = F.O.n, np = F.O.npad;
    const int e = 1 << (F.D - level);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x < p) tch[threadIdx.x] = F.O.cheb_t[threadIdx.x];
    __syncthreads();
    for (int j = threadIdx.x; j < p * e; j += blockDim.x) {
        const int a = j / e, x = j % e;
        const float u = (float)(2 * x + 1 - e) / (float)e;
        float v = 1.f;
        for (int k = 0; k < p; ++k)
            if (k != a) v *= (u - tch[k]) / (tch[a] - tch[k]);
        Sb[j] = v;
    }
    __syncthreads();
    const TreeDev &T = F.T;
    const bool rows4 = (e % 4) == 0 && (F.nx % 4) == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0;
    int le = 0;
    while ((1 << le) < e) ++le;
    const int em = e - 1;
    float *d = sd[warp], *t1 = T1[warp], *t2 = T2[warp];
    // the next box's d is fetched into registers while the current box is evaluated
    const int stride = gridDim.x * SEPW_WARPS;
    int i = blockIdx.x * SEPW_WARPS + warp;
    float4 nd[2];
    auto fetch = [&](int ii, float4 *r) {
        if (ii < box_count) {
            const float *src = F.dchk + (size_t)list[ii] * np;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int j = 4 * lane + 128 * k;
                r[k] = j < np ? __ldg(reinterpret_cast<const float4 *>(src + j)) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
    };
    fetch(i, nd);
    for (; i < box_count; i += stride) {
        const int b = list[i];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int j = 4 * lane + 128 * k;
            if (j < np) *reinterpret_cast<float4 *>(d + j) = nd[k];
        }
        fetch(i + stride, nd);
        const bool use = T.b_leaf[b] && T.b_te[b] > T.b_tb[b];
        const bool full = use && T.b_te[b] - T.b_tb[b] == e * e * e;
        uint32_t ux, uy, uz;
        demorton3(T.b_key[b], ux, uy, uz);
        const int bx = (int)ux * e, by = (int)uy * e, bz = (int)uz * e;
        __syncwarp();
        if (use) {
            for (int j = lane; j < p * p * e; j += 32) {
                const int x = j & em, cb = j >> le;
                const float *row = d + p * cb;
                float acc = 0.f;
                for (int a = 0; a < p; ++a) acc = fmaf(row[a], Sb[a * e + x], acc);
                t1[j] = acc;
            }
            __syncwarp();
            for (int j = lane; j < p * e * e; j += 32) {
                const int x = j & em, y = (j >> le) & em, c = j >> (2 * le);
                float acc = 0.f;
                for (int bb = 0; bb < p; ++bb) acc = fmaf(t1[(c * p + bb) * e + x], Sb[bb * e + y], acc);
                t2[j] = acc;
            }
            __syncwarp();
            if (full && rows4) {
                for (int r = lane; r < (e * e * e) >> 2; r += 32) {
                    const int c4 = r << 2;
                    const int x = c4 & em, y = (c4 >> le) & em, z = c4 >> (2 * le);
                    float v[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        float acc = 0.f;
                        for (int c = 0; c < p; ++c) acc = fmaf(t2[(c * e + y) * e + x + u], Sb[c * e + z], acc);
                        v[u] = acc;
                    }
                    const int64_t o =
                        (int64_t)(bx + x) + (int64_t)F.nx * ((int64_t)(by + y) + (int64_t)F.ny * (bz + z));
                    *reinterpret_cast<float4 *>(out + o) = make_float4(v[0], v[1], v[2], v[3]);
                }
            } else {
                // the mask bytes of this lane's cells (at most 16: e <= 8) first, then the sums and
                // stores (a byte load placed after a float store would wait for it)
                uint32_t keep = 0;
                for (int j = lane, it = 0; j < e * e * e; j += 32, ++it) {
                    const int gx = bx + (j & em), gy = by + ((j >> le) & em), gz = bz + (j >> (2 * le));
                    if (gx >= F.nx || gy >= F.ny || gz >= F.nz) continue;
                    const int64_t o = (int64_t)gx + (int64_t)F.nx * ((int64_t)gy + (int64_t)F.ny * gz);
                    if (full || __ldg(F.tmask + o)) keep |= 1u << it;
                }
                for (int j = lane, it = 0; j < e * e * e; j += 32, ++it) {
                    if (!((keep >> it) & 1u)) continue;
                    const int x = j & em, y = (j >> le) & em, z = j >> (2 * le);
                    const int64_t o = (int64_t)(bx + x) + (int64_t)F.nx * ((int64_t)(by + y) + (int64_t)F.ny * (bz + z));
                    float acc = 0.f;
                    for (int c = 0; c < p; ++c) acc = fmaf(t2[(c * e + y) * e + x], Sb[c * e + z], acc);
                    out[o] = acc;
                }
            }
        }
        __syncwarp();
    }
    (void)n;
}

void fmm_l2p_sep_level(const FmmDev &F, int level, const int *list, const int *count, int box_count, float *out,
                       cudaStream_t st) {
    if (box_count <= 0 || level < 2) return;
    if ((1 << (F.D - level)) <= SEPW_MAXE && F.O.order <= SEPW_MAXP && F.O.npad <= SEPW_NP) {
        const int per = SEPW_WARPS;
        int grid = (box_count + per - 1) / per;
        if (grid > 152 * 8) grid = 152 * 8;
        launch_pdl(k_l2p_sep_small, grid, SEPW_WARPS * 32, 0, st, F, level, list, count, out);
        return;
    }
    const int e = 1 << (F.D - level), p = F.O.order;
    const int band = sep_band_rows(p, e);
    const size_t smem = sep_smem_bytes(p, F.O.npad, e);
    const int zs = (e + SEP_SLAB - 1) / SEP_SLAB;
    int gx = box_count < 152 * 4 ? box_count : 152 * 4;
    launch_pdl(k_l2p_sep, dim3(gx, zs), 256, smem, st, F, level, list, count, band, out);
}

// Shared-memory opt-in of the FMM kernels that may need more than 48 KiB (host, once, before
// any launch that could be captured into a graph).  k_l2p_sep needs at most
// 4 * (512 + 8 * 256 + 64 * 256 + 16384) bytes = 141 KiB (order <= 8, edge <= 256).
void fmm_init_attributes() {
    static bool done = false;
    if (done) return;
    cudaFuncSetAttribute(k_l2p_sep, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    done = true;
}

// ---------------------------------------------------------------- near field (U and W lists), warp-tiled
// One CTA (4 warps) per leaf of the list.  Point sources are staged in shared memory in
// rounds of up to P2P_CAP: the sources of the leaf's U-list boxes (P2P, Eq. nearfar), then the
// Chebyshev nodes of its W-list boxes with their upward weights (M2P).  A staged point holds
// its position in cell units (cell (i, j, k) at (i, j, k)) and its weight pre-multiplied by
// C / h^3, so that with s = |offset| in cells
//     G(R) * w = w' e^{-alpha h s} (1 - e^{-(beta - alpha) h s}) / s^3.
// A warp owns 32 of the leaf's targets (one per lane) and a share of the staged points,
// read with broadcast loads.  Small leaves (one or two chunks of 32 targets) split the points
// across 4 or 2 warps; every target's sum is added once per warp.  TAYLOR = false when
// (beta - alpha) h >= 0.5: then 1 - e^{-x} needs no series at any distance >= 1 cell.
constexpr int P2P_WARPS = 4;
constexpr int P2P_CAP = 1536;        // staged points per round (24 KiB)
constexpr int P2P_MAXU = 128;        // list entries handled per pass over the box table

struct P2PConst {
    float k1, k2;        // alpha h log2(e), (beta - alpha) h log2(e)
    float bma_h;         // (beta - alpha) h
    float wself;         // G_self h^3 / C  (self term, in the scaled weight units)
    float k12;           // k1 + k2 = beta h log2(e)
};

// the scaled kernel g(s^2) of the near-field sum (see above); d2 >= 1 (distinct cells, or a
// node of a non-adjacent box).  Where (beta - alpha) h >= 1/2 the factor 1 - e^{-(beta-alpha) s}
// is at least 0.29, and e^{-alpha s} - e^{-beta s} is formed directly (no cancellation to fear).
template <bool TAYLOR>
__device__ __forceinline__ float p2p_g(float d2, const P2PConst &K) {
    const float rs = rsqrt_approx(d2);
    const float sdist = d2 * rs;
    const float diff = TAYLOR ? ex2_approx(-K.k1 * sdist) * one_minus_exp_neg(K.bma_h * sdist, K.k2 * sdist)
                              : ex2_approx(-K.k1 * sdist) - ex2_approx(-K.k12 * sdist);
    return diff * (rs * rs * rs);
}

// TABLE: the offsets of point sources are integers; g is read from the shared-memory table
// for d2 < GTAB_N (values computed by p2p_g itself, so the sums are the same).
// SELF: the range may hold the target's own cell (d2 = 0: the self term); otherwise every
// source lies in another cell.
template <bool TAYLOR, bool TABLE, bool SELF = false>
__device__ __forceinline__ float p2p_sum(const float4 *__restrict__ pts, int lo, int hi, float tx, float ty,
                                         float tz, const P2PConst &K, const float *__restrict__ tab) {
    float a = 0.f;
#pragma unroll 4
    for (int j = lo; j < hi; ++j) {
        const float4 sp = pts[j];
        const float dx = tx - sp.x, dy = ty - sp.y, dz = tz - sp.z;
        const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        float g;
        if (TABLE) {
            const int di = (int)d2;
            g = di < GTAB_N ? tab[di] : p2p_g<TAYLOR>(d2, K);
        } else if (SELF) {
            const float gv = p2p_g<TAYLOR>(fmaxf(d2, 1.f), K);   // computed for every pair, then selected
            g = d2 > 0.f ? gv : K.wself;
        } else {
            g = p2p_g<TAYLOR>(d2, K);
        }
        a = fmaf(g, sp.w, a);
    }
    return a;
}

template <bool TAYLOR>
__global__ void k_near_table(P2PConst K, float *tab) {
    pdl_enter();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < GTAB_N) tab[i] = i == 0 ? K.wself : p2p_g<TAYLOR>((float)i, K);
}

// list: P2P_CLASSES lists of `stride` slots, count: their lengths; the leaves are taken class
// by class, the heaviest first.  Passes [pass_lo, pass_hi) of 0 (U list) and 1 (W list); a
// launch of pass 1 alone skips the leaves without W entries and adds to the slots that the
// pass-0 launch cleared.
template <bool TAYLOR, bool TABLE>
__global__ void __launch_bounds__(P2P_WARPS * 32) k_p2p(FmmDev F, const int *__restrict__ list,
                                                         const int *__restrict__ count, int stride,
                                                         float *__restrict__ out, P2PConst K, int pass_lo,
                                                         int pass_hi, const int *__restrict__ w_list,
                                                         const int *__restrict__ w_cnt) {
    pdl_enter();
    __shared__ float4 stage[P2P_CAP];
    __shared__ float tab[TABLE ? GTAB_N : 1];
    __shared__ int4 ubox[P2P_MAXU];        // W boxes: lowest cell corner, edge (strategy 3)
    __shared__ float uwt[P2P_MAXU];        // W boxes: total scaled weight
    __shared__ float usum[P2P_WARPS * 2][32];   // U-list sums per (chunk, lane) (strategy 3)
    if (TABLE)
        for (int j = threadIdx.x; j < GTAB_N; j += blockDim.x) tab[j] = F.gtab[j];
    __shared__ int ub[P2P_MAXU], un[P2P_MAXU], uo[P2P_MAXU + 1];
    __shared__ int s_own;                  // entry of the leaf itself in the staged U list, or -1
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    __shared__ int ccnt[P2P_CLASSES];
    if (tid < P2P_CLASSES) ccnt[tid] = count[tid];
    __syncthreads();
    int cnt = 0;
#pragma unroll
    for (int c = 0; c < P2P_CLASSES; ++c) cnt += ccnt[c];
    // a W-only launch with the list of the leaves that have W entries walks those alone
    const int nitems = w_list ? *w_cnt : cnt;
    const TreeDev &T = F.T;
    const float h = F.kp.h;
    const float wsc = F.wscale * F.kp.C / (h * h * h);          // source weight -> scaled weight
    const float usc = F.kp.C / (h * h * h);                     // upward weight -> scaled weight
    const int n = F.O.n, np = F.O.npad;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        int c = 0, j = it, i = it;
        if (w_list) {
            // slot in the class lists -> (class, index in the class) -> position i in the class order
            const int e = w_list[it];
            c = e / stride;
            j = e - c * stride;
            i = j;
            for (int k = 0; k < c; ++k) i += ccnt[k];
        } else {
            while (c < P2P_CLASSES - 1 && j >= ccnt[c]) j -= ccnt[c++];
        }
        const int b = list[(size_t)c * stride + j];
        if (pass_lo == 1 && F.L.w_off[b + 1] == F.L.w_off[b]) continue;     // uniform
        const int tb = T.b_tb[b], te = T.b_te[b];
        const int nch = (te - tb + 31) >> 5;
        // the leaf's sums: its slots of the scratch (cleared by the launch that starts with the
        // U list), or the output itself
        float *nslot = F.near_buf ? F.near_buf + (size_t)i * F.near_s : nullptr;
        if (nslot && pass_lo == 0) {
            for (int t = tid; t < te - tb; t += blockDim.x) nslot[t] = 0.f;
            __syncthreads();
        }
        auto add_out = [&](int t, uint32_t tp, float v) {
            if (nslot) atomicAdd(nslot + (t - tb), v);
            else atomicAdd(out + (int64_t)pc_i(tp) + (int64_t)F.nx * ((int64_t)pc_j(tp) + (int64_t)F.ny * pc_k(tp)), v);
        };
        const int G = nch >= P2P_WARPS ? 1 : P2P_WARPS / nch;     // warps sharing a target chunk
        const int groups = P2P_WARPS / G;
        const int k = warp % G;
        float acc[2] = {0.f, 0.f};        // the first two chunks of this warp; further chunks flush per round
        // pass 0: U list (point sources); pass 1: W list (Chebyshev nodes of the W boxes)
        const int passes = min(pass_hi, F.O.method == FAR_CHEB ? 2 : 1);   // the surface form keeps M2P in k_leaf
        // strategy 3 applies to leaves whose every chunk stays in this warp's two sum slots
        const bool skip3 = F.r_s > 0.f && nch <= 2 * groups && F.L.w_off[b + 1] > F.L.w_off[b];
        float sest[2] = {0.f, 0.f};
        for (int pass = pass_lo; pass < passes; ++pass) {
            const int l0 = pass == 0 ? F.L.u_off[b] : F.L.w_off[b];
            const int l1 = pass == 0 ? F.L.u_off[b + 1] : F.L.w_off[b + 1];
            if (pass == 1 && skip3) {
                // S_est = far field already in out (L2P) + the leaf's whole U-list sum
                __syncthreads();
                for (int j = tid; j < P2P_WARPS * 2 * 32; j += blockDim.x) (&usum[0][0])[j] = 0.f;
                __syncthreads();
                int sl = 0;
                for (int c = warp / G; c < nch && sl < 2; c += groups, ++sl) atomicAdd(&usum[c][lane], acc[sl]);
                __syncthreads();
                sl = 0;
                for (int c = warp / G; c < nch && sl < 2; c += groups, ++sl) {
                    const int t = tb + c * 32 + lane;
                    float far = 0.f;
                    if (t < te) {
                        const uint32_t tp = key_pc(F.trg_key[t]);
                        far = out[(int64_t)pc_i(tp) + (int64_t)F.nx * ((int64_t)pc_j(tp) + (int64_t)F.ny * pc_k(tp))];
                    }
                    sest[sl] = far + usum[c][lane];
                }
            }
            for (int ub0 = l0; ub0 < l1; ub0 += P2P_MAXU) {
                const int nu = min(P2P_MAXU, l1 - ub0);
                __syncthreads();
                if (tid == 0) s_own = -1;
                __syncthreads();
                if (tid < nu) {
                    const int A = pass == 0 ? F.L.u_src[ub0 + tid] : F.L.w_src[ub0 + tid];
                    if (pass == 0 && A == b) s_own = tid;
                    if (pass == 0) {
                        const int sb = T.b_sb[A];
                        ub[tid] = sb;
                        un[tid] = T.b_se[A] - sb;
                    } else {
                        ub[tid] = A;
                        un[tid] = n;
                        if (F.r_s > 0.f) {
                            const int asz = 1 << (F.D - T.b_level[A]);
                            uint32_t ax, ay, az;
                            demorton3(T.b_key[A], ax, ay, az);
                            ubox[tid] = make_int4((int)ax * asz, (int)ay * asz, (int)az * asz, asz);
                            float wsum = 0.f;
                            for (int m = 0; m < n; ++m) wsum += F.ueq[(size_t)A * np + m];
                            uwt[tid] = wsum * usc;
                        }
                    }
                }
                __syncthreads();
                if (tid == 0) {
                    int o = 0;
                    for (int j = 0; j < nu; ++j) {
                        uo[j] = o;
                        o += un[j];
                    }
                    uo[nu] = o;
                }
                __syncthreads();
                const int total = uo[nu];
                for (int r0 = 0; r0 < total; r0 += P2P_CAP) {
                    const int rn = min(P2P_CAP, total - r0);
                    __syncthreads();
                    for (int j = 0; j < nu; ++j) {
                        const int lo = max(uo[j], r0), hi = min(uo[j + 1], r0 + rn);
                        if (lo >= hi) continue;
                        if (pass == 0) {
                            for (int s = lo + tid; s < hi; s += blockDim.x) {
                                const int si = ub[j] + (s - uo[j]);
                                const uint32_t pc = __ldg(F.src_pc + si);
                                stage[s - r0] = make_float4((float)pc_i(pc), (float)pc_j(pc), (float)pc_k(pc),
                                                            __ldg(F.src_q + si) * wsc);
                            }
                        } else {
                            const int A = ub[j];
                            const int asz = 1 << (F.D - T.b_level[A]);
                            uint32_t ax, ay, az;
                            demorton3(T.b_key[A], ax, ay, az);
                            const float half = 0.5f * (float)asz;
                            const float cx = (float)ax * asz + half - 0.5f, cy = (float)ay * asz + half - 0.5f,
                                        cz = (float)az * asz + half - 0.5f;
                            for (int s = lo + tid; s < hi; s += blockDim.x) {
                                const int m = s - uo[j];
                                stage[s - r0] = make_float4(cx + half * F.O.nodes[4 * m], cy + half * F.O.nodes[4 * m + 1],
                                                            cz + half * F.O.nodes[4 * m + 2],
                                                            F.ueq[(size_t)A * np + m] * usc);
                            }
                        }
                    }
                    __syncthreads();
                    const int per = (rn + G - 1) / G;
                    const int s_lo = k * per, s_hi = min(rn, s_lo + per);
                    int slot = 0;
                    for (int c = warp / G; c < nch; c += groups, ++slot) {
                        const int t = tb + c * 32 + lane;
                        const uint32_t tp = t < te ? key_pc(F.trg_key[t]) : 0u;
                        if (pass == 1 && skip3) {
                            // W box by W box: a lane drops box j when G(d_min) * sum(I_h) < r_s * S_est
                            const int tx = pc_i(tp), ty = pc_j(tp), tz = pc_k(tp);
                            float a = 0.f;
                            unsigned long long skipped = 0;
                            for (int j = 0; j < nu; ++j) {
                                const int lo = max(uo[j] - r0, s_lo), hi = min(uo[j + 1] - r0, s_hi);
                                if (lo >= hi) continue;
                                const int4 bx = ubox[j];
                                const int ex = max(0, max(bx.x - tx, tx - (bx.x + bx.w - 1)));
                                const int ey = max(0, max(bx.y - ty, ty - (bx.y + bx.w - 1)));
                                const int ez = max(0, max(bx.z - tz, tz - (bx.z + bx.w - 1)));
                                const float d2 = (float)(ex * ex + ey * ey + ez * ez);
                                const bool drop = t < te && p2p_g<TAYLOR>(fmaxf(d2, 1.f), K) * uwt[j] <
                                                                 F.r_s * sest[slot < 2 ? slot : 1];
                                skipped += drop;
                                if (__all_sync(0xffffffffu, drop || t >= te)) continue;
                                const float part = p2p_sum<TAYLOR, false>(stage, lo, hi, (float)tx, (float)ty,
                                                                          (float)tz, K, tab);
                                if (!drop) a += part;
                            }
                            if (skipped && F.skip_count) atomicAdd(F.skip_count, skipped);
                            if (slot < 2) acc[slot] += a;
                            else if (t < te) add_out(t, tp, a);
                            continue;
                        }
                        // W-list nodes (pass 1) sit off the lattice: the exp form
                        float a;
                        if (TABLE && pass == 0)
                            a = p2p_sum<TAYLOR, true>(stage, s_lo, s_hi, (float)pc_i(tp), (float)pc_j(tp),
                                                      (float)pc_k(tp), K, tab);
                        else {
                            // only the leaf's own cells can be the target's cell: the self-term
                            // select runs there alone
                            const float fx = (float)pc_i(tp), fy = (float)pc_j(tp), fz = (float)pc_k(tp);
                            const int own = pass == 0 ? s_own : -1;
                            const int olo = own >= 0 ? max(uo[own] - r0, s_lo) : s_hi;
                            const int ohi = own >= 0 ? min(uo[own + 1] - r0, s_hi) : s_hi;
                            if (olo < ohi)
                                a = p2p_sum<TAYLOR, false>(stage, s_lo, olo, fx, fy, fz, K, tab) +
                                    p2p_sum<TAYLOR, false, true>(stage, olo, ohi, fx, fy, fz, K, tab) +
                                    p2p_sum<TAYLOR, false>(stage, ohi, s_hi, fx, fy, fz, K, tab);
                            else
                                a = p2p_sum<TAYLOR, false>(stage, s_lo, s_hi, fx, fy, fz, K, tab);
                        }
                        if (slot < 2) acc[slot] += a;
                        else if (t < te) add_out(t, tp, a);
                    }
                }
            }
        }
        int slot = 0;
        for (int c = warp / G; c < nch && slot < 2; c += groups, ++slot) {
            const int t = tb + c * 32 + lane;
            if (t >= te) continue;
            add_out(t, nslot ? 0u : key_pc(F.trg_key[t]), acc[slot]);
        }
    }
}

// out[cell of t] += near_buf[slot of t]: one warp per leaf of the class lists (the items in the
// near field's order); every target belongs to one leaf, so plain read-modify-writes suffice
__global__ void __launch_bounds__(256) k_near_add(FmmDev F, const int *__restrict__ list,
                                                  const int *__restrict__ count, int stride,
                                                  float *__restrict__ out, const int *__restrict__ flags,
                                                  int *flags_host) {
    pdl_enter();
    if (flags_host && blockIdx.x == 0 && threadIdx.x < 2) {
        flags_host[threadIdx.x] = flags[threadIdx.x];
        __threadfence_system();
    }
    int cnt = 0;
#pragma unroll
    for (int c = 0; c < P2P_CLASSES; ++c) cnt += count[c];
    const int lane = threadIdx.x & 31;
    const int nw = (int)((gridDim.x * blockDim.x) >> 5);
    for (int i = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); i < cnt; i += nw) {
        int c = 0, j = i;
        while (c < P2P_CLASSES - 1 && j >= count[c]) j -= count[c++];
        const int b = list[(size_t)c * stride + j];
        const int tb = F.T.b_tb[b], te = F.T.b_te[b];
        const float *ns = F.near_buf + (size_t)i * F.near_s;
        for (int t = tb + lane; t < te; t += 32) {
            const uint32_t tp = key_pc(F.trg_key[t]);
            out[(int64_t)pc_i(tp) + (int64_t)F.nx * ((int64_t)pc_j(tp) + (int64_t)F.ny * pc_k(tp))] += ns[t - tb];
        }
    }
}

static P2PConst p2p_const(const FmmDev &F) {
    P2PConst K;
    const float h = F.kp.h;
    K.k1 = F.kp.a2 * h;                       // a2 = alpha log2(e)
    K.k2 = F.kp.b2 * h;                       // b2 = (beta - alpha) log2(e)
    K.bma_h = F.kp.bma * h;
    K.k12 = K.k1 + K.k2;
    // the self weight multiplies the scaled weight w' = w C / h^3: g_self w = (g_self h^3 / C) w'
    K.wself = F.self_mode ? F.kp.gself * h * h * h / F.kp.C : 0.f;
    return K;
}

void fmm_near_table(const FmmDev &F, float *gtab, cudaStream_t st) {
    const P2PConst K = p2p_const(F);
    if (K.bma_h >= 0.5f) launch_pdl(k_near_table<false>, (GTAB_N + 255) / 256, 256, 0, st, K, gtab);
    else launch_pdl(k_near_table<true>, (GTAB_N + 255) / 256, 256, 0, st, K, gtab);
}

void fmm_p2p(const FmmDev &F, int nboxes, const int *p2p_list, const int *p2p_cnt, int stride, float *out,
             cudaStream_t st, int pass_lo, int pass_hi, int per_sm, const int *w_list, const int *w_cnt, int max_w) {
    if (nboxes <= 0) return;
    const int cap = 152 * per_sm;
    int grid = nboxes < cap ? nboxes : cap;
    if (w_list) {
        if (pass_lo != 1 || max_w <= 0) return;      // the list serves a W-only launch; no W entries
        grid = std::min(grid, max_w);
    }
    const P2PConst K = p2p_const(F);
    const bool taylor = K.bma_h < 0.5f, table = F.gtab != nullptr;
    if (!taylor && !table)
        launch_pdl(k_p2p<false, false>, grid, P2P_WARPS * 32, 0, st, F, p2p_list, p2p_cnt, stride, out, K, pass_lo,
                   pass_hi, w_list, w_cnt);
    else if (taylor && !table)
        launch_pdl(k_p2p<true, false>, grid, P2P_WARPS * 32, 0, st, F, p2p_list, p2p_cnt, stride, out, K, pass_lo,
                   pass_hi, w_list, w_cnt);
    else if (!taylor)
        launch_pdl(k_p2p<false, true>, grid, P2P_WARPS * 32, 0, st, F, p2p_list, p2p_cnt, stride, out, K, pass_lo,
                   pass_hi, w_list, w_cnt);
    else
        launch_pdl(k_p2p<true, true>, grid, P2P_WARPS * 32, 0, st, F, p2p_list, p2p_cnt, stride, out, K, pass_lo,
                   pass_hi, w_list, w_cnt);
}

void fmm_near_add(const FmmDev &F, int nboxes, const int *p2p_list, const int *p2p_cnt, int stride, float *out,
                  cudaStream_t st,
                  const int *flags, int *flags_host) {
    if (nboxes <= 0 || !F.near_buf) return;
    const int grid = std::max(1, std::min((nboxes + 7) / 8, 152 * 8));
    launch_pdl(k_near_add, grid, 256, 0, st, F, p2p_list, p2p_cnt, stride, out, flags, flags_host);
}

void fmm_leaf(const FmmDev &F, int nboxes, const int *list, const int *count, float *out_dense, cudaStream_t st) {
    if (nboxes <= 0) return;
    int grid = nboxes < 152 * 16 ? nboxes : 152 * 16;
    launch_pdl(k_leaf, grid, LT, 0, st, F, list, count, out_dense);
}

}  // namespace sph
