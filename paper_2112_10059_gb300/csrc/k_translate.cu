// Far-field translations as batched, gathered GEMMs (FP32 SIMT, register tiled).
//
// M2L (paper Section 2.4, far interactions through the hierarchy): for a tile
// of 64 consecutive target boxes B of one level and every one of the 316
// offsets o, the rows u_A of the source boxes A = B + o that lie in V(B) are
// gathered (zero where there is none) and multiplied by the level's M2L_o:
//     d_B += sum_o M2L_o u_{B+o}
// so each operator is read once per tile instead of once per box pair.  V(B)
// membership is recomputed from the dense level array: A exists, holds
// sources, and the parents of A and B are adjacent (|o|_inf >= 2 always).
//
// L2L: for a tile of 64 parent boxes P of level l-1 and one child slot c,
//     d_{child c of P} += L2L_c d_P.
//
// Tiling: CTA = 256 threads computes 128 operator rows x 64 boxes; thread
// (ty, tx) holds 8 rows x 4 boxes of FP32 accumulators; the K dimension (the
// operator columns) streams through shared memory 16 at a time.  Operators
// are stored transposed ([k][i], row stride npad), so an operator K-slab is a
// contiguous, coalesced read.
#include "sph_kernels.cuh"

namespace sph {

constexpr int TM = 128, TN = 64, TK = 16;

// thread (ty, tx) owns operator rows ty*8 .. ty*8+7 and tile columns tx*4 .. tx*4+3
__device__ __forceinline__ void mma_tile(const float (*As)[TM], const float (*Bs)[TN], int ty, int tx,
                                         float acc[8][4]) {
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
        const float4 a0 = *reinterpret_cast<const float4 *>(&As[kk][ty * 8]);
        const float4 a1 = *reinterpret_cast<const float4 *>(&As[kk][ty * 8 + 4]);
        const float4 bv = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
        const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float b[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) acc[r][cc] = fmaf(a[r], b[cc], acc[r][cc]);
    }
}

// acc += Op[i0.., :] * X[:, cols]: Op transposed [k][i] with row stride ldA and M valid rows,
// K = np; X columns = state rows src[col] (row stride np).
__device__ __forceinline__ void gemm_slab_g(const float *__restrict__ opT, int ldA, int M, int np, int i0,
                                            const float *__restrict__ state, const int *src, float (*As)[TM],
                                            float (*Bs)[TN], float acc[8][4]) {
    const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
    for (int k0 = 0; k0 < np; k0 += TK) {
        for (int e = tid; e < TK * TM; e += 256) {
            int kk = e / TM, ii = e % TM;
            int i = i0 + ii;
            As[kk][ii] = i < M ? __ldg(opT + (size_t)(k0 + kk) * ldA + i) : 0.f;
        }
        for (int e = tid; e < TK * TN; e += 256) {
            int c = e / TK, kk = e % TK;
            int s = src[c];
            Bs[kk][c] = s >= 0 ? state[(size_t)s * np + k0 + kk] : 0.f;
        }
        __syncthreads();
        mma_tile(As, Bs, ty, tx, acc);
        __syncthreads();
    }
}

__device__ __forceinline__ void gemm_slab(const float *__restrict__ opT, int np, int i0,
                                          const float *__restrict__ state, const int *src, float (*As)[TM],
                                          float (*Bs)[TN], float acc[8][4]) {
    gemm_slab_g(opT, np, np, np, i0, state, src, As, Bs, acc);
}

__device__ __forceinline__ void scatter_atomic(float *__restrict__ out, int np, int n, int i0, const int *dst,
                                               const float acc[8][4]) {
    const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
        int d = dst[tx * 4 + cc];
        if (d < 0) continue;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            int i = i0 + ty * 8 + r;
            if (i < n) atomicAdd(out + (size_t)d * np + i, acc[r][cc]);
        }
    }
}

__device__ __forceinline__ void scatter_add(float *__restrict__ out, int np, int n, int i0, const int *dst,
                                            const float acc[8][4]) {
    const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
        int d = dst[tx * 4 + cc];
        if (d < 0) continue;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            int i = i0 + ty * 8 + r;
            if (i < n) atomicAdd(out + (size_t)d * np + i, acc[r][cc]);   // reduction: no dependent load
        }
    }
}

// ---------------------------------------------------------------- M2L
__global__ void __launch_bounds__(256) k_m2l_gemm(FmmDev F, int level, int box_begin, int box_count) {
    pdl_enter();
    __shared__ __align__(16) float As[TK][TM];
    __shared__ __align__(16) float Bs[TK][TN];
    __shared__ int trg[TN], src[TN];
    __shared__ int tco[TN][3];
    const int tid = threadIdx.x;
    const int np = F.O.npad, n = F.O.n;
    const int t0 = blockIdx.x * TN;
    const int i0 = blockIdx.y * TM;
    const TreeDev &T = F.T;
    // early exit when no box of the tile has a V list
    int first = box_begin + t0, last = box_begin + min(t0 + TN, box_count);
    if (F.L.v_off[first] == F.L.v_off[last]) return;
    if (tid < TN) {
        int b = box_begin + t0 + tid;
        int ok = (t0 + tid < box_count) && (T.b_te[b] > T.b_tb[b]);
        trg[tid] = ok ? b : -1;
        uint32_t x = 0, y = 0, z = 0;
        if (ok) demorton3(T.b_key[b], x, y, z);
        tco[tid][0] = x; tco[tid][1] = y; tco[tid][2] = z;
    }
    __syncthreads();
    const int nside = 1 << level;
    const int *bat = T.box_at + dense_off(level);
    const float *Mlev = F.O.m2l_t + (size_t)level * NSLOT * np * np;
    float acc[8][4];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) acc[r][cc] = 0.f;
    int slot = 0;
    for (int code = 0; code < SPH_NOFF; ++code) {
        const int ox = code % 7 - 3, oy = (code / 7) % 7 - 3, oz = code / 49 - 3;
        if (abs(ox) <= 1 && abs(oy) <= 1 && abs(oz) <= 1) continue;   // uniform: same for all threads
        int found = 0;
        if (tid < TN) {
            int a = -1;
            if (trg[tid] >= 0) {
                int bx = tco[tid][0], by = tco[tid][1], bz = tco[tid][2];
                int ax = bx + ox, ay = by + oy, az = bz + oz;
                bool in = ax >= 0 && ay >= 0 && az >= 0 && ax < nside && ay < nside && az < nside;
                bool padj = abs((ax >> 1) - (bx >> 1)) <= 1 && abs((ay >> 1) - (by >> 1)) <= 1 &&
                            abs((az >> 1) - (bz >> 1)) <= 1;
                if (in && padj) {
                    int A = bat[morton3(ax, ay, az)];
                    if (A >= 0 && T.b_se[A] > T.b_sb[A]) a = A;
                }
            }
            src[tid] = a;
            found = a >= 0;
        }
        if (__syncthreads_or(found)) gemm_slab(Mlev + (size_t)slot * np * np, np, i0, F.ueq, src, As, Bs, acc);
        ++slot;
    }
    scatter_add(F.dchk, np, n, i0, trg, acc);
}

// ---------------------------------------------------------------- L2L
__global__ void __launch_bounds__(256) k_l2l_gemm(FmmDev F, int level, int parent_begin, int parent_count) {
    pdl_enter();
    __shared__ __align__(16) float As[TK][TM];
    __shared__ __align__(16) float Bs[TK][TN];
    __shared__ int par[TN], dst[TN];
    const int tid = threadIdx.x;
    const int np = F.O.npad, n = F.O.n;
    const int t0 = blockIdx.x * TN;
    const int i0 = blockIdx.y * TM;
    const int c = blockIdx.z;
    const TreeDev &T = F.T;
    int any = 0;
    if (tid < TN) {
        int p = parent_begin + t0 + tid;
        int P = -1, C = -1;
        if (t0 + tid < parent_count && !T.b_leaf[p] && T.b_te[p] > T.b_tb[p]) {
            int ch = T.box_at[dense_off(level) + ((T.b_key[p] << 3) | (uint32_t)c)];
            if (ch >= 0 && T.b_te[ch] > T.b_tb[ch]) { P = p; C = ch; }
        }
        par[tid] = P;
        dst[tid] = C;
        any = C >= 0;
    }
    if (!__syncthreads_or(any)) return;
    float acc[8][4];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) acc[r][cc] = 0.f;
    gemm_slab(F.O.l2l_t + ((size_t)level * 8 + c) * np * np, np, i0, F.dchk, par, As, Bs, acc);
    scatter_add(F.dchk, np, n, i0, dst, acc);
}

// ---------------------------------------------------------------- V pairs grouped by offset
// key = level * 316 + slot.  The list kernels count the pairs per key, k_lists_layout (k_tree.cu)
// scans the counts and cuts every key's range into tiles of VPAIR_TILE pairs, and the list fill
// places every pair in its key's range (any order within a key) and writes the key of every tile.


// One CTA per tile of up to 64 V pairs sharing (level, offset): d_B += M2L_{l,o} u_A, scatter-added.
__global__ void __launch_bounds__(256) k_m2l_pairs(FmmDev F, PairsDev Pd) {
    pdl_enter();
    __shared__ __align__(16) float As[TK][TM];
    __shared__ __align__(16) float Bs[TK][TN];
    __shared__ int trg[TN], src[TN];
    __shared__ int s_key;
    const int tid = threadIdx.x;
    const int np = F.O.npad, n = F.O.n;
    const int tile = blockIdx.x;
    if (tile >= Pd.tile_off[Pd.nkeys]) return;
    if (tid == 0) s_key = Pd.tile_key[tile];
    __syncthreads();
    const int key = s_key;
    const int level = key / NSLOT, slot = key % NSLOT;
    const int p0 = Pd.off[key] + (tile - Pd.tile_off[key]) * TN;
    const int p1 = min(p0 + TN, Pd.off[key + 1]);
    if (tid < TN) {
        int q = p0 + tid;
        trg[tid] = q < p1 ? Pd.trg[q] : -1;
        src[tid] = q < p1 ? Pd.src[q] : -1;
    }
    __syncthreads();
    const float *M = F.O.m2l_t + ((size_t)level * NSLOT + slot) * np * np;
    for (int i0 = 0; i0 < np; i0 += TM) {
        float acc[8][4];
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) acc[r][cc] = 0.f;
        gemm_slab(M, np, i0, F.ueq, src, As, Bs, acc);
        scatter_atomic(F.dchk, np, n, i0, trg, acc);
    }
}

void fmm_m2l_pairs(const FmmDev &F, const PairsDev &Pd, int nV, int m2l_prec, cudaStream_t st) {
    (void)m2l_prec;
    if (nV <= 0) return;
    // upper bound on the tile count: every key adds at most one partial tile
    int grid = (nV + TN - 1) / TN + Pd.nkeys;
    launch_pdl(k_m2l_pairs, grid, 256, 0, st, F, Pd);
}

// ---------------------------------------------------------------- L2P for whole leaf boxes
// Chebyshev far field: S(cell m of leaf B) = sum_k E_l[m][k] d_B[k], E_l the interpolation
// table of the box's e^3 cells (rows in local Morton order, stored transposed [k][m]).
// A CTA handles 64 leaves of one level; its 128 x 64 result tile goes through shared
// memory to the leaves' targets, whose local Morton index is the low 3 log2(e) bits of
// their key.  Writes (=) every target of every leaf of this level.
__global__ void __launch_bounds__(256) k_l2p_gemm(FmmDev F, int level, int box_begin, int box_count,
                                                  float *__restrict__ out) {
    pdl_enter();
    __shared__ __align__(16) float As[TK][TM];
    __shared__ __align__(16) float Bs[TK][TN];
    __shared__ float Cs[TM][TN + 1];
    __shared__ int col[TN];
    const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
    const int np = F.O.npad;
    const TreeDev &T = F.T;
    const int t0 = blockIdx.x * TN;
    const int i0 = blockIdx.y * TM;
    const int e = 1 << (F.D - level);
    const int rows = e * e * e;
    int any = 0;
    if (tid < TN) {
        int b = box_begin + t0 + tid;
        int ok = t0 + tid < box_count && T.b_leaf[b] && T.b_te[b] > T.b_tb[b];
        col[tid] = ok ? b : -1;
        any = ok;
    }
    if (!__syncthreads_or(any)) return;
    float acc[8][4];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) acc[r][cc] = 0.f;
    gemm_slab_g(F.O.e_tab + F.O.e_off[level], rows, rows, np, i0, F.dchk, col, As, Bs, acc);
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) Cs[ty * 8 + r][tx * 4 + cc] = acc[r][cc];
    __syncthreads();
    const uint32_t lmask = (uint32_t)rows - 1u;
    // warp w handles columns w, w + 8, ...; lanes stride over the column's targets
    const int warp = tid >> 5, lane = tid & 31;
    for (int c = warp; c < TN; c += 8) {
        int b = col[c];
        if (b < 0) continue;
        for (int t = T.b_tb[b] + lane; t < T.b_te[b]; t += 32) {
            int m = (int)(F.trg_key[t] & lmask) - i0;
            if (m < 0 || m >= TM) continue;
            uint32_t pc = key_pc(F.trg_key[t]);
            out[(int64_t)pc_i(pc) + (int64_t)F.nx * ((int64_t)pc_j(pc) + (int64_t)F.ny * pc_k(pc))] = Cs[m][c];
        }
    }
}

void fmm_l2p_gemm_level(const FmmDev &F, int level, int box_begin, int box_count, float *out, cudaStream_t st) {
    if (box_count <= 0 || level < 2 || F.O.e_off[level] < 0) return;
    int e = 1 << (F.D - level);
    dim3 grid((box_count + TN - 1) / TN, (e * e * e + TM - 1) / TM);
    launch_pdl(k_l2p_gemm, grid, 256, 0, st, F, level, box_begin, box_count, out);
}

void fmm_m2l_gemm_level(const FmmDev &F, int level, int box_begin, int box_count, cudaStream_t st) {
    if (box_count <= 0 || level < 2) return;
    dim3 grid((box_count + TN - 1) / TN, (F.O.npad + TM - 1) / TM);
    launch_pdl(k_m2l_gemm, grid, 256, 0, st, F, level, box_begin, box_count);
}

void fmm_l2l_gemm_level(const FmmDev &F, int level, int parent_begin, int parent_count, cudaStream_t st) {
    if (parent_count <= 0 || level < 3) return;
    dim3 grid((parent_count + TN - 1) / TN, (F.O.npad + TM - 1) / TM, 8);
    launch_pdl(k_l2l_gemm, grid, 256, 0, st, F, level, parent_begin, parent_count);
}

}  // namespace sph
