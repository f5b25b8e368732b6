// Far-field translations on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// M2L (paper Section 2.4, far interactions through the hierarchy) and L2L are
// dense contractions of 128 x 128 operators with gathered state vectors:
//     D[i][j] = sum_k Op[i][k] X[k][j],   X[:, j] = state row of box j.
// Split-precision BF16: Op = Op_hi + Op_lo, X = X_hi + X_lo (each BF16), and
//     D ~ Op_hi X_hi + Op_hi X_lo + Op_lo X_hi
// accumulated in FP32 in tensor memory (TMEM); the dropped Op_lo X_lo term is
// ~2^-16 relative, so the product keeps about 16 significant bits.
//
// One CTA (128 threads, one warpgroup) per tile of 64 columns:
//   * thread 0 loads the operator's two 32 KiB BF16 images (pre-swizzled in
//     global memory, see k_make_image) with bulk async copies on an mbarrier;
//   * all threads gather the 64 FP32 state rows, split them into BF16 hi / lo
//     and store them K-major with the 128-byte swizzle;
//   * thread 0 issues 3 x 8 tcgen05.mma (M = 128, N = 64, K = 16 each) into a
//     64-column TMEM accumulator and commits to a second mbarrier;
//   * warp w reads TMEM lanes 32w..32w+31 (rows i) and adds the result into the
//     destination boxes' downward state with global reductions (red.add): M2L
//     targets receive many tiles, and for L2L a reduction avoids a dependent
//     DRAM read per element.
// Every wait is bounded; on expiry the tile records an error code and still
// releases its TMEM.
#include <algorithm>

#include "sph_kernels.cuh"
#include "tc_sm103.cuh"

namespace sph {

constexpr int TCM = 128, TCN = 64, TCK = 128;
constexpr uint32_t A_BYTES = TCM * TCK * 2;        // one BF16 operator image (32 KiB)
constexpr uint32_t B_BYTES = TCN * TCK * 2;        // one BF16 gathered tile (16 KiB)
constexpr uint32_t TC_TAIL = 32 + 2 * TCN * 4;                     // 2 mbarriers, TMEM address, column indices
// dynamic shared memory: up to 1008 bytes of padding to the 1024-byte aligned base, the
// four operand tiles, then the tail
constexpr uint32_t TC_SMEM = 1024 + 2 * A_BYTES + 2 * B_BYTES + TC_TAIL;
constexpr uint32_t WAIT_LIMIT = 1u << 24;
void tc_init_attributes();
// target-stationary M2L (below): parts of the 216 positions around the parent, positions per part,
// dynamic shared memory (two operator buffers, the gathered tile, the source table, the tail)
constexpr int MT_P = 4;
constexpr int MT_OFFS = 216 / MT_P;
constexpr uint32_t MT_SMEM = 1024 + 4 * A_BYTES + 2 * A_BYTES + MT_OFFS * TCM * 4 + 1024;
__global__ void __launch_bounds__(256, 1) k_m2l_tiles(FmmDev F, const int *__restrict__ groups,
                                                      const int *__restrict__ ngroups, int *__restrict__ counter,
                                                      const uint16_t *__restrict__ images, int *err);

// Operator (FP32, transposed [k][i], stride np) -> BF16 hi / lo images, K-major SW128.
__global__ void k_make_image(const float *__restrict__ opT, int np, uint16_t *__restrict__ img) {
    pdl_enter();
    const float *src = opT + (size_t)blockIdx.y * np * np;
    uint16_t *hi = img + (size_t)blockIdx.y * 2 * (A_BYTES / 2);
    uint16_t *lo = hi + A_BYTES / 2;
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= TCM * TCK) return;
    int i = e / TCK, k = e % TCK;
    float v = (i < np && k < np) ? src[(size_t)k * np + i] : 0.f;
    uint16_t h, l;
    tc::split_bf16(v, h, l);
    uint32_t off = tc::sw128_offset(i, k, TCM) / 2;
    hi[off] = h;
    lo[off] = l;
}

void make_images(const float *opT, int np, int count, uint16_t *img, cudaStream_t st) {
    if (count <= 0) return;
    launch_pdl(k_make_image, dim3((TCM * TCK + 255) / 256, count), 256, 0, st, opT, np, img);
}

struct TcSmem {
    uint8_t *a_hi, *a_lo, *b_hi, *b_lo;
    uint64_t *bar_a, *bar_mma;
    uint32_t *tmem_base;
    int *col_src, *col_dst;
};

__device__ __forceinline__ TcSmem carve(uint8_t *raw) {
    uintptr_t p = reinterpret_cast<uintptr_t>(raw);
    p = (p + 1023) & ~(uintptr_t)1023;
    uint8_t *b = reinterpret_cast<uint8_t *>(p);
    TcSmem s;
    s.a_hi = b;
    s.a_lo = b + A_BYTES;
    s.b_hi = b + 2 * A_BYTES;
    s.b_lo = b + 2 * A_BYTES + B_BYTES;
    uint8_t *tail = b + 2 * A_BYTES + 2 * B_BYTES;
    s.bar_a = reinterpret_cast<uint64_t *>(tail);
    s.bar_mma = reinterpret_cast<uint64_t *>(tail + 8);
    s.tmem_base = reinterpret_cast<uint32_t *>(tail + 16);
    s.col_src = reinterpret_cast<int *>(tail + 32);
    s.col_dst = s.col_src + TCN;      // ends at tail + TC_TAIL <= raw + TC_SMEM
    return s;
}

// Gather the FP32 state rows col_src[j] (row stride np) into the BF16 hi / lo B tiles.
// Split 4 FP32 values into BF16 hi / lo and store them at element (row, k0..k0+3) of two
// K-major SW128 tiles with `rows` rows.
__device__ __forceinline__ void put_split4(uint8_t *hi, uint8_t *lo, int row, int k0, int rows, const float4 &v) {
    // cvt.rn.bf16x2 rounds two values to nearest even at once (first operand to the upper
    // half); the residuals x - hi are exact in FP32 and rounded the same way
    uint32_t h01, h23, l01, l23;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(h01) : "f"(v.y), "f"(v.x));
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(h23) : "f"(v.w), "f"(v.z));
    const float r0 = v.x - __uint_as_float(h01 << 16), r1 = v.y - __uint_as_float(h01 & 0xFFFF0000u);
    const float r2 = v.z - __uint_as_float(h23 << 16), r3 = v.w - __uint_as_float(h23 & 0xFFFF0000u);
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(l01) : "f"(r1), "f"(r0));
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(l23) : "f"(r3), "f"(r2));
    const uint32_t off = tc::sw128_offset(row, k0, rows);
    *reinterpret_cast<uint2 *>(hi + off) = make_uint2(h01, h23);
    *reinterpret_cast<uint2 *>(lo + off) = make_uint2(l01, l23);
}

// Gather `rows` FP32 state rows (index list `idx`, -1 = zero row; row stride np) into BF16
// hi / lo K-major SW128 tiles.  Loads are issued eight at a time per thread before any is
// converted, so a thread has eight row segments in flight instead of one.
__device__ __forceinline__ void gather_rows_split(uint8_t *hi, uint8_t *lo, const int *idx, int rows,
                                                  const float *__restrict__ state, int np) {
    constexpr int Q = TCK / 4;   // float4 per row
    const int total = rows * Q;
    for (int e0 = threadIdx.x; e0 < total; e0 += 8 * blockDim.x) {
        float4 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * blockDim.x;
            v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (e < total) {
                const int j = e / Q, q = e % Q;
                const int src = idx[j];
                if (src >= 0 && 4 * q < np) v[u] = __ldg(reinterpret_cast<const float4 *>(state + (size_t)src * np) + q);
            }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e < total) put_split4(hi, lo, e / Q, 4 * (e % Q), rows, v[u]);
        }
    }
}

__device__ __forceinline__ void gather_split(const TcSmem &s, const float *__restrict__ state, int np) {
    gather_rows_split(s.b_hi, s.b_lo, s.col_src, TCN, state, np);
}

// Issue the 3 x 8 MMAs of one tile (thread 0 only).
__device__ __forceinline__ void issue_mmas(const TcSmem &s, uint32_t tmem) {
    const uint32_t idesc = tc::idesc_bf16_f32(TCM, TCN);
    const uint32_t a_hi = tc::smem_u32(s.a_hi), a_lo = tc::smem_u32(s.a_lo);
    const uint32_t b_hi = tc::smem_u32(s.b_hi), b_lo = tc::smem_u32(s.b_lo);
#pragma unroll
    for (int ks = 0; ks < TCK / 16; ++ks) {
        uint32_t ao = tc::sw128_offset(0, 16 * ks, TCM);
        uint32_t bo = tc::sw128_offset(0, 16 * ks, TCN);
        tc::mma_bf16(tmem, tc::sdesc_sw128(a_hi + ao), tc::sdesc_sw128(b_hi + bo), idesc, ks > 0);
        tc::mma_bf16(tmem, tc::sdesc_sw128(a_hi + ao), tc::sdesc_sw128(b_lo + bo), idesc, 1);
        tc::mma_bf16(tmem, tc::sdesc_sw128(a_lo + ao), tc::sdesc_sw128(b_hi + bo), idesc, 1);
    }
    tc::mma_commit(tc::smem_u32(s.bar_mma));
}

// The common body: operator image `img` (hi followed by lo), columns already in smem.
// Adds D into out[col_dst[j] * np + i] (atomically if `atomic`).  Returns false on a timeout.
// Copy of the operator image `img` (hi followed by lo) into the A tile (thread 0).
__device__ __forceinline__ void tile_issue_image(const TcSmem &s, const uint16_t *__restrict__ img) {
    if (threadIdx.x == 0) {
        tc::mbar_expect_tx(tc::smem_u32(s.bar_a), 2 * A_BYTES);
        tc::bulk_g2s(tc::smem_u32(s.a_hi), img, A_BYTES, tc::smem_u32(s.bar_a));
        tc::bulk_g2s(tc::smem_u32(s.a_lo), img + A_BYTES / 2, A_BYTES, tc::smem_u32(s.bar_a));
    }
}

__device__ __forceinline__ void tile_body(const TcSmem &s, const uint16_t *__restrict__ img,
                                          const float *__restrict__ state, float *__restrict__ out, int np,
                                          int n, bool atomic, int *err, bool image_issued = false,
                                          bool bulk = false) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (!image_issued) tile_issue_image(s, img);
    gather_split(s, state, np);
    tc::fence_proxy_async_smem();
    __syncthreads();
    const uint32_t tmem = *s.tmem_base;
    __shared__ int ok_s;
    if (threadIdx.x == 0) {
        int ok = tc::mbar_wait_bounded(tc::smem_u32(s.bar_a), 0, WAIT_LIMIT);
        if (ok) {
            tc::fence_after_sync();
            issue_mmas(s, tmem);
        } else {
            atomicOr(err, 1);
            tc::mbar_wait_bounded(tc::smem_u32(s.bar_a), 0, WAIT_LIMIT);   // let the copies land
        }
        ok_s = ok;
    }
    __syncthreads();
    if (!ok_s) return;
    // every thread waits for the MMAs; the outcome is made uniform over the CTA (the bulk
    // epilogue below has barriers of its own)
    const bool mma_ok = tc::mbar_wait_bounded(tc::smem_u32(s.bar_mma), 0, WAIT_LIMIT);
    if (__syncthreads_or(!mma_ok)) {
        if (threadIdx.x == 0) atomicOr(err, 2);
        if (!mma_ok) tc::mbar_wait_bounded(tc::smem_u32(s.bar_mma), 0, WAIT_LIMIT);   // let the MMAs finish
        return;
    }
    tc::fence_after_sync();
    // warp w reads TMEM lanes 32 (w % 4) ..; with 8 warps, w and w + 4 take half the columns each
    const int q = warp & 3, i = q * 32 + lane;   // TMEM lane = operator row
    const int cw = TCN / ((int)blockDim.x / 128), cbeg = (warp >> 2) * cw;
    if (bulk) {
        // each column's np results staged as one contiguous row in the B tiles (free once the
        // MMAs have completed: TCN x np FP32 = 2 B_BYTES), then added into its target row by one
        // bulk reduction; padding rows (i >= n) add zeros
        float *stage = reinterpret_cast<float *>(s.b_hi);
        for (int c0 = cbeg; c0 < cbeg + cw; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
            if (i < np) {
#pragma unroll
                for (int j = 0; j < 16; ++j) stage[(c0 + j) * np + i] = i < n ? v[j] : 0.f;
            }
        }
        tc::fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x < TCN) {
            const int d = s.col_dst[threadIdx.x];
            if (d >= 0) {
                tc::bulk_reduce_add_f32(out + (size_t)d * np, tc::smem_u32(stage + threadIdx.x * np),
                                        (uint32_t)np * 4u);
                tc::bulk_commit();
                tc::bulk_wait_read_all();
            }
        }
        return;
    }
    for (int c0 = cbeg; c0 < cbeg + cw; c0 += 16) {
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
        if (i < n) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                int d = s.col_dst[c0 + j];
                if (d < 0) continue;
                // reductions (fire and forget) in both cases; `atomic` only documents whether
                // several tiles may add into the same element
                (void)atomic;
                atomicAdd(out + (size_t)d * np + i, v[j]);
            }
        }
    }
}

__device__ __forceinline__ void tile_setup(const TcSmem &s) {
    if (threadIdx.x < 32) {
        tc::tmem_alloc(tc::smem_u32(s.tmem_base), TCN);
        tc::tmem_relinquish();
    }
    if (threadIdx.x == 0) {
        tc::mbar_init(tc::smem_u32(s.bar_a), 1);
        tc::mbar_init(tc::smem_u32(s.bar_mma), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

__device__ __forceinline__ void tile_teardown(const TcSmem &s) {
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) tc::tmem_dealloc(*s.tmem_base, TCN);
}

// ---------------------------------------------------------------- M2L over offset-grouped V pairs
__global__ void __launch_bounds__(256) k_m2l_tc(FmmDev F, PairsDev Pd, const uint16_t *__restrict__ images,
                                                int *err) {
    // prologue (the V pairs, their tiles and the operator images were written before the passes)
    extern __shared__ uint8_t smem_raw[];
    const int tile = blockIdx.x;
    if (tile >= Pd.tile_off[Pd.nkeys]) return;
    TcSmem s = carve(smem_raw);
    __shared__ int s_key;
    if (threadIdx.x == 0) s_key = Pd.tile_key[tile];
    tile_setup(s);
    const int key = s_key;
    const int p0 = Pd.off[key] + (tile - Pd.tile_off[key]) * TCN;
    const int p1 = min(p0 + TCN, Pd.off[key + 1]);
    if (threadIdx.x < TCN) {
        int q = p0 + threadIdx.x;
        s.col_src[threadIdx.x] = q < p1 ? Pd.src[q] : -1;
        s.col_dst[threadIdx.x] = q < p1 ? Pd.trg[q] : -1;
    }
    const uint16_t *img = images + (size_t)key * (2 * A_BYTES / 2);
    tile_issue_image(s, img);
    pdl_enter();
    __syncthreads();
    tile_body(s, img, F.ueq, F.dchk, F.O.npad, F.O.n, true, err, true, true);
    tile_teardown(s);
}

// ---------------------------------------------------------------- M2L, persistent tile loop
// Two CTAs per SM, each taking tile blockIdx.x first and then the tiles gridDim.x + ticket (a
// counter, cleared before the passes, so that CTAs that start late beside other kernels take
// fewer), with the tensor memory and barriers set up once.  Per tile: (1) the previous tile's bulk reductions
// have read the staged rows (the B tiles), (2) gather and split the 64 source rows, (3) MMAs
// once the operator image has landed, (4) the next tile's pair indices while they run, (5) the
// MMAs complete, (6) the next tile's operator image streams into the A tile, (7) the results
// are staged in the B tiles and added into the targets by bulk reductions that complete under
// the next tile's steps (1)-(2).  The same sums as k_m2l_tc.
__global__ void __launch_bounds__(256) k_m2l_tc_loop(FmmDev F, PairsDev Pd, const uint16_t *__restrict__ images,
                                                     int *err, int *ticket) {
    // prologue (the V pairs, their tiles and the operator images were written before the passes)
    extern __shared__ uint8_t smem_raw[];
    const int ntile = Pd.tile_off[Pd.nkeys];
    if ((int)blockIdx.x >= ntile) return;                // uniform, before any allocation
    TcSmem s = carve(smem_raw);
    __shared__ int s_src[2][TCN], s_dst[2][TCN];
    __shared__ int s_ok, s_next;
    const int tid = threadIdx.x;
    // pair indices of `tile` into slot `slot` (threads < TCN; each finds the tile's key itself)
    auto tile_meta = [&](int tile, int slot) {
        const int key = Pd.tile_key[tile];
        const int p0 = Pd.off[key] + (tile - Pd.tile_off[key]) * TCN;
        const int p1 = min(p0 + TCN, Pd.off[key + 1]);
        const int q = p0 + tid;
        s_src[slot][tid] = q < p1 ? Pd.src[q] : -1;
        s_dst[slot][tid] = q < p1 ? Pd.trg[q] : -1;
        return key;
    };
    auto issue_image = [&](int key) {
        const uint16_t *img = images + (size_t)key * (2 * A_BYTES / 2);
        tc::mbar_expect_tx(tc::smem_u32(s.bar_a), 2 * A_BYTES);
        tc::bulk_g2s(tc::smem_u32(s.a_hi), img, A_BYTES, tc::smem_u32(s.bar_a));
        tc::bulk_g2s(tc::smem_u32(s.a_lo), img + A_BYTES / 2, A_BYTES, tc::smem_u32(s.bar_a));
    };
    tile_setup(s);
    if (tid < TCN) {
        const int key0 = tile_meta(blockIdx.x, 0);
        if (tid == 0) issue_image(key0);
    }
    pdl_enter();
    const uint32_t tmem = *s.tmem_base;
    const int np = F.O.npad, n = F.O.n;
    const int warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, i = q * 32 + lane;           // TMEM lane = operator row
    const int cbeg = (warp >> 2) * (TCN / 2);
    float *stage = reinterpret_cast<float *>(s.b_hi);    // TCN rows of TCK FP32 (the two B tiles)
    int it = 0, flag = 0;
    bool image_pending = true;                            // an image copy not yet waited for
    for (int tile = blockIdx.x; tile < ntile; ++it) {
        const int slot = it & 1;
        if (tid == 0) s_next = (int)gridDim.x + atomicAdd(ticket, 1);
        // (1) the previous tile's staged rows have been read (and slot's indices are visible)
        if (tid < TCN) tc::bulk_wait_read_all();
        __syncthreads();
        const int nt = s_next;
        // (2) the source rows into the B tiles
        gather_rows_split(s.b_hi, s.b_lo, s_src[slot], TCN, F.ueq, np);
        tc::fence_proxy_async_smem();
        __syncthreads();
        // (3) MMAs once the image has landed
        if (tid == 0) {
            int ok = tc::mbar_wait_bounded(tc::smem_u32(s.bar_a), it & 1, WAIT_LIMIT);
            if (ok) {
                image_pending = false;
                tc::fence_after_sync();
                issue_mmas(s, tmem);
            }
            s_ok = ok;
        }
        // (4) the next tile's pair indices while the MMAs run
        int nkey = 0;
        if (nt < ntile && tid < TCN) nkey = tile_meta(nt, slot ^ 1);
        __syncthreads();
        if (!s_ok) {
            flag = 1;
            break;
        }
        // (5) the MMAs complete (uniform outcome)
        const bool mma_ok = tc::mbar_wait_bounded(tc::smem_u32(s.bar_mma), it & 1, WAIT_LIMIT);
        if (__syncthreads_or(!mma_ok)) {
            flag = 2;
            if (!mma_ok) tc::mbar_wait_bounded(tc::smem_u32(s.bar_mma), it & 1, WAIT_LIMIT);
            break;
        }
        tc::fence_after_sync();
        // (6) the next tile's image into the A tile (its readers, the MMAs, have completed)
        if (tid == 0 && nt < ntile) {
            issue_image(nkey);
            image_pending = true;
        }
        // (7) results staged as one FP32 row per pair in the B tiles, then one bulk reduction per
        // pair into its target's row (padding rows add zeros)
        for (int c0 = cbeg; c0 < cbeg + TCN / 2; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) stage[(c0 + j) * TCK + i] = i < n ? v[j] : 0.f;
        }
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();                         // the TMEM reads before the next tile's MMAs
        __syncthreads();
        if (tid < TCN) {
            const int d = s_dst[slot][tid];
            if (d >= 0) {
                tc::bulk_reduce_add_f32(F.dchk + (size_t)d * np, tc::smem_u32(stage + tid * TCK), (uint32_t)np * 4u);
                tc::bulk_commit();
            }
        }
        tile = nt;
    }
    if (tid == 0 && flag) {
        atomicOr(err, flag);
        // an image copy in flight lands before this CTA's memory is released
        if (image_pending) tc::mbar_wait_bounded(tc::smem_u32(s.bar_a), it & 1, WAIT_LIMIT);
    }
    if (tid < TCN) tc::bulk_wait_read_all();
    tile_teardown(s);
}

// ---------------------------------------------------------------- M2L, persistent and pipelined
// One CTA per SM walks a contiguous range of tiles (tiles of one (level, offset) group are
// consecutive, so the operator image is reused while the group lasts).  Per tile i:
//   (a) the FP32 source rows of tile i, copied by cp.async during tile i-1, have landed;
//   (b) MMA(i-1) has completed (the B tile and its TMEM accumulator are free / ready);
//   (c) the rows are split into the BF16 hi / lo B tile;
//   (d, e) tile i+1's pair indices are read and its rows start to stream in (cp.async);
//   (f) thread 0 issues MMA(i) into accumulator i % 2 and, if tile i+1 needs another
//       operator, its image into the other A buffer;
//   (g) all threads stage accumulator (i-1) % 2 as one FP32 row per pair, and one thread per
//       pair adds its row into the target by a bulk reduction,
// so the epilogue of one tile runs under the MMAs and loads of the next.  Pair metadata
// rotates through three slots (i+1 is written while i-1 is still being scattered).
constexpr uint32_t PIPE_RAW = TCN * TCK * 4;       // 64 rows x 128 FP32
constexpr uint32_t PIPE_STG = TCN * TCK * 4;       // staged results, 64 pairs x 128 FP32
constexpr uint32_t PIPE_SMEM = 1024 + 4 * A_BYTES + 2 * B_BYTES + PIPE_RAW + PIPE_STG + 64 + 6 * TCN * 4 + 64;
static_assert(PIPE_SMEM <= 227 * 1024, "pipelined M2L: shared memory above the per-CTA limit");

__device__ __forceinline__ void m2l_tile_range(const PairsDev &Pd, int key, int tile, int &p0, int &p1) {
    p0 = Pd.off[key] + (tile - Pd.tile_off[key]) * TCN;
    p1 = min(p0 + TCN, Pd.off[key + 1]);
}

__global__ void __launch_bounds__(128, 1) k_m2l_tc_pipe(FmmDev F, PairsDev Pd, const uint16_t *__restrict__ images,
                                                        int *err) {
    pdl_enter();
    const int T = Pd.tile_off[Pd.nkeys];
    const int chunk = (T + gridDim.x - 1) / gridDim.x;
    const int t_begin = blockIdx.x * chunk, t_end = min(T, t_begin + chunk);
    if (t_begin >= t_end) return;                  // uniform, before any allocation
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *abuf[2] = {base, base + 2 * A_BYTES};
    uint8_t *b_hi = base + 4 * A_BYTES, *b_lo = b_hi + B_BYTES;
    float *raw = reinterpret_cast<float *>(b_lo + B_BYTES);
    float *stg = raw + TCN * TCK;
    uint8_t *tail = reinterpret_cast<uint8_t *>(stg) + PIPE_STG;
    uint64_t *bar_a = reinterpret_cast<uint64_t *>(tail);       // [2]
    uint64_t *bar_mma = bar_a + 2;                              // [2]
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar_a + 4);
    int *ctl = reinterpret_cast<int *>(tslot + 1);              // [0] error, [1] next key, [2] next aslot
    int *msrc = reinterpret_cast<int *>(tail + 64);             // [3][TCN]
    int *mdst = msrc + 3 * TCN;                                 // [3][TCN]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int np = F.O.npad, n = F.O.n;
    if (tid < 32) {
        tc::tmem_alloc(tc::smem_u32(tslot), 128);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int k = 0; k < 2; ++k) {
            tc::mbar_init(tc::smem_u32(bar_a + k), 1);
            tc::mbar_init(tc::smem_u32(bar_mma + k), 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        int key = 0, lo = 0, hi = Pd.nkeys;
        while (hi - lo > 1) {                      // key of the first tile
            const int mid = (lo + hi) >> 1;
            if (Pd.tile_off[mid] <= t_begin) lo = mid; else hi = mid;
        }
        key = lo;
        ctl[0] = 0;
        ctl[1] = key;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    // thread-0 state of the image buffers
    int a_loads[2] = {0, 0}, a_landed[2] = {0, 0};
    int cur_key = ctl[1], cur_slot = 0;
    auto fill_meta = [&](int tile, int key, int ms) {
        if (tid < TCN) {
            int p0, p1;
            m2l_tile_range(Pd, key, tile, p0, p1);
            const int q = p0 + tid;
            msrc[ms * TCN + tid] = q < p1 ? Pd.src[q] : -1;
            mdst[ms * TCN + tid] = q < p1 ? Pd.trg[q] : -1;
        }
    };
    auto issue_raw = [&](int ms) {
        for (int e = tid; e < TCN * (TCK / 4); e += 128) {
            const int row = e >> 5, q = e & 31;
            const int src = msrc[ms * TCN + row];
            const float *g = src >= 0 && 4 * q < np ? F.ueq + (size_t)src * np + 4 * q : F.ueq;
            tc::cp_async16(tc::smem_u32(raw + row * TCK + 4 * q), g, (src >= 0 && 4 * q < np) ? 16u : 0u);
        }
        tc::cp_async_commit();
    };
    auto epilogue = [&](int i) {
        const int ms = i % 3;
        const uint32_t col = (uint32_t)((i & 1) * TCN);
        const int row = warp * 32 + lane;
        // the previous tile's bulk reductions have read the staged rows
        if (tid < TCN) tc::bulk_wait_read_all();
        __syncthreads();
#pragma unroll
        for (int c0 = 0; c0 < TCN; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + col + (uint32_t)c0, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) stg[(c0 + j) * TCK + row] = row < n ? v[j] : 0.f;
        }
        tc::fence_proxy_async_smem();
        __syncthreads();
        if (tid < TCN) {
            const int d = mdst[ms * TCN + tid];
            if (d >= 0) {
                tc::bulk_reduce_add_f32(F.dchk + (size_t)d * np, tc::smem_u32(stg + tid * TCK), (uint32_t)np * 4u);
                tc::bulk_commit();
            }
        }
    };
    // prologue: tile t_begin's metadata, rows and image
    fill_meta(t_begin, cur_key, 0);
    __syncthreads();
    issue_raw(0);
    if (tid == 0) {
        tc::mbar_expect_tx(tc::smem_u32(bar_a), 2 * A_BYTES);
        tc::bulk_g2s(tc::smem_u32(abuf[0]), images + (size_t)cur_key * (2 * A_BYTES / 2), 2 * A_BYTES,
                     tc::smem_u32(bar_a));
        a_loads[0] = 1;
    }
    const int ntile = t_end - t_begin;
    const uint32_t idesc = tc::idesc_bf16_f32(TCM, TCN);
    int done_epi = -1;
    for (int i = 0; i < ntile; ++i) {
        const int t = t_begin + i;
        // (a) rows of tile i landed (every thread's copies)
        tc::cp_async_wait<0>();
        // (b) MMA(i-1) complete
        if (tid == 0 && i >= 1) {
            if (!tc::mbar_wait_bounded(tc::smem_u32(bar_mma + ((i - 1) & 1)), ((i - 1) >> 1) & 1, WAIT_LIMIT))
                ctl[0] |= 2;
        }
        __syncthreads();
        if (ctl[0]) break;
        tc::fence_after_sync();
        // (c) split the rows into the B tile
        for (int e = tid; e < TCN * (TCK / 4); e += 128) {
            const int row = e >> 5, q = e & 31;
            put_split4(b_hi, b_lo, row, 4 * q, TCN, *reinterpret_cast<const float4 *>(raw + row * TCK + 4 * q));
        }
        tc::fence_proxy_async_smem();
        // (d) next tile's key and metadata
        if (tid == 0 && i + 1 < ntile) {
            int k = cur_key;
            while (Pd.tile_off[k + 1] <= t + 1) ++k;
            ctl[1] = k;
        }
        __syncthreads();
        const int next_key = ctl[1];
        if (i + 1 < ntile) fill_meta(t + 1, next_key, (i + 1) % 3);
        __syncthreads();
        // (e) rows of tile i+1 start streaming into the raw buffer (free: converted above)
        if (i + 1 < ntile) issue_raw((i + 1) % 3);
        // (f) MMA(i), and the image of tile i+1 if its operator differs
        if (tid == 0) {
            int ok = 1;
            if (a_landed[cur_slot] < a_loads[cur_slot]) {
                ok = tc::mbar_wait_bounded(tc::smem_u32(bar_a + cur_slot), (a_loads[cur_slot] - 1) & 1, WAIT_LIMIT);
                a_landed[cur_slot] = a_loads[cur_slot];
            }
            if (ok) {
                tc::fence_after_sync();
                const uint32_t ahi = tc::smem_u32(abuf[cur_slot]), alo = ahi + A_BYTES;
                const uint32_t bhi = tc::smem_u32(b_hi), blo = tc::smem_u32(b_lo);
                const uint32_t d = tmem + (uint32_t)((i & 1) * TCN);
#pragma unroll
                for (int ks = 0; ks < TCK / 16; ++ks) {
                    const uint32_t ao = tc::sw128_offset(0, 16 * ks, TCM);
                    const uint32_t bo = tc::sw128_offset(0, 16 * ks, TCN);
                    tc::mma_bf16(d, tc::sdesc_sw128(ahi + ao), tc::sdesc_sw128(bhi + bo), idesc, ks > 0);
                    tc::mma_bf16(d, tc::sdesc_sw128(ahi + ao), tc::sdesc_sw128(blo + bo), idesc, 1);
                    tc::mma_bf16(d, tc::sdesc_sw128(alo + ao), tc::sdesc_sw128(bhi + bo), idesc, 1);
                }
                tc::mma_commit(tc::smem_u32(bar_mma + (i & 1)));
                if (i + 1 < ntile && next_key != cur_key) {
                    // the other buffer's last reader was tile i-1 or earlier, complete at (b)
                    const int o = cur_slot ^ 1;
                    tc::mbar_expect_tx(tc::smem_u32(bar_a + o), 2 * A_BYTES);
                    tc::bulk_g2s(tc::smem_u32(abuf[o]), images + (size_t)next_key * (2 * A_BYTES / 2),
                                 2 * A_BYTES, tc::smem_u32(bar_a + o));
                    ++a_loads[o];
                    cur_slot = o;
                }
            } else {
                ctl[0] |= 1;
            }
            cur_key = next_key;
        }
        // (g) scatter tile i-1 while MMA(i) runs
        if (i >= 1) {
            epilogue(i - 1);
            done_epi = i - 1;
        }
        tc::fence_before_sync();
    }
    __syncthreads();
    // last tile: wait for its MMAs, then scatter it
    const int last = ntile - 1;
    if (tid == 0 && !ctl[0]) {
        if (!tc::mbar_wait_bounded(tc::smem_u32(bar_mma + (last & 1)), (last >> 1) & 1, WAIT_LIMIT)) ctl[0] |= 2;
    }
    __syncthreads();
    if (!ctl[0] && done_epi < last) {
        tc::fence_after_sync();
        epilogue(last);
    }
    if (ctl[0] && tid == 0) {
        atomicOr(err, ctl[0]);
        // let this CTA's copies and MMAs finish before its memory is released
        for (int k = 0; k < 2; ++k)
            if (a_landed[k] < a_loads[k])
                tc::mbar_wait_bounded(tc::smem_u32(bar_a + k), (a_loads[k] - 1) & 1, WAIT_LIMIT);
        for (int k = 0; k < 2 && k <= last; ++k) {
            const int i_last = last - ((last - k) & 1);      // last tile that used accumulator k
            tc::mbar_wait_bounded(tc::smem_u32(bar_mma + (i_last & 1)), (i_last >> 1) & 1, WAIT_LIMIT);
        }
    }
    tc::cp_async_wait<0>();
    if (tid < TCN) tc::bulk_wait_read_all();
    tc::fence_before_sync();
    __syncthreads();
    if (tid < 32) tc::tmem_dealloc(tmem, 128);
}

// ---------------------------------------------------------------- L2L for one level
__global__ void __launch_bounds__(256) k_l2l_tc(FmmDev F, int level, int parent_begin, int parent_count,
                                                const uint16_t *__restrict__ images, int *err) {
    // prologue: tree arrays and operator images only
    extern __shared__ uint8_t smem_raw[];
    TcSmem s = carve(smem_raw);
    const int t0 = blockIdx.x * TCN;
    const int c = blockIdx.y;
    const TreeDev &T = F.T;
    int any = 0;
    if (threadIdx.x < TCN) {
        int p = parent_begin + t0 + threadIdx.x;
        int P = -1, C = -1;
        if (t0 + (int)threadIdx.x < parent_count && !T.b_leaf[p] && T.b_te[p] > T.b_tb[p]) {
            int ch = T.box_at[dense_off(level) + ((T.b_key[p] << 3) | (uint32_t)c)];
            if (ch >= 0 && T.b_te[ch] > T.b_tb[ch]) { P = p; C = ch; }
        }
        any = C >= 0;
        s.col_src[threadIdx.x] = P;
        s.col_dst[threadIdx.x] = C;
    }
    if (!__syncthreads_or(any)) return;
    tile_setup(s);
    const uint16_t *img = images + ((size_t)level * 8 + c) * (2 * A_BYTES / 2);
    tile_issue_image(s, img);
    pdl_enter();
    tile_body(s, img, F.dchk, F.dchk, F.O.npad, F.O.n, false, err, true, true);
    tile_teardown(s);
}

// ---------------------------------------------------------------- M2M, one child slot per CTA
// Tiles of 64 split boxes with sources of one level (from the level's compact source list)
// x child slot c = blockIdx.y:  u_P += M2M_c u_{child c of P}, BF16 hi / lo x3, added with
// reductions into rows that the work-list kernel zeroed.
__global__ void __launch_bounds__(256) k_m2m_tc(FmmDev F, int level, const int *__restrict__ list,
                                                const int *__restrict__ count, const uint16_t *__restrict__ images,
                                                int *err) {
    // prologue: this CTA's tensor memory, barriers and operator image (the source list and its
    // count come from the work lists, read after the wait)
    extern __shared__ uint8_t smem_raw[];
    TcSmem s = carve(smem_raw);
    const int t0 = blockIdx.x * TCN;
    const int c = blockIdx.y;
    tile_setup(s);
    const uint16_t *img = images + ((size_t)level * 8 + c) * (2 * A_BYTES / 2);
    tile_issue_image(s, img);
    pdl_enter();
    const int cnt = *count;
    int any = 0;
    const TreeDev &T = F.T;
    if (threadIdx.x < TCN) {
        const int j = t0 + threadIdx.x;
        int P = -1, C = -1;
        if (t0 < cnt && j < cnt) {
            const int p = list[j];
            if (!T.b_leaf[p]) {
                const int ch = T.box_at[dense_off(level + 1) + ((T.b_key[p] << 3) | (uint32_t)c)];
                if (ch >= 0 && T.b_se[ch] > T.b_sb[ch]) { P = p; C = ch; }
            }
        }
        any = C >= 0;
        s.col_src[threadIdx.x] = C;
        s.col_dst[threadIdx.x] = P;
    }
    if (!__syncthreads_or(any)) {
        // nothing to do: let the image copy land before the shared memory is released
        if (threadIdx.x == 0) tc::mbar_wait_bounded(tc::smem_u32(s.bar_a), 0, WAIT_LIMIT);
        tile_teardown(s);
        return;
    }
    tile_body(s, img, F.ueq, F.ueq, F.O.npad, F.O.n, true, err, true, true);
    tile_teardown(s);
}

void fmm_m2m_tc_level(const FmmDev &F, int level, int box_count, const int *list, const int *count,
                      const uint16_t *images, int *err, cudaStream_t st) {
    if (box_count <= 0 || level < 2) return;
    tc_init_attributes();
    dim3 grid((box_count + TCN - 1) / TCN, 8);
    launch_pdl(k_m2m_tc, grid, 256, TC_SMEM, st, F, level, list, count, images, err);
}

// ---------------------------------------------------------------- L2L, all 8 children per CTA
// 64 parents per CTA; their downward states are gathered once (B tile), and the 8 child
// operators stream through two 64 KiB image buffers: image c + 2 is loaded into the
// buffer of image c as soon as the MMAs reading it have completed.  Child c accumulates
// into TMEM columns [64c, 64c + 64), all 512 columns of the SM's tensor memory.
constexpr uint32_t L8_SMEM = 1024 + 4 * A_BYTES + 2 * B_BYTES + 64 + 9 * TCN * 4;

__global__ void __launch_bounds__(128) k_l2l_tc8(FmmDev F, int level, int parent_begin, int parent_count,
                                                 const uint16_t *__restrict__ images, int *err) {
    // prologue: tree arrays, tensor memory, barriers and the first two operator images
    extern __shared__ uint8_t smem_raw[];
    uintptr_t pa = (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023;
    uint8_t *base = reinterpret_cast<uint8_t *>(pa);
    uint8_t *abuf[2] = {base, base + 2 * A_BYTES};        // each: hi (32 KiB) then lo (32 KiB)
    TcSmem s;
    s.a_hi = abuf[0];
    s.a_lo = abuf[0] + A_BYTES;
    s.b_hi = base + 4 * A_BYTES;
    s.b_lo = s.b_hi + B_BYTES;
    uint8_t *tail = s.b_lo + B_BYTES;
    uint64_t *bar_a = reinterpret_cast<uint64_t *>(tail);          // [2]
    uint64_t *bar_free = bar_a + 2;                                 // [2]
    s.bar_mma = bar_a + 4;
    s.tmem_base = reinterpret_cast<uint32_t *>(tail + 40);
    s.col_src = reinterpret_cast<int *>(tail + 64);
    int *dst = s.col_src + TCN;                                     // [8][TCN]
    s.col_dst = dst;
    const int t0 = blockIdx.x * TCN;
    const TreeDev &T = F.T;
    const int np = F.O.npad, n = F.O.n;
    int any = 0;
    if (threadIdx.x < TCN) {
        int p = parent_begin + t0 + threadIdx.x;
        int P = -1;
        if (t0 + (int)threadIdx.x < parent_count && !T.b_leaf[p] && T.b_te[p] > T.b_tb[p]) P = p;
        for (int c = 0; c < 8; ++c) {
            int C = -1;
            if (P >= 0) {
                int ch = T.box_at[dense_off(level) + ((T.b_key[P] << 3) | (uint32_t)c)];
                if (ch >= 0 && T.b_te[ch] > T.b_tb[ch]) C = ch;
            }
            dst[c * TCN + threadIdx.x] = C;
            any |= C >= 0;
        }
        s.col_src[threadIdx.x] = P;
    }
    if (!__syncthreads_or(any)) return;
    if (threadIdx.x < 32) {
        tc::tmem_alloc(tc::smem_u32(s.tmem_base), 512);
        tc::tmem_relinquish();
    }
    if (threadIdx.x == 0) {
        for (int k = 0; k < 2; ++k) {
            tc::mbar_init(tc::smem_u32(bar_a + k), 1);
            tc::mbar_init(tc::smem_u32(bar_free + k), 1);
        }
        tc::mbar_init(tc::smem_u32(s.bar_mma), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint16_t *img0 = images + (size_t)level * 8 * (2 * A_BYTES / 2);
    if (threadIdx.x == 0) {
        for (int k = 0; k < 2; ++k) {
            tc::mbar_expect_tx(tc::smem_u32(bar_a + k), 2 * A_BYTES);
            tc::bulk_g2s(tc::smem_u32(abuf[k]), img0 + (size_t)k * (2 * A_BYTES / 2), 2 * A_BYTES,
                         tc::smem_u32(bar_a + k));
        }
    }
    pdl_enter();
    gather_split(s, F.dchk, np);
    tc::fence_proxy_async_smem();
    __syncthreads();
    const uint32_t tmem = *s.tmem_base;
    __shared__ int ok_s;
    if (threadIdx.x == 0) {
        int ok = 1;
        int issued[2] = {1, 1}, landed[2] = {0, 0};   // image loads per buffer
        const uint32_t idesc = tc::idesc_bf16_f32(TCM, TCN);
        const uint32_t b_hi = tc::smem_u32(s.b_hi), b_lo = tc::smem_u32(s.b_lo);
        for (int c = 0; c < 8 && ok; ++c) {
            const int k = c & 1;
            ok = tc::mbar_wait_bounded(tc::smem_u32(bar_a + k), (c >> 1) & 1, WAIT_LIMIT);
            if (!ok) break;
            ++landed[k];
            tc::fence_after_sync();
            const uint32_t a_hi = tc::smem_u32(abuf[k]), a_lo = a_hi + A_BYTES;
            const uint32_t d = tmem + (uint32_t)(c * TCN);
#pragma unroll
            for (int ks = 0; ks < TCK / 16; ++ks) {
                uint32_t ao = tc::sw128_offset(0, 16 * ks, TCM);
                uint32_t bo = tc::sw128_offset(0, 16 * ks, TCN);
                tc::mma_bf16(d, tc::sdesc_sw128(a_hi + ao), tc::sdesc_sw128(b_hi + bo), idesc, ks > 0);
                tc::mma_bf16(d, tc::sdesc_sw128(a_hi + ao), tc::sdesc_sw128(b_lo + bo), idesc, 1);
                tc::mma_bf16(d, tc::sdesc_sw128(a_lo + ao), tc::sdesc_sw128(b_hi + bo), idesc, 1);
            }
            tc::mma_commit(tc::smem_u32(bar_free + k));
            if (c + 2 < 8) {
                ok = tc::mbar_wait_bounded(tc::smem_u32(bar_free + k), (c >> 1) & 1, WAIT_LIMIT);
                if (!ok) break;
                tc::mbar_expect_tx(tc::smem_u32(bar_a + k), 2 * A_BYTES);
                tc::bulk_g2s(tc::smem_u32(abuf[k]), img0 + (size_t)(c + 2) * (2 * A_BYTES / 2), 2 * A_BYTES,
                             tc::smem_u32(bar_a + k));
                ++issued[k];
            }
        }
        tc::mma_commit(tc::smem_u32(s.bar_mma));   // tracks every MMA issued so far
        if (!ok) {
            atomicOr(err, 4);
            // let this CTA's own copies and MMAs finish before its memory is released
            for (int k = 0; k < 2; ++k)
                if (issued[k] > landed[k])
                    tc::mbar_wait_bounded(tc::smem_u32(bar_a + k), (issued[k] - 1) & 1, WAIT_LIMIT);
            tc::mbar_wait_bounded(tc::smem_u32(s.bar_mma), 0, WAIT_LIMIT);
        }
        ok_s = ok;
    }
    __syncthreads();
    const bool mma_ok = ok_s && tc::mbar_wait_bounded(tc::smem_u32(s.bar_mma), 0, WAIT_LIMIT);
    const bool done = !__syncthreads_or(ok_s && !mma_ok);   // uniform over the CTA
    if (ok_s && !mma_ok) atomicOr(err, 8);
    if (ok_s && done) {
        tc::fence_after_sync();
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int i = warp * 32 + lane;
        // each child's results staged as one FP32 row per parent in the operator buffers (free once
        // every MMA has completed: 4 x 32 KiB, four children at a time), each row added into the
        // child's downward state by one bulk reduction; padding rows add zeros
        float *stg = reinterpret_cast<float *>(base);
        for (int c = 0; c < 8; ++c) {
            if (c == 4) {
                if (threadIdx.x < TCN) tc::bulk_wait_read_all();
                __syncthreads();
            }
            float *sc = stg + (c & 3) * TCN * TCK;
#pragma unroll
            for (int c0 = 0; c0 < TCN; c0 += 16) {
                float v[16];
                tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * TCN + c0), v);
#pragma unroll
                for (int j = 0; j < 16; ++j) sc[(c0 + j) * TCK + i] = i < n ? v[j] : 0.f;
            }
            if ((c & 3) == 3) {
                tc::fence_proxy_async_smem();
                __syncthreads();
                if (threadIdx.x < TCN) {
                    for (int cc = c - 3; cc <= c; ++cc) {
                        const int C = dst[cc * TCN + threadIdx.x];
                        if (C >= 0)
                            tc::bulk_reduce_add_f32(F.dchk + (size_t)C * np,
                                                    tc::smem_u32(stg + (cc & 3) * TCN * TCK + threadIdx.x * TCK),
                                                    (uint32_t)np * 4u);
                    }
                    tc::bulk_commit();
                }
            }
        }
        if (threadIdx.x < TCN) tc::bulk_wait_read_all();
    }
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) tc::tmem_dealloc(tmem, 512);
}

void fmm_l2l_tc8_level(const FmmDev &F, int level, int parent_begin, int parent_count, const uint16_t *images,
                       int *err, cudaStream_t st) {
    if (parent_count <= 0 || level < 3) return;
    tc_init_attributes();
    launch_pdl(k_l2l_tc8, (parent_count + TCN - 1) / TCN, 128, L8_SMEM, st, F, level, parent_begin, parent_count, images,
                                                                     err);
}

// ---------------------------------------------------------------- L2P on the tensor cores
// S(cell c of leaf B) = sum_k E_l[c][k] d_B[k] for every leaf of one level, as
//     D[box][cell] = sum_k d[box][k] E[cell][k]    (M = 128 boxes, N = up to 64 cells, K = 128)
// with BF16 hi / lo splits of both operands (3 products).  The table of a level is stored
// as images of N cells each (lexicographic order inside the box, x fastest), ready for a
// bulk copy into shared memory.  One CTA gathers 128 boxes' d once and loops over the
// level's cell tiles; thread r (TMEM lane r) writes box r's cells.  A box whose every cell
// is a target is written whole; a partly selected box writes where the target mask is set.
constexpr uint32_t L2P_A = TCM * TCK * 2;               // 32 KiB: 128 boxes x 128 coefficients
constexpr uint32_t L2P_B = 64 * TCK * 2;                // 16 KiB: up to 64 cells x 128
constexpr uint32_t L2P_SMEM = 1024 + 2 * L2P_A + 2 * L2P_B + 64 + 2 * TCM * 4;

__global__ void k_l2p_image(const float *__restrict__ etab, int e, int n, int N, int ntiles, uint16_t *img) {
    pdl_enter();
    const int rows = e * e * e;
    const size_t total = (size_t)ntiles * N * TCK;
    const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int t = (int)(idx / ((size_t)N * TCK));
    const int rem = (int)(idx % ((size_t)N * TCK));
    const int j = rem / TCK, k = rem % TCK;
    const int c = t * N + j;
    float v = 0.f;
    if (c < rows && k < n) {
        const uint32_t lx = c % e, ly = (c / e) % e, lz = c / (e * e);
        v = etab[(size_t)k * rows + morton3(lx, ly, lz)];
    }
    uint16_t hi, lo;
    tc::split_bf16(v, hi, lo);
    uint16_t *base = img + (size_t)t * 2 * N * TCK;
    const uint32_t off = tc::sw128_offset(j, k, N) / 2;
    base[off] = hi;
    base[(size_t)N * TCK + off] = lo;
}

__host__ __device__ int l2p_tile_n(int e) {
    const int rows = e * e * e;
    const int r16 = (rows + 15) / 16 * 16;
    return r16 < 64 ? r16 : 64;
}

void make_l2p_images(const float *etab, int e, int n, uint16_t *img, cudaStream_t st) {
    const int N = l2p_tile_n(e), ntiles = (e * e * e + N - 1) / N;
    const size_t total = (size_t)ntiles * N * TCK;
    launch_pdl(k_l2p_image, (unsigned)((total + 255) / 256), 256, 0, st, etab, e, n, N, ntiles, img);
}

size_t l2p_image_elems(int e) {
    const int N = l2p_tile_n(e), ntiles = (e * e * e + N - 1) / N;
    return (size_t)ntiles * 2 * N * TCK;
}

__global__ void __launch_bounds__(128) k_l2p_tc(FmmDev F, int level, int box_begin, int box_count,
                                                const uint16_t *__restrict__ img, float *__restrict__ out,
                                                int *err) {
    pdl_enter();
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *a_hi = base, *a_lo = base + L2P_A, *b_hi = base + 2 * L2P_A, *b_lo = b_hi + L2P_B;
    uint8_t *tail = base + 2 * L2P_A + 2 * L2P_B;
    uint64_t *bar_b = reinterpret_cast<uint64_t *>(tail);
    uint64_t *bar_mma = bar_b + 1;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(tail + 16);
    int *ok_s = reinterpret_cast<int *>(tail + 20);
    int *sbox = reinterpret_cast<int *>(tail + 64);
    int *sfull = sbox + TCM;
    const TreeDev &T = F.T;
    const int r = threadIdx.x, warp = r >> 5;
    const int e = 1 << (F.D - level), rows = e * e * e;
    const int N = l2p_tile_n(e), ntiles = (rows + N - 1) / N;
    const int i = blockIdx.x * TCM + r;
    const int b = box_begin + i;
    bool ok = false;
    if (i < box_count) ok = T.b_leaf[b] && T.b_te[b] > T.b_tb[b];
    sbox[r] = ok ? b : -1;
    sfull[r] = ok && (T.b_te[b] - T.b_tb[b] == rows);
    if (!__syncthreads_or(ok)) return;
    if (r < 32) {
        tc::tmem_alloc(tc::smem_u32(tslot), 64);
        tc::tmem_relinquish();
    }
    if (r == 0) {
        tc::mbar_init(tc::smem_u32(bar_b), 1);
        tc::mbar_init(tc::smem_u32(bar_mma), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // A: the 128 boxes' d (FP32 [npad]) split into BF16 hi / lo, K-major SW128
    gather_rows_split(a_hi, a_lo, sbox, TCM, F.dchk, F.O.npad);
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const int bb = sbox[r];
    const bool full = sfull[r] != 0;
    int bx = 0, by = 0, bz = 0;
    if (bb >= 0) {
        uint32_t ux, uy, uz;
        demorton3(T.b_key[bb], ux, uy, uz);
        bx = (int)ux * e; by = (int)uy * e; bz = (int)uz * e;
    }
    const uint32_t idesc = tc::idesc_bf16_f32(TCM, N);
    const bool vec4 = full && (e % 4) == 0 && (F.nx % 4) == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0;
    const uint32_t sa_hi = tc::smem_u32(a_hi), sa_lo = tc::smem_u32(a_lo);
    const uint32_t sb_hi = tc::smem_u32(b_hi), sb_lo = tc::smem_u32(b_lo);
    const uint32_t bbytes = (uint32_t)N * TCK * 2;
    for (int t = 0; t < ntiles; ++t) {
        if (r == 0) {
            const uint16_t *src = img + (size_t)t * 2 * N * TCK;
            tc::mbar_expect_tx(tc::smem_u32(bar_b), 2 * bbytes);
            tc::bulk_g2s(sb_hi, src, bbytes, tc::smem_u32(bar_b));
            tc::bulk_g2s(sb_lo, src + (size_t)N * TCK, bbytes, tc::smem_u32(bar_b));
            int good = tc::mbar_wait_bounded(tc::smem_u32(bar_b), t & 1, WAIT_LIMIT);
            if (good) {
                tc::fence_after_sync();
#pragma unroll
                for (int ks = 0; ks < TCK / 16; ++ks) {
                    const uint32_t ao = tc::sw128_offset(0, 16 * ks, TCM);
                    const uint32_t bo = tc::sw128_offset(0, 16 * ks, N);
                    tc::mma_bf16(tmem, tc::sdesc_sw128(sa_hi + ao), tc::sdesc_sw128(sb_hi + bo), idesc, ks > 0);
                    tc::mma_bf16(tmem, tc::sdesc_sw128(sa_hi + ao), tc::sdesc_sw128(sb_lo + bo), idesc, 1);
                    tc::mma_bf16(tmem, tc::sdesc_sw128(sa_lo + ao), tc::sdesc_sw128(sb_hi + bo), idesc, 1);
                }
                tc::mma_commit(tc::smem_u32(bar_mma));
                good = tc::mbar_wait_bounded(tc::smem_u32(bar_mma), t & 1, WAIT_LIMIT);
                if (!good) {
                    atomicOr(err, 8);
                    tc::mbar_wait_bounded(tc::smem_u32(bar_mma), t & 1, WAIT_LIMIT);
                }
            } else {
                atomicOr(err, 4);
                tc::mbar_wait_bounded(tc::smem_u32(bar_b), t & 1, WAIT_LIMIT);
            }
            *ok_s = good;
        }
        __syncthreads();
        if (!*ok_s) break;
        tc::fence_after_sync();
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (bb < 0) continue;
            if (vec4) {   // whole box, rows of 4k cells: one 16-byte store per 4 cells of a row
#pragma unroll
                for (int j = 0; j < 16; j += 4) {
                    const int c = t * N + c0 + j;
                    if (c >= rows) break;
                    const int x = bx + c % e, y = by + (c / e) % e, z = bz + c / (e * e);
                    const int64_t o = (int64_t)x + (int64_t)F.nx * ((int64_t)y + (int64_t)F.ny * z);
                    *reinterpret_cast<float4 *>(out + o) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                }
                continue;
            }
            // mask bytes first, then the stores (a byte load after a float store would wait for it)
            bool keep[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int c = t * N + c0 + j;
                const int x = bx + c % e, y = by + (c / e) % e, z = bz + c / (e * e);
                const bool inb = c < rows && (full || (x < F.nx && y < F.ny && z < F.nz));
                const int64_t o = (int64_t)x + (int64_t)F.nx * ((int64_t)y + (int64_t)F.ny * z);
                keep[j] = inb && (full || __ldg(F.tmask + o) != 0);
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int c = t * N + c0 + j;
                const int x = bx + c % e, y = by + (c / e) % e, z = bz + c / (e * e);
                if (keep[j]) out[(int64_t)x + (int64_t)F.nx * ((int64_t)y + (int64_t)F.ny * z)] = v[j];
            }
        }
        tc::fence_before_sync();
        __syncthreads();
    }
    if (r < 32) tc::tmem_dealloc(tmem, 64);
}

// ---------------------------------------------------------------- L2L + L2P, deepest level
// Where every box of the level is a leaf of edge 4, the last L2L and the L2P compose: for
// child c of parent P (cells j of the child, coefficients k)
//     S(j) = sum_k E[j][k] d_c[k] + sum_k (E L2L_c)[j][k] d_P[k],
// d_c the child's own local terms (M2L, P2L: its L2L never runs), d_P the parent's complete
// local expansion.  This kernel takes the second sum for every leaf of the level: one CTA takes
// 128 parents (M = 128, TMEM lane = parent) and all 8 children, child c accumulating its 64
// cells in TMEM columns [64c, 64c + 64) from one K = 128 contraction (parent x composed
// table), BF16 hi / lo x3, and stores S at the child's targets.  The first sum is zero unless
// the child has V or X entries; k_l2p_own adds it for those leaves afterwards.
// The composed tables stream through two buffers: round g (child g mod 8 of the CTA's g / 8-th
// chunk) reads buffer g mod 2, and the table of round g + 2 is copied into it as soon as round
// g's MMAs have completed, so a copy has a whole round to land.  Child c's cells are written
// while child c+1's MMAs run.
constexpr uint32_t LP_A = TCM * TCK * 2;               // 32 KiB: 128 rows x 128 coefficients
constexpr uint32_t LP_B = 64 * TCK * 2;                // 16 KiB: 64 cells x 128 coefficients
constexpr int LP_T = 256;
constexpr int LP_V = TCM * (TCK / 4) / LP_T;           // float4 row segments per thread per tile (16)
constexpr uint32_t LP_SMEM = 1024 + 2 * LP_A + 4 * LP_B + 64 + 17 * TCM * 4;

// rows idx[0..128) of the FP32 state (-1: zero row), 16 float4 per thread, all in flight at once
__device__ __forceinline__ void lp_load(float4 (&v)[LP_V], const int *idx, const float *__restrict__ state, int np) {
#pragma unroll
    for (int u = 0; u < LP_V; ++u) {
        const int e = threadIdx.x + u * LP_T, j = e / (TCK / 4), q = e % (TCK / 4);
        const int src = idx[j];
        v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (src >= 0 && 4 * q < np) v[u] = __ldg(reinterpret_cast<const float4 *>(state + (size_t)src * np) + q);
    }
}
__device__ __forceinline__ void lp_store(uint8_t *hi, uint8_t *lo, const float4 (&v)[LP_V]) {
#pragma unroll
    for (int u = 0; u < LP_V; ++u) {
        const int e = threadIdx.x + u * LP_T;
        put_split4(hi, lo, e / (TCK / 4), 4 * (e % (TCK / 4)), TCM, v[u]);
    }
}

// One persistent CTA per SM: CTA b takes the chunks b, b + gridDim.x, ... of `ppc` parents
// each (the launch makes every CTA take the same number of chunks), so no SM runs an extra
// chunk while others idle.  The composed tables are the same for every chunk (table of round
// g: child g mod 8), so the copies run ahead across chunk boundaries; a chunk without leaves
// has no rounds.  Barrier phases run on across chunks: the k-th use of table buffer j waits on
// bar_t[j] with parity k & 1, the g-th round's MMAs complete bar_mma's phase g.
__global__ void __launch_bounds__(LP_T, 1) k_l2lp_tc(FmmDev F, int level, int parent_begin, int parent_count,
                                                     int ppc, int nchunks, const uint16_t *__restrict__ img_c,
                                                     float *__restrict__ out, int *err) {
    // prologue: tensor memory, barriers, the first two tables and the first chunk's tree
    // lookups; the wait comes before the first parent row is read
    if ((int)blockIdx.x >= nchunks) {              // uniform, before any allocation
        pdl_enter();
        return;
    }
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *ap_hi = base, *ap_lo = base + LP_A;
    uint8_t *tbuf = base + 2 * LP_A;                        // table buffer j: hi at tbuf + 2 j LP_B, lo after it
    uint8_t *tail = base + 2 * LP_A + 4 * LP_B;
    uint64_t *bar_t = reinterpret_cast<uint64_t *>(tail);   // [2]
    uint64_t *bar_mma = bar_t + 2;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(tail + 24);
    int *ok_s = reinterpret_cast<int *>(tail + 28);
    int *spar = reinterpret_cast<int *>(tail + 64);         // [128] parent box or -1
    int *sch = spar + TCM;                                  // [8][128] child box or -1
    int *sfull = sch + 8 * TCM;                             // [8][128] child has every cell as target
    const TreeDev &T = F.T;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int np = F.O.npad;
    const size_t img_elems = (size_t)2 * 64 * TCK;          // one image: hi then lo
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_u32(tslot), 512);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int k = 0; k < 3; ++k) tc::mbar_init(tc::smem_u32(bar_t + k), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *ok_s = 1;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    // thread 0's record of what is in flight, for a clean exit after a timeout: copies issued /
    // landed per table buffer (0, 1), MMA commits issued / completed
    int t_iss0 = 0, t_iss1 = 0, t_land0 = 0, t_land1 = 0, m_issued = 0, m_done = 0;
    auto copy_table = [&](int j, int child) {           // thread 0
        const uint32_t hi = tc::smem_u32(tbuf + 2 * (uint32_t)j * LP_B);
        tc::mbar_expect_tx(tc::smem_u32(bar_t + j), 2 * LP_B);
        const uint16_t *src = img_c + (size_t)child * img_elems;
        tc::bulk_g2s(hi, src, LP_B, tc::smem_u32(bar_t + j));
        tc::bulk_g2s(hi + LP_B, src + LP_B / 2, LP_B, tc::smem_u32(bar_t + j));
        if (j) ++t_iss1; else ++t_iss0;
    };
    if (tid == 0) {
        copy_table(0, 0);
        copy_table(1, 1);
    }
    float4 v[LP_V];
    const uint32_t idesc = tc::idesc_bf16_f32(TCM, 64);
    const int q = warp & 3, r = q * 32 + lane;              // TMEM lane quadrant, parent row
    const bool vec_ok = (F.nx % 4) == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0;
    // child c's cells: warps w and w + 4 share TMEM lanes 32 (w % 4) .. and take half of
    // the 64 columns each
    auto epilogue = [&](int c) {
        const int C = sch[c * TCM + r];
        const bool full = sfull[c * TCM + r] != 0;
        int bx = 0, by = 0, bz = 0;
        if (C >= 0) {
            uint32_t ux, uy, uz;
            demorton3(T.b_key[C], ux, uy, uz);
            bx = (int)ux * 4; by = (int)uy * 4; bz = (int)uz * 4;
        }
        float w[2][16];
#pragma unroll
        for (int h = 0; h < 2; ++h)
            tc::tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(64 * c + 32 * (warp >> 2) + 16 * h), w[h]);
        if (C < 0) return;
        const bool inside = bx + 4 <= F.nx && by + 4 <= F.ny && bz + 4 <= F.nz;
        if (vec_ok && inside) {
            // one 16-byte store per row of 4 cells; in a partly selected box the non-target
            // cells of a row get their zero in the same store (never a partial 32-byte sector,
            // which the memory system would have to merge), the row's 4 mask bytes read as one
            // word, every word before the first store
            uint32_t mw[2][4];
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int j = 0; j < 16; j += 4) {
                    const int cell = 32 * (warp >> 2) + 16 * h + j;
                    const int y = by + ((cell >> 2) & 3), z = bz + (cell >> 4);
                    const int64_t o = (int64_t)bx + (int64_t)F.nx * ((int64_t)y + (int64_t)F.ny * z);
                    mw[h][j >> 2] = full ? 0x01010101u : __ldg(reinterpret_cast<const uint32_t *>(F.tmask + o));
                }
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int j = 0; j < 16; j += 4) {
                    const int cell = 32 * (warp >> 2) + 16 * h + j;
                    const int y = by + ((cell >> 2) & 3), z = bz + (cell >> 4);
                    const int64_t o = (int64_t)bx + (int64_t)F.nx * ((int64_t)y + (int64_t)F.ny * z);
                    const uint32_t m = mw[h][j >> 2];
                    *reinterpret_cast<float4 *>(out + o) =
                        make_float4((m & 0xFFu) ? w[h][j] : 0.f, (m & 0xFF00u) ? w[h][j + 1] : 0.f,
                                    (m & 0xFF0000u) ? w[h][j + 2] : 0.f, (m & 0xFF000000u) ? w[h][j + 3] : 0.f);
                }
            return;
        }
        // partly selected or overhanging box: every mask byte is fetched before the first
        // store (a byte load placed after a float store would wait for it)
        bool keep[2][16];
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int cell = 32 * (warp >> 2) + 16 * h + j;
                const int x = bx + (cell & 3), y = by + ((cell >> 2) & 3), z = bz + (cell >> 4);
                const bool inb = full || (x < F.nx && y < F.ny && z < F.nz);   // box overhangs the grid
                const int64_t o = (int64_t)x + (int64_t)F.nx * ((int64_t)y + (int64_t)F.ny * z);
                keep[h][j] = inb && (full || __ldg(F.tmask + o) != 0);
            }
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int cell = 32 * (warp >> 2) + 16 * h + j;
                const int x = bx + (cell & 3), y = by + ((cell >> 2) & 3), z = bz + (cell >> 4);
                if (keep[h][j]) out[(int64_t)x + (int64_t)F.nx * ((int64_t)y + (int64_t)F.ny * z)] = w[h][j];
            }
    };
    int g = 0;                                              // rounds of this CTA so far
    bool waited = false;
    for (int chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
        const bool more = chunk + (int)gridDim.x < nchunks;   // this CTA has another chunk after this one
        __syncthreads();                                       // previous chunk's epilogue read sch / sfull
        int any = 0;
        if (tid < TCM) {
            const int i = chunk * ppc + tid;
            const int p = parent_begin + i;
            int P = -1;
            if (tid < ppc && i < parent_count && !T.b_leaf[p] && T.b_te[p] > T.b_tb[p]) P = p;
            spar[tid] = P;
            for (int c = 0; c < 8; ++c) {
                int C = -1, full = 0;
                if (P >= 0) {
                    const int ch = T.box_at[dense_off(level) + ((T.b_key[P] << 3) | (uint32_t)c)];
                    if (ch >= 0 && T.b_leaf[ch] && T.b_te[ch] > T.b_tb[ch]) {
                        C = ch;
                        full = T.b_te[ch] - T.b_tb[ch] == 64;
                    }
                }
                sch[c * TCM + tid] = C;
                sfull[c * TCM + tid] = full;
                any |= C >= 0;
            }
        }
        // a chunk without leaves has no rounds (the tables in flight serve the next chunk's)
        if (!__syncthreads_or(any)) continue;
        if (!waited) {
            pdl_enter();
            waited = true;
        }
        lp_load(v, spar, F.dchk, np);
        lp_store(ap_hi, ap_lo, v);
        bool ok = true;
#pragma unroll 1
        for (int c = 0; c < 8; ++c, ++g) {
            const int j = g & 1;
            // (a) the parent tile (written above) and table g are in shared memory: MMAs (thread
            //     0); the TMEM reads of earlier epilogues (the same columns in the previous
            //     chunk) are ordered before them
            tc::fence_proxy_async_smem();
            tc::fence_before_sync();
            __syncthreads();
            if (tid == 0 && *ok_s) {
                if (tc::mbar_wait_bounded(tc::smem_u32(bar_t + j), (g >> 1) & 1, WAIT_LIMIT)) {
                    if (j) ++t_land1; else ++t_land0;
                    tc::fence_after_sync();
                    const uint32_t d = tmem + (uint32_t)(64 * c);
                    const uint32_t aph = tc::smem_u32(ap_hi), apl = tc::smem_u32(ap_lo);
                    const uint32_t th = tc::smem_u32(tbuf + 2 * (uint32_t)j * LP_B), tl = th + LP_B;
#pragma unroll
                    for (int ks = 0; ks < TCK / 16; ++ks) {
                        const uint32_t ao = tc::sw128_offset(0, 16 * ks, TCM);
                        const uint32_t bo = tc::sw128_offset(0, 16 * ks, 64);
                        tc::mma_bf16(d, tc::sdesc_sw128(aph + ao), tc::sdesc_sw128(th + bo), idesc, ks > 0);
                        tc::mma_bf16(d, tc::sdesc_sw128(aph + ao), tc::sdesc_sw128(tl + bo), idesc, 1);
                        tc::mma_bf16(d, tc::sdesc_sw128(apl + ao), tc::sdesc_sw128(th + bo), idesc, 1);
                    }
                    tc::mma_commit(tc::smem_u32(bar_mma));
                    ++m_issued;
                    // (b) round g's MMAs complete: its table buffer is free for round g + 2's
                    //     table (this chunk's child c + 2, or the next chunk's first ones)
                    if (tc::mbar_wait_bounded(tc::smem_u32(bar_mma), g & 1, WAIT_LIMIT)) {
                        ++m_done;
                        if (c + 2 < 8 || more) copy_table(j, (c + 2) & 7);
                    } else {
                        atomicOr(err, 8);
                        *ok_s = 0;
                    }
                } else {
                    atomicOr(err, 4);
                    *ok_s = 0;
                }
            }
            // (c) child c-1's cells written while child c's MMAs run
            if (c > 0) epilogue(c - 1);
            __syncthreads();
            if (!*ok_s) {
                ok = false;
                break;
            }
            tc::fence_after_sync();
        }
        if (!ok) break;
        epilogue(7);
    }
    if (!waited) pdl_enter();                   // a CTA whose chunks had no leaves
    if (tid == 0) {
        // let this CTA's own copies and MMAs finish before its memory is released (after a
        // timeout, or copies issued for rounds of chunks that had no leaves)
        if (t_iss0 > t_land0) tc::mbar_wait_bounded(tc::smem_u32(bar_t), (t_iss0 - 1) & 1, WAIT_LIMIT);
        if (t_iss1 > t_land1) tc::mbar_wait_bounded(tc::smem_u32(bar_t + 1), (t_iss1 - 1) & 1, WAIT_LIMIT);
        if (m_issued > m_done) tc::mbar_wait_bounded(tc::smem_u32(bar_mma), (m_issued - 1) & 1, WAIT_LIMIT);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// S += E d_own at the targets of the deepest-level leaves (edge 4) in `list` (count[0] of them:
// the leaves with V or X entries, whose own local terms the fused kernel leaves out), FP32
// from the level's interpolation table E ([n][64], cells in local Morton order), staged in
// shared memory once per CTA.  One warp per leaf: lane k takes the cells of local index k and
// k + 32; every cell belongs to one leaf, so plain read-modify-writes suffice.  The next
// leaf's index and expansion are fetched while the current one is evaluated, and the current
// leaf's cell values (and mask bytes) are read before its contraction, so that a warp's
// loads overlap its arithmetic instead of following it.
constexpr int OWN_W = 8;
__global__ void __launch_bounds__(OWN_W * 32) k_l2p_own(FmmDev F, int level, const int *__restrict__ list,
                                                        const int *__restrict__ count, float *__restrict__ out) {
    pdl_enter();
    const int cnt = *count;
    if ((int)blockIdx.x * OWN_W >= cnt) return;            // uniform, before the table is staged
    __shared__ float Es[TCK * 64];                          // [n][64]
    __shared__ __align__(16) float sd[OWN_W][TCK];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = F.O.n, np = F.O.npad;
    const float4 *E4 = reinterpret_cast<const float4 *>(F.O.e_tab + F.O.e_off[level]);
    for (int j = threadIdx.x; j < n * 16; j += blockDim.x) reinterpret_cast<float4 *>(Es)[j] = __ldg(E4 + j);
    const TreeDev &T = F.T;
    const int stride = gridDim.x * OWN_W;
    int i = blockIdx.x * OWN_W + warp;
    const bool lane_d = 4 * lane < np;                      // np <= TCK = 128: one float4 per lane
    auto fetch_d = [&](int b) {
        return lane_d ? __ldg(reinterpret_cast<const float4 *>(F.dchk + (size_t)b * np) + lane)
                      : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    int bn = i < cnt ? list[i] : 0;
    float4 dn = i < cnt ? fetch_d(bn) : make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    for (; i < cnt; i += stride) {
        const int b = bn;
        if (lane_d) reinterpret_cast<float4 *>(sd[warp])[lane] = dn;
        if (i + stride < cnt) {
            bn = list[i + stride];
            dn = fetch_d(bn);
        }
        uint32_t ux, uy, uz;
        demorton3(T.b_key[b], ux, uy, uz);
        const bool full = T.b_te[b] - T.b_tb[b] == 64;
        int64_t o[2];
        bool keep[2];
        float old[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint32_t lx, ly, lz;
            demorton3((uint32_t)(lane + 32 * h), lx, ly, lz);
            const int x = (int)(ux * 4 + lx), y = (int)(uy * 4 + ly), z = (int)(uz * 4 + lz);
            keep[h] = x < F.nx && y < F.ny && z < F.nz;
            o[h] = keep[h] ? (int64_t)x + (int64_t)F.nx * ((int64_t)y + (int64_t)F.ny * z) : 0;
            keep[h] = keep[h] && (full || F.tmask[o[h]]);
            old[h] = keep[h] ? out[o[h]] : 0.f;
        }
        __syncwarp();
        float a0 = 0.f, a1 = 0.f;
#pragma unroll 5
        for (int k = 0; k < n; ++k) {
            const float dk = sd[warp][k];
            a0 = fmaf(Es[k * 64 + lane], dk, a0);
            a1 = fmaf(Es[k * 64 + lane + 32], dk, a1);
        }
        if (keep[0]) out[o[0]] = old[0] + a0;
        if (keep[1]) out[o[1]] = old[1] + a1;
        __syncwarp();
    }
}

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
    }
    return n;
}

void fmm_l2lp_tc_level(const FmmDev &F, int level, int parent_begin, int parent_count, float *out, int *err,
                       cudaStream_t st) {
    if (parent_count <= 0 || level < 3 || F.O.l2pc_off < 0 || F.O.l2p_off[level] < 0) return;
    tc_init_attributes();
    // one CTA per SM, each taking the same number k of chunks of up to 128 parents (the MMA's M)
    const int nsm = sm_count();
    const int k = std::max(1, (parent_count + TCM * nsm - 1) / (TCM * nsm));
    const int ppc = std::max(1, std::min(TCM, (parent_count + k * nsm - 1) / (k * nsm)));
    const int nchunks = (parent_count + ppc - 1) / ppc;
    const int grid = std::min(nchunks, nsm);
    launch_pdl(k_l2lp_tc, grid, LP_T, LP_SMEM, st, F, level, parent_begin, parent_count, ppc, nchunks,
                                                         F.O.l2p_img + F.O.l2pc_off, out, err);
}

void fmm_l2p_own(const FmmDev &F, int level, const int *list, const int *count, int max_count, float *out,
                 cudaStream_t st) {
    if (max_count <= 0 || F.O.e_off[level] < 0 || F.O.npad > TCK || (1 << (F.D - level)) != 4) return;
    const int grid = std::max(1, std::min((max_count + OWN_W - 1) / OWN_W, 4 * sm_count()));
    launch_pdl(k_l2p_own, grid, OWN_W * 32, 0, st, F, level, list, count, out);
}

bool tc_supported(const OpsDev &O) { return O.npad == TCK; }

// Opt in to the dynamic shared memory of the tensor-core kernels (host-side, once;
// called before any launch so that launches can be captured into a graph).
void tc_init_attributes() {
    static bool done = false;
    if (done) return;
    cudaFuncSetAttribute(k_m2l_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
    cudaFuncSetAttribute(k_m2l_tc_loop, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
    cudaFuncSetAttribute(k_l2l_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
    cudaFuncSetAttribute(k_m2m_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
    cudaFuncSetAttribute(k_l2l_tc8, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L8_SMEM);
    cudaFuncSetAttribute(k_l2p_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L2P_SMEM);
    cudaFuncSetAttribute(k_l2lp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LP_SMEM);
    cudaFuncSetAttribute(k_m2l_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MT_SMEM);
    cudaFuncSetAttribute(k_m2l_tc_pipe, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PIPE_SMEM);
    done = true;
}

size_t tc_image_elems(int count) { return (size_t)count * 2 * (A_BYTES / 2); }

void fmm_l2p_tc_level(const FmmDev &F, int level, int box_begin, int box_count, float *out, int *err,
                      cudaStream_t st) {
    if (box_count <= 0 || level < 2 || F.O.l2p_off[level] < 0) return;
    tc_init_attributes();
    launch_pdl(k_l2p_tc, (box_count + TCM - 1) / TCM, 128, L2P_SMEM, st, F, level, box_begin, box_count,
                                                                 F.O.l2p_img + F.O.l2p_off[level], out, err);
}

// ---------------------------------------------------------------- M2L, target-stationary tiles
// A work item is a group of up to 128 target boxes of one level and one octant (child index c
// within the parent: the 128 children c of 128 consecutive parent slots) and one of MT_P parts
// of the 216 = 6^3 positions around the parent.  Every box of the group has the same 189 V-list
// offsets (source minus target: o + c in [-2, 3] per axis, |o|_inf >= 2), so the MMA's columns
// are the group's boxes and its A operand the operator of one offset.  Per offset, the source of
// column j is the box at its key + o when that slot holds a box with sources (the V rule of the
// list kernel, by dense lookup), else a zero column.  The 128 x 128 result accumulates in TMEM
// over the item's offsets and is added into the boxes' rows once (reductions: the other parts
// and the X list add into the same rows).  Operators stream through two buffers (the copy of
// offset k+2 issued once MMA k has read its buffer); the gathered sources of offset k+1 are in
// registers while MMA k runs.  One persistent CTA per SM takes items from a counter.

__device__ __forceinline__ void mt_offset(int v, int c, int &ox, int &oy, int &oz) {
    ox = v % 6 - 2 - (c & 1);
    oy = (v / 6) % 6 - 2 - ((c >> 1) & 1);
    oz = v / 36 - 2 - (c >> 2);
}

// member j of group (l, tile, c): the child c of parent slot tile * 128 + j, if it holds
// targets and has V-list entries (its parent's 3^3 neighbourhood holds sources); else -1
__device__ __forceinline__ int mt_member(const FmmDev &F, int l, int tile, int c, int j) {
    const TreeDev &T = F.T;
    const int P = tile * TCM + j;
    if (P >= (1 << (3 * (l - 1))) || !T.near[dense_off(l - 1) + P]) return -1;
    const int b = T.box_at[dense_off(l) + ((uint32_t)P << 3 | (uint32_t)c)];
    if (b < 0 || T.b_te[b] <= T.b_tb[b] || F.L.v_cnt[b] <= 0) return -1;
    return b;
}

__global__ void __launch_bounds__(256) k_m2l_groups(FmmDev F, MtLevels ML, int *__restrict__ groups,
                                                    int *__restrict__ ngroups) {
    pdl_enter();
    const int g = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (g >= ML.gbase[ML.lmax + 1]) return;
    int l = ML.lmin;
    while (g >= ML.gbase[l + 1]) ++l;
    const int r = g - ML.gbase[l], tile = r >> 3, c = r & 7;
    bool any = false;
#pragma unroll
    for (int u = 0; u < TCM / 32; ++u) any |= mt_member(F, l, tile, c, lane + 32 * u) >= 0;
    if (__any_sync(0xffffffffu, any) && lane == 0) groups[atomicAdd(ngroups, 1)] = (l << 24) | (tile << 3) | c;
}

__global__ void __launch_bounds__(256, 1) k_m2l_tiles(FmmDev F, const int *__restrict__ groups,
                                                      const int *__restrict__ ngroups, int *__restrict__ counter,
                                                      const uint16_t *__restrict__ images, int *err) {
    pdl_enter();
    const int nitems = MT_P * *ngroups;
    if ((int)blockIdx.x >= nitems) return;         // uniform, before any allocation
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    // operator images at base + 2 A_BYTES buf (buf = 0, 1: hi then lo), then the gathered tile
    uint8_t *b_hi = base + 4 * A_BYTES, *b_lo = b_hi + A_BYTES;
    int *tab = reinterpret_cast<int *>(b_lo + A_BYTES);        // [MT_OFFS][128] source box or -1
    uint8_t *tail = reinterpret_cast<uint8_t *>(tab + MT_OFFS * TCM);
    uint64_t *bar_a = reinterpret_cast<uint64_t *>(tail);     // [2]
    uint64_t *bar_mma = bar_a + 2;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(tail + 24);
    int *ctl = reinterpret_cast<int *>(tail + 32);            // [0] item, [1] offsets, [2] ok
    int *mem = reinterpret_cast<int *>(tail + 64);            // [128] member box or -1
    int *offs = mem + TCM;                                    // [MT_OFFS] positions with a source
    int *oflag = offs + MT_OFFS;                              // [MT_OFFS]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int np = F.O.npad, n = F.O.n;
    const TreeDev &T = F.T;
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_u32(tslot), TCM);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int k = 0; k < 3; ++k) tc::mbar_init(tc::smem_u32(bar_a + k), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        ctl[2] = 1;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t idesc = tc::idesc_bf16_f32(TCM, TCM);
    // thread 0's barrier bookkeeping: completed waits per operator buffer and on the MMA barrier
    int a_done[2] = {0, 0}, a_iss[2] = {0, 0}, m_done = 0, m_iss = 0;
    float4 v[LP_V];
    auto issue_op = [&](int buf, int l, int c, int vpos) {
        int ox, oy, oz;
        mt_offset(vpos, c, ox, oy, oz);
        const uint16_t *img = images + (size_t)(l * NSLOT + m2l_slot(ox, oy, oz)) * (2 * A_BYTES / 2);
        tc::mbar_expect_tx(tc::smem_u32(bar_a + buf), 2 * A_BYTES);
        uint8_t *dst = base + 2 * A_BYTES * buf;
        tc::bulk_g2s(tc::smem_u32(dst), img, A_BYTES, tc::smem_u32(bar_a + buf));
        tc::bulk_g2s(tc::smem_u32(dst + A_BYTES), img + A_BYTES / 2, A_BYTES, tc::smem_u32(bar_a + buf));
        ++a_iss[buf];
    };
    while (true) {
        tc::fence_before_sync();                   // the previous item's TMEM reads
        __syncthreads();
        if (tid == 0) ctl[0] = atomicAdd(counter, 1);
        if (tid < MT_OFFS) oflag[tid] = 0;
        __syncthreads();
        const int item = ctl[0];
        if (item >= nitems || !ctl[2]) break;
        const int g = groups[item / MT_P], part = item % MT_P;
        const int l = g >> 24, tile = (g >> 3) & 0x1FFFFF, c = g & 7;
        if (tid < TCM) mem[tid] = mt_member(F, l, tile, c, tid);
        __syncthreads();
        // sources of every (position, member) of this part, by dense lookup
        const int edge = 1 << l;
        const uint8_t *vs = T.vsrc + dense_off(l);
        const int *ba = T.box_at + dense_off(l);
        // a thread's 27 lookups are independent: every slot is computed first, then both loads of
        // every lookup are issued before any is used (one round trip instead of 27)
        {
            constexpr int PER = MT_OFFS * TCM / 256;           // 27
            const int j = tid % TCM;                           // the same member in every lookup
            const int mj = mem[j];
            uint32_t bx = 0, by = 0, bz = 0;
            demorton3((uint32_t)(tile * TCM + j) << 3 | (uint32_t)c, bx, by, bz);
            int slot[PER];
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                const int vi = (tid + 256 * u) / TCM;
                int ox, oy, oz;
                mt_offset(part * MT_OFFS + vi, c, ox, oy, oz);
                const int sx = (int)bx + ox, sy = (int)by + oy, sz = (int)bz + oz;
                const bool ok = mj >= 0 && !(abs(ox) <= 1 && abs(oy) <= 1 && abs(oz) <= 1) && sx >= 0 && sy >= 0 &&
                                sz >= 0 && sx < edge && sy < edge && sz < edge;
                slot[u] = ok ? (int)morton3((uint32_t)sx, (uint32_t)sy, (uint32_t)sz) : -1;
            }
            uint8_t has[PER];
            int box[PER];
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                has[u] = slot[u] >= 0 ? __ldg(vs + slot[u]) : (uint8_t)0;
                box[u] = slot[u] >= 0 ? __ldg(ba + slot[u]) : -1;
            }
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                const int e = tid + 256 * u;
                const int A = has[u] ? box[u] : -1;
                tab[e] = A;
                if (A >= 0) oflag[e / TCM] = 1;
            }
        }
        __syncthreads();
        if (tid == 0) {
            int k = 0;
            for (int vi = 0; vi < MT_OFFS; ++vi)
                if (oflag[vi]) offs[k++] = vi;
            ctl[1] = k;
        }
        __syncthreads();
        const int n_off = ctl[1];
        if (n_off == 0) continue;
        if (tid == 0) {
            issue_op(0, l, c, part * MT_OFFS + offs[0]);
            if (n_off > 1) issue_op(1, l, c, part * MT_OFFS + offs[1]);
        }
        lp_load(v, tab + offs[0] * TCM, F.ueq, np);
        lp_store(b_hi, b_lo, v);
        for (int k = 0; k < n_off; ++k) {
            // (a) the gathered sources of offset k are in shared memory: MMAs (thread 0)
            tc::fence_proxy_async_smem();
            tc::fence_before_sync();
            __syncthreads();
            const int buf = k & 1;
            if (tid == 0 && ctl[2]) {
                if (tc::mbar_wait_bounded(tc::smem_u32(bar_a + buf), a_done[buf] & 1, WAIT_LIMIT)) {
                    ++a_done[buf];
                    tc::fence_after_sync();
                    const uint32_t ah = tc::smem_u32(base + 2 * A_BYTES * buf), al = ah + A_BYTES;
                    const uint32_t bh = tc::smem_u32(b_hi), bl = tc::smem_u32(b_lo);
#pragma unroll
                    for (int ks = 0; ks < TCK / 16; ++ks) {
                        const uint32_t o = tc::sw128_offset(0, 16 * ks, TCM);
                        tc::mma_bf16(tmem, tc::sdesc_sw128(ah + o), tc::sdesc_sw128(bh + o), idesc, (k | ks) > 0);
                        tc::mma_bf16(tmem, tc::sdesc_sw128(ah + o), tc::sdesc_sw128(bl + o), idesc, 1);
                        tc::mma_bf16(tmem, tc::sdesc_sw128(al + o), tc::sdesc_sw128(bh + o), idesc, 1);
                    }
                    tc::mma_commit(tc::smem_u32(bar_mma));
                    ++m_iss;
                } else {
                    atomicOr(err, 16);
                    ctl[2] = 0;
                }
            }
            // (b) the sources of offset k+1 in flight while the MMAs run
            if (k + 1 < n_off) lp_load(v, tab + offs[k + 1] * TCM, F.ueq, np);
            // (c) MMAs of offset k complete: the B tile and operator buffer k % 2 are free; the
            //     operator of offset k+2 streams into that buffer
            if (tid == 0 && ctl[2]) {
                if (tc::mbar_wait_bounded(tc::smem_u32(bar_mma), m_done & 1, WAIT_LIMIT)) {
                    ++m_done;
                    if (k + 2 < n_off) issue_op(buf, l, c, part * MT_OFFS + offs[k + 2]);
                } else {
                    atomicOr(err, 32);
                    ctl[2] = 0;
                }
            }
            __syncthreads();
            if (!ctl[2]) break;
            tc::fence_after_sync();
            // (e) the B tile of offset k+1
            if (k + 1 < n_off) lp_store(b_hi, b_lo, v);
        }
        if (!ctl[2]) break;
        // the accumulated check potentials into the members' rows: warps w and w + 4 read TMEM
        // lanes 32 (w % 4) .. (rows i) and half of the 128 columns each, staged as one FP32 row
        // per member in the operator buffers (free: every MMA and copy of the item has completed),
        // each row added into the member's downward state by one bulk reduction
        const int q = warp & 3, i = q * 32 + lane;
        float *stg = reinterpret_cast<float *>(base);      // [128 members][TCK]
#pragma unroll 1
        for (int c0 = (warp >> 2) * 64; c0 < (warp >> 2) * 64 + 64; c0 += 16) {
            float r[16];
            tc::tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, r);
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) stg[(c0 + jj) * TCK + i] = i < n ? r[jj] : 0.f;
        }
        tc::fence_proxy_async_smem();
        __syncthreads();
        if (tid < TCM) {
            const int d = mem[tid];
            if (d >= 0) {
                tc::bulk_reduce_add_f32(F.dchk + (size_t)d * np, tc::smem_u32(stg + tid * TCK), (uint32_t)np * 4u);
                tc::bulk_commit();
                tc::bulk_wait_read_all();   // before the next item's operators land in these buffers
            }
        }
    }
    if (tid == 0 && !ctl[2]) {
        // let this CTA's own copies and MMAs finish before its memory is released
        for (int b = 0; b < 2; ++b)
            if (a_iss[b] > a_done[b]) tc::mbar_wait_bounded(tc::smem_u32(bar_a + b), (a_iss[b] - 1) & 1, WAIT_LIMIT);
        if (m_iss > m_done) tc::mbar_wait_bounded(tc::smem_u32(bar_mma), (m_iss - 1) & 1, WAIT_LIMIT);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, TCM);
}

MtLevels m2l_tile_levels(int Lmax) {
    MtLevels ML{};
    ML.lmin = 2;
    ML.lmax = Lmax;
    int g = 0;
    for (int l = 0; l <= Lmax + 1 && l < 18; ++l) {
        ML.gbase[l] = g;
        if (l >= 2 && l <= Lmax) g += ((1 << (3 * (l - 1))) + TCM - 1) / TCM * 8;
    }
    return ML;
}

void fmm_m2l_tiles(const FmmDev &F, const MtLevels &ML, int *groups, int *ngroups, int *counter,
                   const uint16_t *images, int *err, cudaStream_t st) {
    if (ML.lmax < ML.lmin) return;
    tc_init_attributes();
    const int total = ML.gbase[ML.lmax + 1];
    launch_pdl(k_m2l_groups, (total + 7) / 8, 256, 0, st, F, ML, groups, ngroups);
    launch_pdl(k_m2l_tiles, sm_count(), 256, MT_SMEM, st, F, (const int *)groups, (const int *)ngroups, counter,
               images, err);
}

void fmm_m2l_tc(const FmmDev &F, const PairsDev &Pd, int nV, const uint16_t *images, int *err, cudaStream_t st,
                bool pipelined, bool tile_loop, int *ticket, int loop_ctas) {
    if (nV <= 0) return;
    tc_init_attributes();
    if (pipelined) {
        launch_pdl(k_m2l_tc_pipe, 152, 128, PIPE_SMEM, st, F, Pd, images, err);
        return;
    }
    if (tile_loop && ticket) {
        const int upper = (nV + TCN - 1) / TCN + Pd.nkeys;   // tiles at most
        const int ctas = loop_ctas > 0 ? loop_ctas : 2 * sm_count();
        launch_pdl(k_m2l_tc_loop, std::min(upper, ctas), 256, TC_SMEM, st, F, Pd, images, err, ticket);
        return;
    }
    int grid = (nV + TCN - 1) / TCN + Pd.nkeys;
    launch_pdl(k_m2l_tc, grid, 256, TC_SMEM, st, F, Pd, images, err);
}

void fmm_l2l_tc_level(const FmmDev &F, int level, int parent_begin, int parent_count, const uint16_t *images,
                      int *err, cudaStream_t st) {
    if (parent_count <= 0 || level < 3) return;
    tc_init_attributes();
    dim3 grid((parent_count + TCN - 1) / TCN, 8);
    launch_pdl(k_l2l_tc, grid, 256, TC_SMEM, st, F, level, parent_begin, parent_count, images, err);
}

}  // namespace sph
