// Kernels of the learned surrogate (see nn_kernels.cuh for layouts).
//
// k_conv_tc<C, N>: 3x3x3 convolution (forward, or data gradient with a flipped,
// transposed weight image) as an implicit GEMM on tcgen05.  One CTA (128 threads) per
// 128 output voxels; thread r gathers row r of the A tile (its voxel's 27 neighbours,
// 16-byte cp.async copies with zero fill outside the grid) one 64-element K chunk at a
// time into a 4-stage ring, and thread 0 issues 4 MMAs (M = 128, N, K = 16) per chunk
// two chunks behind the copies.  The FP32 accumulator (TMEM, 32 columns) is read back
// by the four warps (lane = voxel) and the epilogue adds bias, ReLU, a residual tensor
// and a ReLU mask before rounding to BF16.
//
// k_wgrad_tc<C, N>: the weight gradient dW[n][tap][c] = sum_m dz[m][n] x[m + off(tap)][c]
// as a GEMM whose reduction runs over voxels: M = (tap, c) rows in tiles of 128, N = out
// channels, K = voxels split across CTAs.  Both operands are transposed from the
// channels-last tensors while they are staged in shared memory; a constant-one row at
// tap 27 yields the bias gradient.  Partial tiles are added into FP32 with reductions.
//
// Every mbarrier wait is bounded; on expiry the kernel sets its error flag and carries
// on (the result is then invalid and the host reports it).
#include <math.h>

#include <algorithm>

#include "nn_kernels.cuh"
#include "tc_sm103.cuh"

namespace sph {
namespace nn {

using namespace tc;

constexpr int STAGES = 4, LAG = 2;
constexpr uint32_t A_STAGE = 128 * 128;     // 128 rows x 64 BF16
constexpr uint32_t NN_WAIT = 1u << 22;

__host__ __device__ constexpr uint32_t conv_smem(int N) { return 1024 + STAGES * (A_STAGE + N * 128) + 64; }
__host__ __device__ constexpr uint32_t wgrad_smem(int N) { return 1024 + 2 * (A_STAGE + N * 128) + 64; }

__device__ __forceinline__ uint8_t *align1024(uint8_t *p) {
    return reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(p) + 1023) & ~(uintptr_t)1023);
}

__device__ __forceinline__ void unpack8(const uint4 &q, float *f) {
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        f[2 * i] = __uint_as_float(w[i] << 16);
        f[2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
    }
}
__device__ __forceinline__ uint4 pack8(const float *f) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) w[i] = (uint32_t)f2bf(f[2 * i]) | ((uint32_t)f2bf(f[2 * i + 1]) << 16);
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// ---------------------------------------------------------------- convolution (forward / data gradient)
template <int C, int N>
__global__ void __launch_bounds__(128) k_conv_tc(ConvArgs a) {
    constexpr int T = 64 / C;                 // taps per K chunk
    constexpr int NCH = conv_chunks(C);
    constexpr int GPR = C / 8;                // 16-byte groups per tap
    constexpr uint32_t STAGE = A_STAGE + N * 128;
    extern __shared__ uint8_t raw[];
    uint8_t *base = align1024(raw);
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + STAGES * STAGE);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + STAGES);
    int *eflag = reinterpret_cast<int *>(tslot + 1);

    const int r = threadIdx.x;
    const int m = blockIdx.x * 128 + r;
    const bool valid = m < a.nvox;
    const int lg = a.lg, D = 1 << lg, dm = D - 1;
    const int x0 = m & dm, y0 = (m >> lg) & dm, z0 = (m >> (2 * lg)) & dm;

    if (r < 32) {
        tmem_alloc(smem_u32(tslot), 32);
        tmem_relinquish();
    }
    if (r == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(smem_u32(&bar[s]), 1);
        *eflag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t sbase = smem_u32(base);
    const uint32_t idesc = idesc_bf16_f32(128, N);

    for (int kc = 0; kc < NCH + LAG; ++kc) {
        if (kc < NCH) {
            const int s = kc % STAGES;
            if (kc >= STAGES && !mbar_wait_bounded(smem_u32(&bar[s]), ((kc / STAGES) - 1) & 1, NN_WAIT)) *eflag = 1;
            const uint32_t sa = sbase + s * STAGE, sb = sa + A_STAGE;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int tap = kc * T + u / GPR, cg = u % GPR;
                const void *src = a.x;
                uint32_t bytes = 0;
                if (valid && tap < NTAPS) {
                    const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
                    if ((unsigned)(x0 + dx) < (unsigned)D && (unsigned)(y0 + dy) < (unsigned)D &&
                        (unsigned)(z0 + dz) < (unsigned)D) {
                        src = a.x + (size_t)(m + (dz * D + dy) * D + dx) * C + cg * 8;
                        bytes = 16;
                    }
                }
                cp_async16(sa + r * 128 + ((u ^ (r & 7)) << 4), src, bytes);
            }
            const uint16_t *wsrc = a.w + (size_t)kc * N * 64;
#pragma unroll
            for (int i = r; i < N * 8; i += 128) cp_async16(sb + i * 16, wsrc + i * 8, 16);
        }
        cp_async_commit();
        if (kc >= LAG) {
            cp_async_wait<LAG>();
            fence_proxy_async_smem();
            __syncthreads();
            if (r == 0) {
                fence_after_sync();
                const int c = kc - LAG, s = c % STAGES;
                const uint32_t sa = sbase + s * STAGE, sb = sa + A_STAGE;
#pragma unroll
                for (int ks = 0; ks < 4; ++ks)
                    mma_bf16(tmem, sdesc_sw128(sa + 32 * ks), sdesc_sw128(sb + 32 * ks), idesc,
                             (c > 0 || ks > 0) ? 1u : 0u);
                mma_commit(smem_u32(&bar[s]));
            }
        }
    }
    // the last use of every stage (the final one covers every MMA)
#pragma unroll
    for (int s = 0; s < STAGES && s < NCH; ++s) {
        const int last = s + STAGES * ((NCH - 1 - s) / STAGES);
        if (!mbar_wait_bounded(smem_u32(&bar[s]), (last / STAGES) & 1, NN_WAIT)) *eflag = 1;
    }
    fence_after_sync();
    const int warp = r >> 5;
    float v[N];
    tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16), v);
    if constexpr (N == 32) tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + 16, v + 16);
    if (valid) {
        const size_t o = (size_t)m * N;
#pragma unroll
        for (int g = 0; g < N / 8; ++g) {
            float f[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                float x = v[8 * g + j];
                if (a.bias) x += a.bias[8 * g + j];
                if (a.relu) x = fmaxf(x, 0.f);
                f[j] = x;
            }
            if (a.add) {
                float ad[8];
                unpack8(*reinterpret_cast<const uint4 *>(a.add + o + 8 * g), ad);
#pragma unroll
                for (int j = 0; j < 8; ++j) f[j] += ad[j];
            }
            if (a.mask) {
                float mk[8];
                unpack8(*reinterpret_cast<const uint4 *>(a.mask + o + 8 * g), mk);
#pragma unroll
                for (int j = 0; j < 8; ++j) f[j] = mk[j] > 0.f ? f[j] : 0.f;
            }
            *reinterpret_cast<uint4 *>(a.out + o + 8 * g) = pack8(f);
        }
    }
    fence_before_sync();
    __syncthreads();
    if (r == 0 && *eflag) atomicOr(a.err, 1);
    if (r < 32) tmem_dealloc(tmem, 32);
}

// ---------------------------------------------------------------- weight gradient
__device__ __forceinline__ uint4 load_tap(const uint16_t *__restrict__ x, int v, int nvox, int tap, int cg, int C,
                                          int lg) {
    if (v >= nvox) return make_uint4(0, 0, 0, 0);
    if (tap >= NTAPS) return make_uint4(tap == NTAPS && cg == 0 ? 0x3F80u : 0u, 0, 0, 0);   // bias row: 1.0
    const int D = 1 << lg, dm = D - 1;
    const int xv = v & dm, yv = (v >> lg) & dm, zv = (v >> (2 * lg)) & dm;
    const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
    if ((unsigned)(xv + dx) >= (unsigned)D || (unsigned)(yv + dy) >= (unsigned)D || (unsigned)(zv + dz) >= (unsigned)D)
        return make_uint4(0, 0, 0, 0);
    return __ldg(reinterpret_cast<const uint4 *>(x + (size_t)(v + (dz * D + dy) * D + dx) * C + cg * 8));
}

__device__ __forceinline__ void put_pair_rows(uint8_t *tile, int rows, int row0, int kp, const uint4 &q0,
                                              const uint4 &q1) {
    const uint16_t *h0 = reinterpret_cast<const uint16_t *>(&q0);
    const uint16_t *h1 = reinterpret_cast<const uint16_t *>(&q1);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const uint32_t word = (uint32_t)h0[j] | ((uint32_t)h1[j] << 16);
        *reinterpret_cast<uint32_t *>(tile + sw128_offset(row0 + j, 2 * kp, rows)) = word;
    }
}

template <int C, int N>
__global__ void __launch_bounds__(128) k_wgrad_tc(WgradArgs a) {
    constexpr int T = 128 / C;                // taps per M tile
    constexpr int GPR = C / 8;
    constexpr uint32_t STAGE = A_STAGE + N * 128;
    const int nchunks = (a.nvox + 63) / 64;
    const int c0 = blockIdx.y * a.chunks_per_cta;
    const int c1 = min(c0 + a.chunks_per_cta, nchunks);
    if (c0 >= c1) return;                     // uniform over the CTA, before any allocation
    extern __shared__ uint8_t raw[];
    uint8_t *base = align1024(raw);
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + 2 * STAGE);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 2);
    int *eflag = reinterpret_cast<int *>(tslot + 1);
    const int r = threadIdx.x;
    if (r < 32) {
        tmem_alloc(smem_u32(tslot), 32);
        tmem_relinquish();
    }
    if (r == 0) {
        mbar_init(smem_u32(&bar[0]), 1);
        mbar_init(smem_u32(&bar[1]), 1);
        *eflag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t idesc = idesc_bf16_f32(128, N);
    const int t0 = blockIdx.x * T;

    for (int c = c0; c < c1; ++c) {
        const int j = c - c0, s = j & 1;
        if (j >= 2 && !mbar_wait_bounded(smem_u32(&bar[s]), ((j >> 1) - 1) & 1, NN_WAIT)) *eflag = 1;
        uint8_t *ta = base + s * STAGE;
        uint8_t *tb = ta + A_STAGE;
        for (int e = r; e < T * GPR * 32; e += 128) {
            const int kp = e & 31, rest = e >> 5, cg = rest % GPR, tt = rest / GPR;
            const int v = c * 64 + 2 * kp;
            const uint4 q0 = load_tap(a.x, v, a.nvox, t0 + tt, cg, C, a.lg);
            const uint4 q1 = load_tap(a.x, v + 1, a.nvox, t0 + tt, cg, C, a.lg);
            put_pair_rows(ta, 128, tt * C + cg * 8, kp, q0, q1);
        }
        for (int e = r; e < (N / 8) * 32; e += 128) {
            const int kp = e & 31, ng = e >> 5;
            const int v = c * 64 + 2 * kp;
            const uint4 z = make_uint4(0, 0, 0, 0);
            const uint4 q0 = v < a.nvox ? __ldg(reinterpret_cast<const uint4 *>(a.dz + (size_t)v * N + ng * 8)) : z;
            const uint4 q1 =
                v + 1 < a.nvox ? __ldg(reinterpret_cast<const uint4 *>(a.dz + (size_t)(v + 1) * N + ng * 8)) : z;
            put_pair_rows(tb, N, ng * 8, kp, q0, q1);
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (r == 0) {
            fence_after_sync();
            const uint32_t sa = smem_u32(ta), sb = smem_u32(tb);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
                mma_bf16(tmem, sdesc_sw128(sa + 32 * ks), sdesc_sw128(sb + 32 * ks), idesc, (j > 0 || ks > 0) ? 1u : 0u);
            mma_commit(smem_u32(&bar[s]));
        }
    }
    const int count = c1 - c0;
    for (int s = 0; s < 2 && s < count; ++s) {
        const int last = s + 2 * ((count - 1 - s) / 2);
        if (!mbar_wait_bounded(smem_u32(&bar[s]), (last >> 1) & 1, NN_WAIT)) *eflag = 1;
    }
    fence_after_sync();
    const int warp = r >> 5;
    float v[N];
    tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16), v);
    if constexpr (N == 32) tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + 16, v + 16);
    if (a.part) {   // this CTA's partial, summed with the others' in a fixed order by k_wgrad_sum
        const size_t rows = (size_t)gridDim.x * 128;
        float4 *dst = reinterpret_cast<float4 *>(a.part + ((size_t)blockIdx.y * rows + blockIdx.x * 128 + r) * N);
#pragma unroll
        for (int n = 0; n < N; n += 4) dst[n / 4] = make_float4(v[n], v[n + 1], v[n + 2], v[n + 3]);
    } else {
        float *dst = a.dw + (size_t)(blockIdx.x * 128 + r) * N;
#pragma unroll
        for (int n = 0; n < N; ++n) atomicAdd(dst + n, v[n]);
    }
    fence_before_sync();
    __syncthreads();
    if (r == 0 && *eflag) atomicOr(a.err, 1);
    if (r < 32) tmem_dealloc(tmem, 32);
}

// dw[e] += sum over the splits y = 0, 1, ... of part[y][e], in that order
__global__ void k_wgrad_sum(const float *__restrict__ part, float *__restrict__ dw, int elems, int splits) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= elems) return;
    float acc = dw[e];
    for (int y = 0; y < splits; ++y) acc += part[(size_t)y * elems + e];
    dw[e] = acc;
}

template <int C, int N>
static void set_attrs() {
    cudaFuncSetAttribute(k_conv_tc<C, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, conv_smem(N));
    cudaFuncSetAttribute(k_wgrad_tc<C, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, wgrad_smem(N));
}

void init_attributes() {
    static bool done = false;
    if (done) return;
    set_attrs<16, 16>();
    set_attrs<16, 32>();
    set_attrs<32, 16>();
    set_attrs<32, 32>();
    done = true;
}

template <int C, int N>
static void launch_conv(const ConvArgs &a, cudaStream_t st) {
    const int grid = (a.nvox + 127) / 128;
    if (grid > 0) k_conv_tc<C, N><<<grid, 128, conv_smem(N), st>>>(a);
}

int conv(const ConvArgs &a, int C, int N, cudaStream_t st) {
    if (C == 16 && N == 16) launch_conv<16, 16>(a, st);
    else if (C == 16 && N == 32) launch_conv<16, 32>(a, st);
    else if (C == 32 && N == 16) launch_conv<32, 16>(a, st);
    else if (C == 32 && N == 32) launch_conv<32, 32>(a, st);
    else return -1;
    return 0;
}

template <int C, int N>
static void launch_wgrad(WgradArgs a, cudaStream_t st) {
    const int mtiles = wgrad_rows(C) / 128;
    const int nchunks = (a.nvox + 63) / 64;
    if (nchunks == 0) return;
    const int target = 4 * 152;
    int cpc = (nchunks * mtiles + target - 1) / target;
    if (cpc < 4) cpc = 4;
    if (a.part) cpc = std::max(cpc, (nchunks + WGRAD_MAX_SPLIT - 1) / WGRAD_MAX_SPLIT);   // splits fit the scratch
    a.chunks_per_cta = cpc;
    dim3 grid(mtiles, (nchunks + cpc - 1) / cpc);
    k_wgrad_tc<C, N><<<grid, 128, wgrad_smem(N), st>>>(a);
    if (a.part) {
        const int elems = wgrad_rows(C) * N;
        k_wgrad_sum<<<(elems + 255) / 256, 256, 0, st>>>(a.part, a.dw, elems, (int)grid.y);
    }
}

int wgrad(const WgradArgs &a, int C, int N, cudaStream_t st) {
    if (C == 16 && N == 16) launch_wgrad<16, 16>(a, st);
    else if (C == 16 && N == 32) launch_wgrad<16, 32>(a, st);
    else if (C == 32 && N == 16) launch_wgrad<32, 16>(a, st);
    else if (C == 32 && N == 32) launch_wgrad<32, 32>(a, st);
    else return -1;
    return 0;
}

// ---------------------------------------------------------------- resampling and element-wise
// index of the fine voxel (child ci of coarse voxel p), both grids [B][D^3], D_fine = 2 D_coarse
__device__ __forceinline__ size_t child_of(size_t p, int lgc, int ci) {
    const int Dc = 1 << lgc, dm = Dc - 1;
    const size_t b = p >> (3 * lgc);
    const int x = (int)(p & dm), y = (int)((p >> lgc) & dm), z = (int)((p >> (2 * lgc)) & dm);
    const int lgf = lgc + 1;
    const int fx = 2 * x + (ci & 1), fy = 2 * y + ((ci >> 1) & 1), fz = 2 * z + (ci >> 2);
    return (b << (3 * lgf)) + ((size_t)fz << (2 * lgf)) + ((size_t)fy << lgf) + fx;
}
__device__ __forceinline__ size_t parent_of(size_t q, int lgf) {
    const int Df = 1 << lgf, dm = Df - 1;
    const size_t b = q >> (3 * lgf);
    const int x = (int)(q & dm), y = (int)((q >> lgf) & dm), z = (int)((q >> (2 * lgf)) & dm);
    const int lgc = lgf - 1;
    return (b << (3 * lgc)) + ((size_t)(z >> 1) << (2 * lgc)) + ((size_t)(y >> 1) << lgc) + (x >> 1);
}

__global__ void k_pool2(const uint16_t *__restrict__ in, uint16_t *__restrict__ out, size_t nout, int lgc, int C) {
    const int G = C / 8;
    const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (e >= nout * G) return;
    const size_t p = e / G;
    const int g = (int)(e % G);
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int ci = 0; ci < 8; ++ci) {
        float f[8];
        unpack8(__ldg(reinterpret_cast<const uint4 *>(in + child_of(p, lgc, ci) * C + 8 * g)), f);
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j] += f[j];
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] *= 0.125f;
    *reinterpret_cast<uint4 *>(out + p * C + 8 * g) = pack8(acc);
}

__global__ void k_up_add(const uint16_t *__restrict__ coarse, const uint16_t *__restrict__ skip,
                         uint16_t *__restrict__ out, size_t nout, int lgf, int C) {
    const int G = C / 8;
    const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (e >= nout * G) return;
    const size_t q = e / G;
    const int g = (int)(e % G);
    float f[8];
    unpack8(__ldg(reinterpret_cast<const uint4 *>(coarse + parent_of(q, lgf) * C + 8 * g)), f);
    if (skip) {
        float s[8];
        unpack8(__ldg(reinterpret_cast<const uint4 *>(skip + q * C + 8 * g)), s);
#pragma unroll
        for (int j = 0; j < 8; ++j) f[j] += s[j];
    }
    *reinterpret_cast<uint4 *>(out + q * C + 8 * g) = pack8(f);
}

__global__ void k_add(const uint16_t *__restrict__ a, const uint16_t *__restrict__ b, uint16_t *__restrict__ out,
                      size_t n8) {
    const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (e >= n8) return;
    float x[8], y[8];
    unpack8(__ldg(reinterpret_cast<const uint4 *>(a) + e), x);
    unpack8(__ldg(reinterpret_cast<const uint4 *>(b) + e), y);
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] += y[j];
    reinterpret_cast<uint4 *>(out)[e] = pack8(x);
}

__global__ void k_mask_mul(const uint16_t *__restrict__ g, const uint16_t *__restrict__ mask,
                           uint16_t *__restrict__ out, size_t n8) {
    const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (e >= n8) return;
    float x[8], m[8];
    unpack8(__ldg(reinterpret_cast<const uint4 *>(g) + e), x);
    unpack8(__ldg(reinterpret_cast<const uint4 *>(mask) + e), m);
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = m[j] > 0.f ? x[j] : 0.f;
    reinterpret_cast<uint4 *>(out)[e] = pack8(x);
}

__global__ void k_up_back_mask(const uint16_t *__restrict__ gf, const uint16_t *__restrict__ mask,
                               uint16_t *__restrict__ out, size_t nout, int lgc, int C) {
    const int G = C / 8;
    const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (e >= nout * G) return;
    const size_t p = e / G;
    const int g = (int)(e % G);
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int ci = 0; ci < 8; ++ci) {
        float f[8];
        unpack8(__ldg(reinterpret_cast<const uint4 *>(gf + child_of(p, lgc, ci) * C + 8 * g)), f);
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j] += f[j];
    }
    float m[8];
    unpack8(__ldg(reinterpret_cast<const uint4 *>(mask + p * C + 8 * g)), m);
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = m[j] > 0.f ? acc[j] : 0.f;
    *reinterpret_cast<uint4 *>(out + p * C + 8 * g) = pack8(acc);
}

__global__ void k_pool_back_add_mask(const uint16_t *__restrict__ gc, const uint16_t *__restrict__ add,
                                     const uint16_t *__restrict__ mask, uint16_t *__restrict__ out, size_t nout,
                                     int lgf, int C) {
    const int G = C / 8;
    const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (e >= nout * G) return;
    const size_t q = e / G;
    const int g = (int)(e % G);
    float f[8], ad[8], m[8];
    unpack8(__ldg(reinterpret_cast<const uint4 *>(gc + parent_of(q, lgf) * C + 8 * g)), f);
    unpack8(__ldg(reinterpret_cast<const uint4 *>(add + q * C + 8 * g)), ad);
    unpack8(__ldg(reinterpret_cast<const uint4 *>(mask + q * C + 8 * g)), m);
#pragma unroll
    for (int j = 0; j < 8; ++j) f[j] = m[j] > 0.f ? ad[j] + 0.125f * f[j] : 0.f;
    *reinterpret_cast<uint4 *>(out + q * C + 8 * g) = pack8(f);
}

static unsigned blocks_for(size_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

void pool2(const uint16_t *in, uint16_t *out, int B, int lg_out, int C, cudaStream_t st) {
    const size_t n = (size_t)B << (3 * lg_out);
    if (n) k_pool2<<<blocks_for(n * (C / 8)), 256, 0, st>>>(in, out, n, lg_out, C);
}
void up_add(const uint16_t *coarse, const uint16_t *skip, uint16_t *out, int B, int lg_out, int C, cudaStream_t st) {
    const size_t n = (size_t)B << (3 * lg_out);
    if (n) k_up_add<<<blocks_for(n * (C / 8)), 256, 0, st>>>(coarse, skip, out, n, lg_out, C);
}
void add(const uint16_t *a, const uint16_t *b, uint16_t *out, size_t n, cudaStream_t st) {
    if (n) k_add<<<blocks_for(n / 8), 256, 0, st>>>(a, b, out, n / 8);
}
void mask_mul(const uint16_t *g, const uint16_t *mask, uint16_t *out, size_t n, cudaStream_t st) {
    if (n) k_mask_mul<<<blocks_for(n / 8), 256, 0, st>>>(g, mask, out, n / 8);
}
void up_back_mask(const uint16_t *g_fine, const uint16_t *mask, uint16_t *out, int B, int lg_out, int C,
                  cudaStream_t st) {
    const size_t n = (size_t)B << (3 * lg_out);
    if (n) k_up_back_mask<<<blocks_for(n * (C / 8)), 256, 0, st>>>(g_fine, mask, out, n, lg_out, C);
}
void pool_back_add_mask(const uint16_t *g_coarse, const uint16_t *addt, const uint16_t *mask, uint16_t *out, int B,
                        int lg_out, int C, cudaStream_t st) {
    const size_t n = (size_t)B << (3 * lg_out);
    if (n) k_pool_back_add_mask<<<blocks_for(n * (C / 8)), 256, 0, st>>>(g_coarse, addt, mask, out, n, lg_out, C);
}

// ---------------------------------------------------------------- head and loss (FP32)
__global__ void k_head_forward(const uint16_t *__restrict__ f, const float *__restrict__ hw,
                               const float *__restrict__ hb, float *__restrict__ y, int nvox) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= nvox) return;
    float a[16];
    unpack8(__ldg(reinterpret_cast<const uint4 *>(f + (size_t)m * 16)), a);
    unpack8(__ldg(reinterpret_cast<const uint4 *>(f + (size_t)m * 16 + 8)), a + 8);
    float r = hb[0], e = hb[1];
#pragma unroll
    for (int c = 0; c < 16; ++c) {
        r = fmaf(hw[c], a[c], r);
        e = fmaf(hw[16 + c], a[c], e);
    }
    y[2 * (size_t)m] = r;
    y[2 * (size_t)m + 1] = e;
}

__global__ void k_head_loss_backward(const uint16_t *__restrict__ f, const float *__restrict__ hw,
                                     const float *__restrict__ hb, const float *__restrict__ t,
                                     uint16_t *__restrict__ g_f, float *__restrict__ hg, double *loss_sum, int nvox,
                                     float lambda, float eps, float *__restrict__ hpart) {
    __shared__ float wsum[8][34];
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const bool ok = m < nvox;
    float a[16];
    float gr = 0.f, ge = 0.f, li = 0.f;
    if (ok) {
        unpack8(__ldg(reinterpret_cast<const uint4 *>(f + (size_t)m * 16)), a);
        unpack8(__ldg(reinterpret_cast<const uint4 *>(f + (size_t)m * 16 + 8)), a + 8);
        float r = hb[0], e = hb[1];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            r = fmaf(hw[c], a[c], r);
            e = fmaf(hw[16 + c], a[c], e);
        }
        const float d = r - t[m];
        const float le = logf(fabsf(d) + eps);
        const float inv = 1.0f / (float)nvox;
        li = d * d + lambda * (e - le) * (e - le);
        gr = 2.f * d * inv;
        ge = 2.f * lambda * (e - le) * inv;
        float g[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) g[c] = a[c] > 0.f ? fmaf(hw[c], gr, hw[16 + c] * ge) : 0.f;
        *reinterpret_cast<uint4 *>(g_f + (size_t)m * 16) = pack8(g);
        *reinterpret_cast<uint4 *>(g_f + (size_t)m * 16 + 8) = pack8(g + 8);
    } else {
#pragma unroll
        for (int c = 0; c < 16; ++c) a[c] = 0.f;
    }
    // head gradient: hg[j*16 + c] += g_j f_c, hg[32 + j] += g_j (warp sums, then one reduction per warp)
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 34; ++k) {
        float x = k < 16 ? gr * a[k] : (k < 32 ? ge * a[k - 16] : (k == 32 ? gr : ge));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (hpart) {
            if (lane == 0) wsum[threadIdx.x >> 5][k] = x;
        } else if (lane == 0 && x != 0.f) {
            atomicAdd(hg + k, x);
        }
    }
    if (hpart) {   // the block's partial (its warps in order); summed over the blocks in order later
        __syncthreads();
        if (threadIdx.x < 34) {
            float b = 0.f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += wsum[w][threadIdx.x];
            hpart[(size_t)blockIdx.x * 34 + threadIdx.x] = b;
        }
    }
    double ld = li;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ld += __shfl_down_sync(0xffffffffu, ld, o);
    if (lane == 0) atomicAdd(loss_sum, ld);
}

void head_forward(const uint16_t *f, const float *hw, const float *hb, float *y, int nvox, cudaStream_t st) {
    if (nvox > 0) k_head_forward<<<blocks_for(nvox), 256, 0, st>>>(f, hw, hb, y, nvox);
}
// hg[k] += sum over the blocks b = 0, 1, ... of hpart[b][k], in that order
__global__ void k_head_sum(const float *__restrict__ hpart, float *__restrict__ hg, int nblocks) {
    const int k = threadIdx.x;
    if (k >= 34) return;
    float acc = hg[k];
    for (int b = 0; b < nblocks; ++b) acc += hpart[(size_t)b * 34 + k];
    hg[k] = acc;
}

void head_loss_backward(const uint16_t *f, const float *hw, const float *hb, const float *t, uint16_t *g_f,
                        float *hg, double *loss_sum, int nvox, float lambda, float eps, cudaStream_t st,
                        float *hpart) {
    if (nvox <= 0) return;
    const int nb = blocks_for(nvox);
    if (nb > HEAD_MAX_BLOCKS) hpart = nullptr;   // beyond the scratch: reductions
    k_head_loss_backward<<<nb, 256, 0, st>>>(f, hw, hb, t, g_f, hg, loss_sum, nvox, lambda, eps, hpart);
    if (hpart) k_head_sum<<<1, 64, 0, st>>>(hpart, hg, nb);
}

// ---------------------------------------------------------------- parameters
__global__ void k_collect_grads(const float *__restrict__ dw, int C, int N, float *__restrict__ g) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int nw = N * NTAPS * C;
    if (i >= nw + N) return;
    if (i < nw) {
        const int n = i / (NTAPS * C), rem = i % (NTAPS * C), tap = rem / C, c = rem % C;
        g[i] = dw[(size_t)(tap * C + c) * N + n];
    } else {
        g[i] = dw[(size_t)(NTAPS * C) * N + (i - nw)];
    }
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, size_t n, float lr, float b1, float b2, float eps, float bc1, float bc2) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

__global__ void k_images(const float *__restrict__ w, int C, int N, uint16_t *__restrict__ img_f,
                         uint16_t *__restrict__ img_d, int nf, int nd) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nf) {
        const int kc = i / (N * 64), within = i % (N * 64), n = within / 64, kk = within % 64;
        const int k = kc * 64 + kk, tap = k / C, c = k % C;
        const float val = tap < NTAPS ? w[(size_t)(n * NTAPS + tap) * C + c] : 0.f;
        img_f[(size_t)kc * N * 64 + n * 64 + (((kk >> 3) ^ (n & 7)) << 3) + (kk & 7)] = f2bf(val);
    } else if (i < nf + nd) {
        const int j = i - nf;
        const int kc = j / (C * 64), within = j % (C * 64), n = within / 64, kk = within % 64;
        const int k = kc * 64 + kk, tap = k / N, co = k % N;
        const float val = tap < NTAPS ? w[(size_t)(co * NTAPS + (NTAPS - 1 - tap)) * C + n] : 0.f;
        img_d[(size_t)kc * C * 64 + n * 64 + (((kk >> 3) ^ (n & 7)) << 3) + (kk & 7)] = f2bf(val);
    }
}

__global__ void k_f32_to_bf16(const float *__restrict__ in, uint16_t *__restrict__ out, size_t n) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = f2bf(in[i]);
}

void collect_grads(const float *dw, int C, int N, float *g, cudaStream_t st) {
    k_collect_grads<<<blocks_for((size_t)N * NTAPS * C + N), 256, 0, st>>>(dw, C, N, g);
}
void adam(float *p, const float *g, float *m, float *v, size_t n, float lr, float b1, float b2, float eps, float bc1,
          float bc2, cudaStream_t st) {
    if (n) k_adam<<<blocks_for(n), 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, bc1, bc2);
}
void make_images(const float *w, int C, int N, uint16_t *img_fwd, uint16_t *img_dgrad, cudaStream_t st) {
    const int nf = conv_chunks(C) * N * 64;
    const int nd = img_dgrad ? conv_chunks(N) * C * 64 : 0;
    k_images<<<blocks_for((size_t)nf + nd), 256, 0, st>>>(w, C, N, img_fwd, img_dgrad, nf, nd);
}
void f32_to_bf16(const float *in, uint16_t *out, size_t n, cudaStream_t st) {
    if (n) k_f32_to_bf16<<<blocks_for(n), 256, 0, st>>>(in, out, n);
}

// ---------------------------------------------------------------- coarse inputs
__global__ void k_pool_avg_f32(const float *__restrict__ fine, int nf, int f, float *__restrict__ coarse) {
    const int nc = nf / f;
    const size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (p >= (size_t)nc * nc * nc) return;
    const int x = (int)(p % nc), y = (int)((p / nc) % nc), z = (int)(p / ((size_t)nc * nc));
    float s = 0.f;
    for (int k = 0; k < f; ++k)
        for (int j = 0; j < f; ++j) {
            const float *row = fine + ((size_t)(z * f + k) * nf + (y * f + j)) * nf + x * f;
            for (int i = 0; i < f; ++i) s += row[i];
        }
    coarse[p] = s / (float)(f * f * f);
}

__global__ void k_pool_max_f32(const float *__restrict__ fine, int nf, int f, float *__restrict__ coarse) {
    const int nc = nf / f;
    const size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (p >= (size_t)nc * nc * nc) return;
    const int x = (int)(p % nc), y = (int)((p / nc) % nc), z = (int)(p / ((size_t)nc * nc));
    float s = 0.f;
    for (int k = 0; k < f; ++k)
        for (int j = 0; j < f; ++j) {
            const float *row = fine + ((size_t)(z * f + k) * nf + (y * f + j)) * nf + x * f;
            for (int i = 0; i < f; ++i) s = fmaxf(s, row[i]);
        }
    coarse[p] = s;
}

// maxima of up to four non-negative fields (b, d may be null) as float bits
__global__ void k_max4(const float *__restrict__ a, const float *__restrict__ b, const float *__restrict__ c,
                       const float *__restrict__ d, size_t n, unsigned *maxbits) {
    float m[4] = {0.f, 0.f, 0.f, 0.f};
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        m[0] = fmaxf(m[0], a[i]);
        if (b) m[1] = fmaxf(m[1], b[i]);
        m[2] = fmaxf(m[2], c[i]);
        if (d) m[3] = fmaxf(m[3], d[i]);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m[k] = fmaxf(m[k], __shfl_down_sync(0xffffffffu, m[k], o));
    }
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < 4; ++k) atomicMax(maxbits + k, __float_as_uint(m[k]));
}

// channel 0: log10(I / max I + 1e-8) / 8 + 1 (I averaged over the coarse cell); channel 1:
// |E| / max |E|; channel 2: ln(S / max S + 1e-12) / ln(1e12) + 1 (coarse FMM estimate);
// channel 3: as channel 0 for the largest fine-cell I in the coarse cell (sub-cell peak);
// channels 4..15 zero
__global__ void k_make_inputs(const float *__restrict__ I, const float *__restrict__ E, const float *__restrict__ S,
                              const float *__restrict__ Imax, const unsigned *__restrict__ maxbits,
                              uint16_t *__restrict__ x, size_t n) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float mi = __uint_as_float(maxbits[0]), me = __uint_as_float(maxbits[1]), ms = __uint_as_float(maxbits[2]);
    const float mx = __uint_as_float(maxbits[3]);
    float f[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) f[c] = 0.f;
    f[0] = mi > 0.f ? fmaxf(0.f, log10f(I[i] / mi + 1e-8f) * 0.125f + 1.f) : 0.f;
    f[1] = (E && me > 0.f) ? E[i] / me : 0.f;
    f[2] = ms > 0.f ? fmaxf(0.f, logf(S[i] / ms + 1e-12f) / 27.631021f + 1.f) : 0.f;
    f[3] = (Imax && mx > 0.f) ? fmaxf(0.f, log10f(Imax[i] / mx + 1e-8f) * 0.125f + 1.f) : 0.f;
    *reinterpret_cast<uint4 *>(x + i * 16) = pack8(f);
    *reinterpret_cast<uint4 *>(x + i * 16 + 8) = pack8(f + 8);
}

__global__ void k_make_target(const float *__restrict__ St, const float *__restrict__ Sb, float *__restrict__ t,
                              size_t n) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float a = St[i], b = Sb[i];
    t[i] = (a > 0.f && b > 0.f) ? logf(a / b) : 0.f;
}

void pool_avg_f32(const float *fine, int n_fine, int f, float *coarse, cudaStream_t st) {
    const size_t nc = (size_t)(n_fine / f);
    if (nc) k_pool_avg_f32<<<blocks_for(nc * nc * nc), 256, 0, st>>>(fine, n_fine, f, coarse);
}
void pool_max_f32(const float *fine, int n_fine, int f, float *coarse, cudaStream_t st) {
    const size_t nc = (size_t)(n_fine / f);
    if (nc) k_pool_max_f32<<<blocks_for(nc * nc * nc), 256, 0, st>>>(fine, n_fine, f, coarse);
}
void max4(const float *a, const float *b, const float *c, const float *d, size_t n, unsigned *maxbits,
          cudaStream_t st) {
    cudaMemsetAsync(maxbits, 0, 4 * sizeof(unsigned), st);
    if (n) k_max4<<<304, 256, 0, st>>>(a, b, c, d, n, maxbits);
}
void make_inputs(const float *I, const float *E, const float *S, const float *Imax, const unsigned *maxbits,
                 uint16_t *x, size_t n, cudaStream_t st) {
    if (n) k_make_inputs<<<blocks_for(n), 256, 0, st>>>(I, E, S, Imax, maxbits, x, n);
}
void make_target(const float *S_true, const float *S_base, float *t, size_t n, cudaStream_t st) {
    if (n) k_make_target<<<blocks_for(n), 256, 0, st>>>(S_true, S_base, t, n);
}


// ---------------------------------------------------------------- judge and fallback
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ int block_of(int v, int lgD) {
    const int D = 1 << lgD, dm = D - 1, nb = D / JUDGE_BLOCK;
    const int x = v & dm, y = (v >> lgD) & dm, z = v >> (2 * lgD);
    return ((z / JUDGE_BLOCK) * nb + y / JUDGE_BLOCK) * nb + x / JUDGE_BLOCK;
}

// coarse voxel j (0..511) of block b
__device__ __forceinline__ int voxel_in_block(int b, int j, int lgD) {
    const int D = 1 << lgD, nb = D / JUDGE_BLOCK;
    const int bx = b % nb, by = (b / nb) % nb, bz = b / (nb * nb);
    const int x = bx * JUDGE_BLOCK + (j & 7), y = by * JUDGE_BLOCK + ((j >> 3) & 7), z = bz * JUDGE_BLOCK + (j >> 6);
    return (z * D + y) * D + x;
}

__device__ __forceinline__ size_t fine_cell(int v, int lgD, int f, int a) {
    const int D = 1 << lgD, dm = D - 1, n = D * f;
    const int x = v & dm, y = (v >> lgD) & dm, z = v >> (2 * lgD);
    const int ax = a % f, ay = (a / f) % f, az = a / (f * f);
    return ((size_t)(z * f + az) * n + (y * f + ay)) * n + (x * f + ax);
}

__global__ void k_apply_residual(const float *__restrict__ Sc, const float *__restrict__ y, int use_net,
                                 float *__restrict__ Sp, size_t n) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) Sp[i] = use_net ? Sc[i] * expf(y[2 * i]) : Sc[i];
}

__global__ void k_block_pred_err(const float *__restrict__ y, int lgD, float *__restrict__ pe, int nblocks) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblocks) return;
    float m = 0.f;
    for (int j = 0; j < JUDGE_BLOCK * JUDGE_BLOCK * JUDGE_BLOCK; ++j)
        m = fmaxf(m, expf(y[2 * (size_t)voxel_in_block(b, j, lgD) + 1]));
    pe[b] = m;
}

__global__ void k_judge_pick(int lgD, int f, uint64_t seed, int samples, uint8_t *__restrict__ mask,
                             int *__restrict__ sample_vox, int nblocks) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nblocks * samples) return;
    const int b = e / samples, s = e % samples;
    const int j = (int)(mix64(seed ^ ((uint64_t)e * 0xD1B54A32D192ED03ull)) & 511u);
    const int v = voxel_in_block(b, j, lgD);
    sample_vox[e] = v;
    for (int a = 0; a < f * f * f; ++a) mask[fine_cell(v, lgD, f, a)] = 1;
    (void)s;
}

__global__ void k_judge_err(const float *__restrict__ Sf, const float *__restrict__ Sp,
                            const int *__restrict__ sample_vox, int lgD, int f, int samples, float *__restrict__ err,
                            int nblocks) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblocks) return;
    float m = 0.f;
    for (int s = 0; s < samples; ++s) {
        const int v = sample_vox[b * samples + s];
        float acc = 0.f;
        for (int a = 0; a < f * f * f; ++a) acc += Sf[fine_cell(v, lgD, f, a)];
        acc /= (float)(f * f * f);
        const float rel = acc > 0.f ? fabsf(Sp[v] - acc) / acc : (Sp[v] != 0.f ? INFINITY : 0.f);
        m = fmaxf(m, rel);
    }
    err[b] = m;
}

__global__ void k_fallback_flags(const float *__restrict__ err, const float *__restrict__ pe, int use_pred,
                                 float tol, int nblocks, int *__restrict__ flags, unsigned *counts) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblocks) return;
    const bool jf = !(err[b] <= tol);
    const bool pf = use_pred && !(pe[b] <= tol);
    flags[b] = (jf || pf) ? 1 : 0;
    if (jf || pf) atomicAdd(counts, 1u);
    if (jf) atomicAdd(counts + 1, 1u);
    if (pf) atomicAdd(counts + 2, 1u);
    atomicMax(counts + 3, __float_as_uint(fminf(err[b], 3.0e38f)));
}

__global__ void k_fallback_mask(const int *__restrict__ flags, int lgD, int f, uint8_t *__restrict__ mask) {
    const int D = 1 << lgD, n = D * f;
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= (size_t)n * n * n) return;
    const int x = (int)(i % n), y = (int)((i / n) % n), z = (int)(i / ((size_t)n * n));
    const int v = ((z / f) * D + y / f) * D + x / f;
    mask[i] = (uint8_t)flags[block_of(v, lgD)];
}

__global__ void k_combine(const float *__restrict__ Sp, const float *__restrict__ Sf, const int *__restrict__ flags,
                          int lgD, int f, float *__restrict__ out) {
    const int D = 1 << lgD;
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= D * D * D) return;
    if (!flags[block_of(v, lgD)]) {
        out[v] = Sp[v];
        return;
    }
    float acc = 0.f;
    for (int a = 0; a < f * f * f; ++a) acc += Sf[fine_cell(v, lgD, f, a)];
    out[v] = acc / (float)(f * f * f);
}

static int nblocks_of(int lgD) {
    const int nb = (1 << lgD) / JUDGE_BLOCK;
    return nb * nb * nb;
}

void apply_residual(const float *Sc, const float *y, int use_net, float *Sp, size_t n, cudaStream_t st) {
    if (n) k_apply_residual<<<blocks_for(n), 256, 0, st>>>(Sc, y, use_net, Sp, n);
}
void block_pred_err(const float *y, int lgD, float *pe, cudaStream_t st) {
    const int nb = nblocks_of(lgD);
    k_block_pred_err<<<blocks_for(nb, 128), 128, 0, st>>>(y, lgD, pe, nb);
}
void judge_mask(int lgD, int factor, uint64_t seed, int samples, uint8_t *mask, int *sample_vox, cudaStream_t st) {
    const size_t n = (size_t)(factor << lgD);
    cudaMemsetAsync(mask, 0, n * n * n, st);
    const int nb = nblocks_of(lgD);
    k_judge_pick<<<blocks_for((size_t)nb * samples, 128), 128, 0, st>>>(lgD, factor, seed, samples, mask, sample_vox,
                                                                      nb);
}
void judge_err(const float *Sf, const float *Sp, const int *sample_vox, int lgD, int factor, int samples, float *err,
               cudaStream_t st) {
    const int nb = nblocks_of(lgD);
    k_judge_err<<<blocks_for(nb, 128), 128, 0, st>>>(Sf, Sp, sample_vox, lgD, factor, samples, err, nb);
}
void fallback_flags(const float *err, const float *pe, int use_pred, float tol, int nblocks, int *flags,
                    unsigned *counts, cudaStream_t st) {
    cudaMemsetAsync(counts, 0, 4 * sizeof(unsigned), st);
    k_fallback_flags<<<blocks_for(nblocks, 128), 128, 0, st>>>(err, pe, use_pred, tol, nblocks, flags, counts);
}
void fallback_mask(const int *flags, int lgD, int factor, uint8_t *mask, cudaStream_t st) {
    const size_t n = (size_t)(factor << lgD);
    k_fallback_mask<<<blocks_for(n * n * n), 256, 0, st>>>(flags, lgD, factor, mask);
}
void combine(const float *Sp, const float *Sf, const int *flags, int lgD, int factor, float *out, cudaStream_t st) {
    const size_t n = (size_t)1 << (3 * lgD);
    k_combine<<<blocks_for(n), 256, 0, st>>>(Sp, Sf, flags, lgD, factor, out);
}

}  // namespace nn
}  // namespace sph
