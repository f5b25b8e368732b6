// Shared device helpers of libsph: Morton codes, packed cell coordinates and
// the FP32 evaluation of the photoionization kernel of Eq. gfun.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#ifdef __CUDACC__
#include <cstdlib>
#include <utility>

// ---------------------------------------------------------------- programmatic dependent launch
// Kernels of the evaluation are launched with programmatic stream serialization: the CTAs of
// a kernel may be scheduled while the previous kernel of the stream drains.  Every such kernel
// begins with pdl_enter(): it waits until the previous kernel has completed and its writes are
// visible (nothing is read or written before that), then lets the next kernel's launch begin.
// Both instructions are no-ops in a kernel launched without the attribute.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
// pdl_enter() after a prologue: a kernel may first touch what no kernel of the FMM passes
// writes -- the tree and list arrays, the operator images and tables (written before the passes
// were queued) -- and set up its own shared memory, barriers and tensor memory, so that this
// work overlaps the previous kernel's tail.  A grid is released only once every CTA of the
// previous one has started, so the early CTAs never keep the previous grid's CTAs waiting.
// SPH_PDL=0 in the environment launches every kernel in plain stream order.
inline bool pdl_enabled() {
    static const bool on = [] {
        const char *e = getenv("SPH_PDL");
        return !e || atoi(e) != 0;
    }();
    return on;
}
template <typename... P, typename... A>
inline cudaError_t launch_pdl(void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A &&...a) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, std::forward<A>(a)...);
}
#endif

#ifndef SPH_NP
#define SPH_NP 6         // surface lattice points per cube edge
#endif
// points on an equivalent / check surface: NP^3 - (NP-2)^3 (152 for NP = 6)
#define SPH_P (SPH_NP * SPH_NP * SPH_NP - (SPH_NP - 2) * (SPH_NP - 2) * (SPH_NP - 2))
// padded row length of a surface vector (multiple of 16)
#define SPH_PP ((SPH_P + 15) / 16 * 16)
#define SPH_NOFF 343     // 7^3 relative offsets of same-level boxes (316 used by M2L)

// ---------------------------------------------------------------- Morton codes
// Key bit layout: x in bit 3b, y in 3b+1, z in 3b+2 (b = 0 is the finest level).
__host__ __device__ __forceinline__ uint32_t spread3(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}
__host__ __device__ __forceinline__ uint32_t compact3(uint32_t v) {
    v &= 0x09249249u;
    v = (v | (v >> 2)) & 0x030c30c3u;
    v = (v | (v >> 4)) & 0x0300f00fu;
    v = (v | (v >> 8)) & 0x030000ffu;
    v = (v | (v >> 16)) & 0x000003ffu;
    return v;
}
__host__ __device__ __forceinline__ uint32_t morton3(uint32_t i, uint32_t j, uint32_t k) {
    return spread3(i) | (spread3(j) << 1) | (spread3(k) << 2);
}
__host__ __device__ __forceinline__ void demorton3(uint32_t m, uint32_t &i, uint32_t &j, uint32_t &k) {
    i = compact3(m);
    j = compact3(m >> 1);
    k = compact3(m >> 2);
}

// Packed cell coordinates: i | j << 10 | k << 20.
__host__ __device__ __forceinline__ uint32_t pack_ijk(uint32_t i, uint32_t j, uint32_t k) {
    return i | (j << 10) | (k << 20);
}
__host__ __device__ __forceinline__ int pc_i(uint32_t p) { return (int)(p & 1023u); }
// packed cell of a point from its Morton key at the grid's depth (the key interleaves the
// cell's three indices, so this is the same cell the selection packed)
__host__ __device__ __forceinline__ uint32_t key_pc(uint32_t key) {
    uint32_t i, j, k;
    demorton3(key, i, j, k);
    return pack_ijk(i, j, k);
}
__host__ __device__ __forceinline__ int pc_j(uint32_t p) { return (int)((p >> 10) & 1023u); }
__host__ __device__ __forceinline__ int pc_k(uint32_t p) { return (int)((p >> 20) & 1023u); }

// ---------------------------------------------------------------- kernel G
// G(R) = (e^{-alpha R} - e^{-beta R}) / (4 pi L R^3)
//      = C * e^{-alpha R} * (1 - e^{-(beta-alpha) R}) / R^3,  C = 1/(4 pi L).
// The factor 1 - e^{-x}, x = (beta-alpha) R, is formed without cancellation:
// for x < 1/2 by its Taylor series x - x^2/2! + x^3/3! - ... (truncated after
// x^8/8!, relative truncation error < 2e-8 on [0, 1/2)); above that the
// subtraction loses at most a factor 1/(1-e^{-1/2}) ~ 2.5 of relative accuracy.
struct KParams {
    float a2;     // alpha * log2(e)
    float b2;     // (beta - alpha) * log2(e)
    float bma;    // beta - alpha
    float C;      // 1 / (4 pi L)
    float h;      // cell edge (cm)
    float gself;  // (ball integral of G) / h^3 : self term per unit I_h
};

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 1 - e^{-x} for x >= 0.
__device__ __forceinline__ float one_minus_exp_neg(float x, float x_log2e) {
    if (x < 0.5f) {
        // Horner form of x * (1 - x/2 + x^2/6 - x^3/24 + x^4/120 - x^5/720 + x^6/5040 - x^7/40320)
        float p = -2.4801587301587302e-05f;            // -1/40320
        p = fmaf(p, x, 1.9841269841269841e-04f);       //  1/5040
        p = fmaf(p, x, -1.3888888888888889e-03f);      // -1/720
        p = fmaf(p, x, 8.3333333333333333e-03f);       //  1/120
        p = fmaf(p, x, -4.1666666666666667e-02f);      // -1/24
        p = fmaf(p, x, 1.6666666666666667e-01f);       //  1/6
        p = fmaf(p, x, -0.5f);
        p = fmaf(p, x, 1.0f);
        return p * x;
    }
    return 1.0f - ex2_approx(-x_log2e);
}

// G at squared distance r2 > 0 (cm^2).
__device__ __forceinline__ float g_of_r2(float r2, const KParams &k) {
    float ir = rsqrt_approx(r2);
    float R = r2 * ir;
    float e1 = ex2_approx(-k.a2 * R);
    float em = one_minus_exp_neg(k.bma * R, k.b2 * R);
    return k.C * e1 * em * (ir * ir * ir);
}

// G between two distinct cells whose integer offset has squared length d2 >= 1.
__device__ __forceinline__ float g_of_cells(int d2, const KParams &k) {
    float r2 = (float)d2 * (k.h * k.h);
    return g_of_r2(r2, k);
}

// Unit surface point m (0..P-1) of the NP x NP x NP lattice on [-1,1]^3 that
// lies on the cube's surface; lattice coordinates -1 + 2a/(NP-1).
// Order: lexicographic in (a, b, c) = lattice indices along (x, y, z), skipping interior points.
__host__ __device__ __forceinline__ void surf_unit(int m, float &x, float &y, float &z) {
    const int n = SPH_NP;
    int cnt = 0;
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b)
            for (int c = 0; c < n; ++c) {
                bool surf = (a == 0 || a == n - 1 || b == 0 || b == n - 1 || c == 0 || c == n - 1);
                if (!surf) continue;
                if (cnt == m) {
                    x = -1.0f + 2.0f * a / (n - 1);
                    y = -1.0f + 2.0f * b / (n - 1);
                    z = -1.0f + 2.0f * c / (n - 1);
                    return;
                }
                ++cnt;
            }
    x = y = z = 0.0f;
}

// FP64 kernel G(R) (operator precompute and the rare FP64 evaluation paths).
__device__ __forceinline__ double g64(double R, double alpha, double beta, double C) {
    return C * exp(-alpha * R) * (-expm1(-(beta - alpha) * R)) / (R * R * R);
}
