// Throughput of the two pipes the kernel evaluations run on: FP32 fused multiply-add and
// the special-function unit (MUFU: ex2 and rsqrt, the three MUFU results of one evaluation of
// G).  These are the denominators of the near-field, direct-sum and L2P rooflines.
//
// Each kernel runs eight independent dependency chains per thread (enough to hide the pipe
// latency with 8 warps per SM scheduler) over a grid of 8 CTAs of 256 threads per SM, and is
// timed with CUDA events after one untimed launch; the best of three timed launches counts.
#include <cuda_runtime.h>

#include "../../include/sph.h"

namespace {

__device__ float g_peak_sink;

constexpr int PK_THREADS = 256;
constexpr int PK_CHAINS = 8;

__global__ void __launch_bounds__(PK_THREADS) k_peak_ffma(int iters, float a, float b) {
    float x[PK_CHAINS];
#pragma unroll
    for (int j = 0; j < PK_CHAINS; ++j) x[j] = 1e-3f * (float)(threadIdx.x + j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int j = 0; j < PK_CHAINS; ++j) x[j] = fmaf(x[j], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < PK_CHAINS; ++j) s += x[j];
    if (s == 1.2345e-30f) g_peak_sink = s;       // never true; keeps the chains alive
}

__global__ void __launch_bounds__(PK_THREADS) k_peak_ex2(int iters) {
    float x[PK_CHAINS];
#pragma unroll
    for (int j = 0; j < PK_CHAINS; ++j) x[j] = 1e-3f * (float)(threadIdx.x + j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int j = 0; j < PK_CHAINS; ++j) {
                float y;
                // x -> 2^(-x): stays in [1/2, 1] for x in [0, 1]
                asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x[j]));
                x[j] = y;
            }
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < PK_CHAINS; ++j) s += x[j];
    if (s == 1.2345e-30f) g_peak_sink = s;
}

__global__ void __launch_bounds__(PK_THREADS) k_peak_rsqrt(int iters) {
    float x[PK_CHAINS];
#pragma unroll
    for (int j = 0; j < PK_CHAINS; ++j) x[j] = 1.0f + 1e-3f * (float)(threadIdx.x + j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int j = 0; j < PK_CHAINS; ++j) {
                float y;
                asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[j]));
                x[j] = y;
            }
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < PK_CHAINS; ++j) s += x[j];
    if (s == 1.2345e-30f) g_peak_sink = s;
}

}  // namespace

extern "C" int sph_measure_pipe_peaks(int device, void *cuda_stream, double *out_host) {
    if (!out_host) return SPH_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return SPH_EINVAL;
    }
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return SPH_ECUDA;
    }
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int blocks = 8 * nsm;
    const double threads = (double)blocks * PK_THREADS;
    const int it_fma = 8192, it_mufu = 1024;
    cudaEvent_t e0, e1;
    int rc = SPH_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        cudaSetDevice(prev);
        return SPH_ECUDA;
    }
    double best[3] = {1e30, 1e30, 1e30};
    for (int kind = 0; kind < 3 && rc == SPH_OK; ++kind) {
        for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(e0, st);
            if (kind == 0) k_peak_ffma<<<blocks, PK_THREADS, 0, st>>>(it_fma, 0.999f, 1e-3f);
            else if (kind == 1) k_peak_ex2<<<blocks, PK_THREADS, 0, st>>>(it_mufu);
            else k_peak_rsqrt<<<blocks, PK_THREADS, 0, st>>>(it_mufu);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = SPH_ECUDA;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms < best[kind]) best[kind] = ms;
        }
    }
    if (rc == SPH_OK && cudaGetLastError() != cudaSuccess) rc = SPH_ECUDA;
    if (rc == SPH_OK) {
        const double per_thread_fma = 4.0 * PK_CHAINS * it_fma;
        const double per_thread_mufu = 4.0 * PK_CHAINS * it_mufu;
        out_host[0] = 2.0 * per_thread_fma * threads / (best[0] * 1e-3);     // FP32 flop/s (FMA = 2)
        out_host[1] = per_thread_mufu * threads / (best[1] * 1e-3);          // ex2 results/s
        out_host[2] = per_thread_mufu * threads / (best[2] * 1e-3);          // rsqrt results/s
        out_host[3] = (double)nsm;
    } else {
        cudaGetLastError();
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaSetDevice(prev);
    return rc;
}
