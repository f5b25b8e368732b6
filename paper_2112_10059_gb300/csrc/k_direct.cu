// Direct quadrature of Eq. summation over the selected sets (paper Section 2.4,
// Section 4 "Classical Int"): every (target, source) pair through the same
// kernel G.  The FP32 variant is the plain direct sum the FMM is compared with;
// the FP64 variant serves the small all-pairs case.
//
// Layout: sources and targets in Morton order as packed (i,j,k) + weights.
// Tiling: each CTA owns 256 targets (one per thread) and streams every source
// through shared memory in tiles of 512.  Distances come from integer cell
// offsets, R^2 = h^2 (di^2 + dj^2 + dk^2), exact in FP32 below 2^24.
#include "sph_kernels.cuh"

namespace sph {

constexpr int DT = 256;   // targets per CTA
constexpr int DS = 512;   // sources per shared-memory tile

__global__ void __launch_bounds__(DT) k_direct_f32(const uint32_t *__restrict__ src_pc,
                                                   const float *__restrict__ src_q, float wscale, int ns,
                                                   const uint32_t *__restrict__ trg_key, int nt,
                                                   KParams kp, int self_mode, int nx, int ny,
                                                   float *__restrict__ out_dense) {
    __shared__ uint32_t sp[DS];
    __shared__ float sw[DS];
    int t = blockIdx.x * DT + threadIdx.x;
    uint32_t tp = t < nt ? key_pc(trg_key[t]) : 0xffffffffu;
    int ti = pc_i(tp), tj = pc_j(tp), tk = pc_k(tp);
    float acc = 0.0f;
    for (int s0 = 0; s0 < ns; s0 += DS) {
        int m = min(DS, ns - s0);
        __syncthreads();
        for (int u = threadIdx.x; u < m; u += DT) {
            sp[u] = src_pc[s0 + u];
            sw[u] = src_q[s0 + u] * wscale;
        }
        __syncthreads();
#pragma unroll 4
        for (int u = 0; u < m; ++u) {
            uint32_t p = sp[u];
            int di = ti - pc_i(p), dj = tj - pc_j(p), dk = tk - pc_k(p);
            int d2 = di * di + dj * dj + dk * dk;
            float g = d2 ? g_of_cells(d2, kp) : (self_mode ? kp.gself : 0.0f);
            acc = fmaf(g, sw[u], acc);
        }
    }
    if (t < nt) out_dense[(int64_t)ti + (int64_t)nx * ((int64_t)tj + (int64_t)ny * tk)] = acc;
}

__global__ void __launch_bounds__(DT) k_direct_f64(const uint32_t *__restrict__ src_pc,
                                                   const float *__restrict__ src_q, int ns,
                                                   const uint32_t *__restrict__ trg_key, int nt,
                                                   KParams64 kp, int self_mode, int nx, int ny,
                                                   double *__restrict__ out_dense) {
    __shared__ uint32_t sp[DS];
    __shared__ float sq[DS];
    int t = blockIdx.x * DT + threadIdx.x;
    uint32_t tp = t < nt ? key_pc(trg_key[t]) : 0xffffffffu;
    int ti = pc_i(tp), tj = pc_j(tp), tk = pc_k(tp);
    double acc = 0.0, comp = 0.0;
    for (int s0 = 0; s0 < ns; s0 += DS) {
        int m = min(DS, ns - s0);
        __syncthreads();
        for (int u = threadIdx.x; u < m; u += DT) {
            sp[u] = src_pc[s0 + u];
            sq[u] = src_q[s0 + u];
        }
        __syncthreads();
        for (int u = 0; u < m; ++u) {
            uint32_t p = sp[u];
            int di = ti - pc_i(p), dj = tj - pc_j(p), dk = tk - pc_k(p);
            int d2 = di * di + dj * dj + dk * dk;
            double v;
            if (d2) {
                double R = kp.h * sqrt((double)d2);
                v = kp.C * exp(-kp.alpha * R) * (-expm1(-kp.bma * R)) / (R * R * R) * kp.vol;
            } else {
                v = self_mode ? kp.self_int : 0.0;
            }
            // Kahan-Babuska (Neumaier) compensated accumulation
            double term = v * kp.scale * (double)sq[u];
            double s = acc + term;
            comp += fabs(acc) >= fabs(term) ? (acc - s) + term : (term - s) + acc;
            acc = s;
        }
    }
    if (t < nt) out_dense[(int64_t)ti + (int64_t)nx * ((int64_t)tj + (int64_t)ny * tk)] = acc + comp;
}

int direct_launch(const DirectArgs &A, cudaStream_t st) {
    if (A.nt == 0) return 0;
    int grid = (A.nt + DT - 1) / DT;
    if (A.fp64)
        k_direct_f64<<<grid, DT, 0, st>>>(A.src_pc, A.src_q, A.ns, A.trg_key, A.nt, A.kp64, A.self_mode,
                                          A.nx, A.ny, (double *)A.out);
    else
        k_direct_f32<<<grid, DT, 0, st>>>(A.src_pc, A.src_q, A.wscale, A.ns, A.trg_key, A.nt, A.kp, A.self_mode,
                                          A.nx, A.ny, (float *)A.out);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace sph
