// sph_select_noalloc: the source / target selection without any device allocation.
//
// Who needs it: code that must not call cudaMalloc while it runs -- for example a
// host application that hands the library a fixed memory budget up front, a caller
// that is itself inside a region where allocation is forbidden or would
// synchronise the device (a real-time time step, a custom allocator that owns all
// device memory), or a harness that checks that a step performs no allocation.
// sph_create + eval_sph allocate their working buffers on first use and grow them;
// this entry point instead takes every output from the caller and keeps its small
// scratch (per-brick counters, offsets and statistics, the two maxima, the totals) in one
// fixed, file-scope device array that exists from library load to process exit.
//
// Limits and behaviour:
//   * grids up to 512 cells per axis (at most 32768 bricks of 16^3 cells);
//     larger grids are rejected with SPH_ECAPACITY before any work is queued;
//   * the scratch array is shared by every call in the process on that device and
//     keeps the last call's contents; the maxima are cleared at the start of every
//     call, everything else is fully rewritten before it is read;
//   * calls whose work overlaps on the GPU (different streams, or different host
//     threads without ordering) race on the shared array: serialise them;
//   * the device address of the array is looked up once per device, with that
//     device current, by the first call made for it (cudaGetSymbolAddress); make
//     that first call before capturing any stream into a CUDA graph.
#include <cstdlib>
#include <mutex>

#include "sph_kernels.cuh"
#include "../../include/sph.h"

namespace {

constexpr int NOALLOC_MAX_EDGE = 512;
constexpr int NOALLOC_MAX_BRICKS = 32768;                 // (512 / 16)^3
constexpr int NOALLOC_HEAD = 64;                          // maxima (2), totals (2) + flag, padding
// head, four ints per brick (counters, offsets), four floats per brick (statistics): 1 MiB + 256 B
constexpr size_t NOALLOC_INTS = NOALLOC_HEAD + 8 * (size_t)NOALLOC_MAX_BRICKS;

static __device__ __align__(256) int g_noalloc_scratch[NOALLOC_INTS];

constexpr int MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
int *g_noalloc_ptr[MAX_DEVICES] = {};

// Device address of the scratch array on `device` (set-up on first use; nullptr on failure).
int *scratch_on(int device) {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (g_noalloc_ptr[device]) return g_noalloc_ptr[device];
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) return nullptr;
    if (cudaSetDevice(device) != cudaSuccess) return nullptr;
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    cudaSetDevice(prev);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return nullptr;
    }
    g_noalloc_ptr[device] = static_cast<int *>(p);
    return g_noalloc_ptr[device];
}

}  // namespace

extern "C" int sph_select_noalloc(int device, void *cuda_stream, int nx, int ny, int nz, const float *q_dev,
                                  const float *emag_dev, const uint8_t *mask_dev, double i_frac, double e_frac,
                                  double e_applied, uint32_t *src_key_dev, uint32_t *src_pc_dev, float *src_q_dev,
                                  uint32_t *trg_key_dev, uint32_t *trg_pc_dev, int32_t *counts_dev) {
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return SPH_ECUDA;
    }
    if (device < 0 || device >= ndev || device >= MAX_DEVICES) return SPH_EINVAL;
    if (nx < 1 || ny < 1 || nz < 1) return SPH_EINVAL;
    if (nx > NOALLOC_MAX_EDGE || ny > NOALLOC_MAX_EDGE || nz > NOALLOC_MAX_EDGE) return SPH_ECAPACITY;
    if (!q_dev || !src_key_dev || !src_pc_dev || !src_q_dev || !trg_key_dev || !trg_pc_dev || !counts_dev)
        return SPH_EINVAL;
    if (emag_dev && mask_dev) return SPH_EINVAL;
    if (!(i_frac >= 0 && i_frac <= 1) || !(e_frac >= 0 && e_frac <= 1)) return SPH_EINVAL;
    int *scratch = scratch_on(device);
    if (!scratch) return SPH_ECUDA;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return SPH_ECUDA;
    }
    int m = nx > ny ? nx : ny;
    m = m > nz ? m : nz;
    int D = 0;
    while ((1 << D) < m) ++D;
    const int b = D < 4 ? D : 4;
    const int nbricks = 1 << (3 * (D - b));
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    sph::SelectArgs A;
    A.nx = nx; A.ny = ny; A.nz = nz; A.D = D; A.brick_log2 = b;
    A.q = q_dev; A.emag = emag_dev; A.mask = mask_dev;
    A.i_frac = i_frac; A.e_frac = e_frac; A.e_app = e_applied;
    A.maxes = reinterpret_cast<unsigned *>(scratch);        // cleared by the launch itself
    A.totals = scratch + 2;
    A.cnt_s = scratch + NOALLOC_HEAD;
    A.cnt_t = A.cnt_s + nbricks;
    A.off_s = A.cnt_t + nbricks;
    A.off_t = A.off_s + nbricks;
    A.bstat = reinterpret_cast<float *>(scratch + NOALLOC_HEAD + 4 * (size_t)NOALLOC_MAX_BRICKS);   // 16-B aligned
    A.src_key = src_key_dev; A.src_pc = src_pc_dev; A.src_q = src_q_dev;
    A.trg_key = trg_key_dev; A.trg_pc = trg_pc_dev;
    if (const char *e = getenv("SPH_SELECT_LOOKBACK")) A.lookback = atoi(e) != 0;   // the look-back form
    if (const char *e = getenv("SPH_WAIT_LIMIT_SELECT")) {   // tests: make the look-back give up
        char *end = nullptr;
        const unsigned long v = strtoul(e, &end, 10);
        if (end && *end == 0) A.wait_limit = (unsigned)v;
    }
    int rc = SPH_OK;
    if (sph::select_launch(A, st) < 0) rc = SPH_ECUDA;
    // (sources, targets, gave-up flag): copied after the selection kernel has completed, so the
    // flag of every brick that gave up waiting is in it
    if (rc == SPH_OK && cudaMemcpyAsync(counts_dev, A.totals, 3 * sizeof(int32_t), cudaMemcpyDeviceToDevice, st) !=
                            cudaSuccess)
        rc = SPH_ECUDA;
    if (rc != SPH_OK) cudaGetLastError();
    cudaSetDevice(prev);
    return rc;
}
