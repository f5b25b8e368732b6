// Kernels of the learned surrogate: a 4-level U-Net-like BF16 convolutional network on a
// coarse grid (16-32 channels), trained and run by the kernels in k_nn.cu.
//
// Tensors are channels-last [B][D][D][D][C] (x fastest, then y, z, batch), BF16 stored
// as uint16_t, D a power of two (D = 1 << lg).  A 3x3x3 convolution with zero padding is
// an implicit GEMM
//     out[m][n] = sum_k A[m][k] W[n][k],   k = tap * C + c,
//     A[m][tap*C + c] = x[m + offset(tap)][c]   (0 outside the grid),
//     tap = 9 (dz+1) + 3 (dy+1) + (dx+1),
// run on the tensor cores (tcgen05, BF16 in, FP32 accumulate in TMEM).  Weight images are
// pre-arranged in global memory in the exact shared-memory layout the MMA reads (K-major,
// 128-byte swizzle, one 64-element K chunk after the other).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sph {
namespace nn {

constexpr int NTAPS = 27;
// K chunks of 64 elements for C channels per tap (taps padded to 28 with zeros)
__host__ __device__ constexpr int conv_chunks(int C) { return (NTAPS + 64 / C - 1) / (64 / C); }
// rows of the weight-gradient accumulator [rows][N]: taps x C padded to whole 128-row tiles;
// row 27 * C accumulates the bias gradient
__host__ __device__ constexpr int wgrad_rows(int C) { return ((28 * C + 127) / 128) * 128; }

struct ConvArgs {
    const uint16_t *x;       // [nvox][C]
    const uint16_t *w;       // weight image: conv_chunks(C) x [N][64], swizzled
    const float *bias;       // [N] or nullptr
    const uint16_t *add;     // [nvox][N] or nullptr: added after the ReLU
    const uint16_t *mask;    // [nvox][N] or nullptr: zero where mask <= 0 (applied last)
    uint16_t *out;           // [nvox][N]
    int relu;
    int nvox, lg;
    int *err;                // bit 0: a bounded wait expired
};

struct WgradArgs {
    const uint16_t *x;       // [nvox][C] layer input
    const uint16_t *dz;      // [nvox][N] gradient w.r.t. the layer's pre-activation
    float *dw;               // [wgrad_rows(C)][N]: added into (reductions, or the fixed-order sum below)
    int nvox, lg;
    int chunks_per_cta;      // chunks of 64 voxels per CTA
    int *err;
    // optional [WGRAD_MAX_SPLIT][wgrad_rows(C)][N] scratch: each CTA stores its partial sum there
    // and a second kernel adds the partials into dw in a fixed order (training is then
    // reproducible bit for bit); nullptr: the CTAs add into dw with reductions
    float *part = nullptr;
};
constexpr int WGRAD_MAX_SPLIT = 160;   // voxel splits of one weight gradient (grid.y) at most
constexpr int HEAD_MAX_BLOCKS = 8192;  // blocks of the head's loss / gradient kernel with partials

// set the shared-memory limits of every instantiation (call once, outside graph capture)
void init_attributes();
// C, N in {16, 32}; returns 0, or -1 for an unsupported shape
int conv(const ConvArgs &a, int C, int N, cudaStream_t st);
int wgrad(const WgradArgs &a, int C, int N, cudaStream_t st);

// element-wise and resampling (BF16 tensors, C a multiple of 8)
void pool2(const uint16_t *in, uint16_t *out, int B, int lg_out, int C, cudaStream_t st);
void up_add(const uint16_t *coarse, const uint16_t *skip, uint16_t *out, int B, int lg_out, int C,
            cudaStream_t st);
void add(const uint16_t *a, const uint16_t *b, uint16_t *out, size_t n, cudaStream_t st);
void mask_mul(const uint16_t *g, const uint16_t *mask, uint16_t *out, size_t n, cudaStream_t st);
void up_back_mask(const uint16_t *g_fine, const uint16_t *mask, uint16_t *out, int B, int lg_out, int C,
                  cudaStream_t st);
void pool_back_add_mask(const uint16_t *g_coarse, const uint16_t *add, const uint16_t *mask, uint16_t *out, int B,
                        int lg_out, int C, cudaStream_t st);

// head: y[m][j] = sum_c hw[j][c] f[m][c] + hb[j], j in {0, 1}; f has 16 channels
void head_forward(const uint16_t *f, const float *hw, const float *hb, float *y, int nvox, cudaStream_t st);
// loss of the residual r = y0 against t and of the error head e = y1 against log(|r - t| + eps);
// writes the masked gradient of f (BF16), accumulates the head's gradient hg[34] and the loss sum
// hpart (optional, [HEAD_MAX_BLOCKS][34] scratch, nvox <= 256 HEAD_MAX_BLOCKS): per-block partials of the
// head gradient summed in a fixed order instead of reductions
void head_loss_backward(const uint16_t *f, const float *hw, const float *hb, const float *t, uint16_t *g_f,
                        float *hg, double *loss_sum, int nvox, float lambda, float eps, cudaStream_t st,
                        float *hpart = nullptr);

// parameters: per layer w [N][27][C] then b [N] (FP32 master copy)
void collect_grads(const float *dw, int C, int N, float *g, cudaStream_t st);
void adam(float *p, const float *g, float *m, float *v, size_t n, float lr, float b1, float b2, float eps,
          float bc1, float bc2, cudaStream_t st);
void make_images(const float *w, int C, int N, uint16_t *img_fwd, uint16_t *img_dgrad, cudaStream_t st);
void f32_to_bf16(const float *in, uint16_t *out, size_t n, cudaStream_t st);

// coarse inputs of the network from pooled fields
void pool_avg_f32(const float *fine, int n_fine, int f, float *coarse, cudaStream_t st);
void pool_max_f32(const float *fine, int n_fine, int f, float *coarse, cudaStream_t st);
void max4(const float *a, const float *b, const float *c, const float *d, size_t n, unsigned *maxbits,
          cudaStream_t st);
void make_inputs(const float *I, const float *E, const float *S, const float *Imax, const unsigned *maxbits,
                 uint16_t *x, size_t n, cudaStream_t st);
void make_target(const float *S_true, const float *S_base, float *t, size_t n, cudaStream_t st);

}  // namespace nn
}  // namespace sph

namespace sph {
namespace nn {
// ---- judge and fallback of the surrogate (single sample, coarse grid D = 1 << lgD, blocks of
// 8^3 coarse voxels, fine grid n = factor * D)
constexpr int JUDGE_BLOCK = 8;
// S_pred = S_coarse * exp(r) (use_net) or S_coarse
void apply_residual(const float *Sc, const float *y, int use_net, float *Sp, size_t n, cudaStream_t st);
// per block: max over its voxels of exp(e) (the error head's estimate of |ln S_pred - ln S|)
void block_pred_err(const float *y, int lgD, float *pe, cudaStream_t st);
// mark `samples` seeded coarse voxels per block: their factor^3 fine cells in mask (cleared here)
void judge_mask(int lgD, int factor, uint64_t seed, int samples, uint8_t *mask, int *sample_vox, cudaStream_t st);
// per block: max relative error of S_pred against the pooled fine S at the sampled voxels
void judge_err(const float *Sf, const float *Sp, const int *sample_vox, int lgD, int factor, int samples, float *err,
               cudaStream_t st);
// flags[b] = err > tol || (use_pred && pe > tol); counts: fallback, judged fail, predicted fail, max err bits
void fallback_flags(const float *err, const float *pe, int use_pred, float tol, int nblocks, int *flags,
                    unsigned *counts, cudaStream_t st);
void fallback_mask(const int *flags, int lgD, int factor, uint8_t *mask, cudaStream_t st);
void combine(const float *Sp, const float *Sf, const int *flags, int lgD, int factor, float *out, cudaStream_t st);
}  // namespace nn
}  // namespace sph
