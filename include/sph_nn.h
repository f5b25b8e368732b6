/*
 * sph_nn.h -- C ABI of the learned surrogate in libsph: a small convolutional network
 * that predicts S_ph on a coarse grid, trained on the GPU by the library's own BF16
 * kernels on fields that the adaptive FMM (sph.h) computes, and judged by the FMM.
 *
 * The paper has no learned component; this is the project's learned surrogate of
 * the S_ph evaluation (Section 2.4, Eq. summation), with the FMM as its judge and
 * fallback.
 *
 * Network (every convolution 3x3x3, zero padding, bias, ReLU):
 *   level 0 (edge D):   c00 16->16, c01 16->16 = s0        pool 2x2x2 (mean)
 *   level 1 (D/2):      c10 16->32, c11 32->32 = s1        pool
 *   level 2 (D/4):      c20 32->32, c21 32->32 = s2        pool
 *   level 3 (D/8):      c30 32->32, c31 32->32 = b3
 *   up (nearest) + s2 -> c22 32->32;  up + s1 -> c12 32->32;  up -> c02 32->16, + s0
 *   c03 16->16 = f;  head (1x1x1, FP32, no ReLU): [r, e] = Wh f + bh
 * Input x: BF16 [B][D][D][D][16] channels-last (x fastest, then y, z, batch); channels 0-3
 * are the log-normalised pooled source, the normalised pooled |E|, the log-normalised
 * coarse FMM estimate and the log-normalised largest fine-cell source in each coarse cell
 * (sph_nn_make_inputs), the rest zero.  Output y: FP32 [B][D^3][2]:
 * r = predicted ln(S_fine_pooled / S_coarse), e = predicted ln |error of r|.
 * D is a power of two, 8 <= D <= 256.
 *
 * Parameters (FP32, flat): for each convolution in the order c00 c01 c10 c11 c20 c21 c30
 * c31 c22 c12 c02 c03: w [Cout][27][Cin] (tap = 9 (dz+1) + 3 (dy+1) + (dx+1)), b [Cout];
 * then head w [2][16], b [2].
 *
 * Loss of a training batch with target t (FP32 [B][D^3]):
 *   L = mean (r - t)^2 + 0.01 * mean (e - ln(|r - t| + 1e-4))^2   (inner |r - t| constant).
 *
 * Conventions as in sph.h: status codes sph_status, *_dev device pointers on the
 * network's device (borrowed), *_host host pointers, all work on the stream given to
 * sph_nn_create.
 */
#ifndef SPH_NN_H
#define SPH_NN_H

#include <stddef.h>
#include <stdint.h>

#include "sph.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sph_nn sph_nn;

/* Network for D^3 inputs and batches of at most max_batch (activations and gradients are
 * allocated here: about 140 MB per sample at D = 64). */
int sph_nn_create(sph_nn **out, int device, void *cuda_stream, int edge, int max_batch);
void sph_nn_destroy(sph_nn *net);
const char *sph_nn_last_error(const sph_nn *net);
int64_t sph_nn_num_params(void);

/* He-normal weights from a SplitMix64 stream of `seed`, zero biases, small head weights,
 * error-head bias ln(1e-2). */
int sph_nn_init(sph_nn *net, uint64_t seed);
/* Copy the flat FP32 parameters in / out (n must equal sph_nn_num_params()); set_params
 * also resets the Adam state. */
int sph_nn_set_params(sph_nn *net, const float *params_host, int64_t n);
int sph_nn_get_params(sph_nn *net, float *params_host, int64_t n);
/* Gradient of the last sph_nn_backward, flat, same layout (synchronises the stream). */
int sph_nn_get_grads(sph_nn *net, float *grads_host, int64_t n);

/* Forward pass: x_dev BF16 [batch][D^3][16] -> y_dev FP32 [batch][D^3][2]. */
int sph_nn_forward(sph_nn *net, int batch, const uint16_t *x_dev, float *y_dev);
/* Forward + backward against t_dev; the gradient stays on the device; *loss_host (optional)
 * receives L (synchronises the stream). */
int sph_nn_backward(sph_nn *net, int batch, const uint16_t *x_dev, const float *t_dev, double *loss_host);
/* One Adam step (bias-corrected, internal step counter) with the last gradient. */
int sph_nn_adam(sph_nn *net, float lr, float beta1, float beta2, float eps);
/* backward + Adam (lr, beta1 = 0.9, beta2 = 0.999, eps = 1e-8). */
int sph_nn_train_step(sph_nn *net, int batch, const uint16_t *x_dev, const float *t_dev, float lr,
                      double *loss_host);

/* Network inputs from fine-grid fields: I_fine_dev and E_fine_dev (optional) FP32 [n^3] with
 * n = factor * D, averaged over factor^3 blocks; S_coarse_dev FP32 [D^3] the coarse FMM
 * estimate.  Writes x_dev BF16 [D^3][16] (one sample). */
int sph_nn_make_inputs(sph_nn *net, int n_fine, int factor, const float *I_fine_dev, const float *E_fine_dev,
                       const float *S_coarse_dev, uint16_t *x_dev);
/* Training target t = ln(pool(S_fine) / S_coarse) (0 where either is 0), FP32 [D^3]. */
int sph_nn_make_target(sph_nn *net, int n_fine, int factor, const float *S_fine_dev, const float *S_coarse_dev,
                       float *t_dev);
/* Mean over factor^3 blocks of an n^3 FP32 field (n = factor * m) into m^3. */
int sph_pool_avg(int device, void *cuda_stream, int n_fine, int factor, const float *fine_dev, float *coarse_dev);

/* Single kernels, for checks against a reference convolution.  Weights FP32 [N][27][C]
 * (device), converted to BF16 inside; these calls allocate scratch and synchronise.
 *   mode 0 (forward):  out[nvox][N] = relu?( conv(x[nvox][C]) + bias ) + add, then * (mask > 0)
 *   mode 1 (data gradient): x is the gradient [nvox][N], out[nvox][C] = conv^T(x) + add,
 *                           then * (mask > 0); bias and relu are ignored.
 * C, N in {16, 32}; nvox = batch * edge^3; add / mask / bias may be NULL. */
int sph_nn_conv3d(int device, void *cuda_stream, int mode, int C, int N, int edge, int batch, const uint16_t *x_dev,
                  const float *w_dev, const float *bias_dev, const uint16_t *add_dev, const uint16_t *mask_dev, int relu,
                  uint16_t *out_dev);
/* Weight gradient: dw_dev FP32 [N][27][C] followed by db [N] (overwritten) from the layer
 * input x [nvox][C] and the pre-activation gradient dz [nvox][N]. */
int sph_nn_conv3d_wgrad(int device, void *cuda_stream, int C, int N, int edge, int batch, const uint16_t *x_dev,
                        const uint16_t *dz_dev, float *dw_dev);

/* ---- Surrogate evaluation with the FMM as judge and fallback ----
 * On the context's grid (cubic, n = factor * D with D the network's edge), sources and
 * criteria (i_frac selects the sources on both grids; the |E| field given to set_targets,
 * if any, is only a network input):
 *   1. S_c: the FMM on the coarse grid D^3 (cell edge factor * h) with the factor^3-pooled
 *      source, every coarse cell a target;
 *   2. S_pred = S_c * exp(r), r from the network (use_net = 0: S_pred = S_c);
 *   3. judge: the FMM on the fine grid at the factor^3 cells of `samples_per_block` seeded
 *      coarse voxels in every block of 8^3 coarse voxels; a block fails if S_pred differs
 *      from the pooled fine value by more than tol (relative) at any sample, or (use_net)
 *      if the error head predicts more than tol anywhere in it;
 *   4. fallback: the FMM on every fine cell of the failing blocks, pooled.
 * coarse_out_dev (FP32 [D^3]) receives the pooled-fine-grid estimate of S_ph: S_pred in
 * passing blocks, the pooled FMM in failing ones.  Synchronises the context's stream. */
typedef struct sph_surrogate_stats {
    int32_t n_blocks;             /* (D/8)^3 */
    int32_t n_fallback;           /* blocks evaluated by the fallback */
    int32_t n_judged_fail;        /* blocks failed by the judge's samples */
    int32_t n_predicted_fail;     /* blocks failed by the error head */
    int64_t n_judge_targets;      /* fine cells evaluated by the judge */
    int64_t n_fallback_targets;   /* fine cells evaluated by the fallback */
    float judged_max_err;         /* largest sampled relative error of S_pred */
    float ms_coarse, ms_net, ms_judge, ms_fallback, ms_total;
} sph_surrogate_stats;

int eval_sph_surrogate(sph_ctx *ctx, sph_nn *net, int factor, double tol, int samples_per_block, uint64_t seed,
                       int use_net, float *coarse_out_dev, sph_surrogate_stats *stats);

#ifdef __cplusplus
}
#endif
#endif
