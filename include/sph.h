/*
 * sph.h -- C ABI of libsph: the photoionization source S_ph of the Zheleznyak
 * integral model evaluated on one GPU by an adaptive kernel-independent fast
 * multipole method (Lin & Zhuang, "Adaptive Strategies to Fast Multipole
 * Method in Photoionization Calculations").
 *
 * What is computed (paper Section 2.1, Eq. integral / Eq. Ifun / Eq. gfun, and
 * Section 2.4, Eq. summation):
 *   S_ph(x_t) = sum_{s in J, s != t} G(|x_t - y_s|) I_h(y_s) + [t in J] I(x_t) * Gself
 *   G(R)      = (e^{-alpha R} - e^{-beta R}) / (4 pi L R^3),
 *   alpha = chi_min p_O2, beta = chi_max p_O2, L = ln(chi_max/chi_min),
 *   I = source_scale * q,  I_h = I * h^3 (cell volume),
 *   Gself = integral of G over the ball with one cell's volume
 *         = 1 - (E1(alpha a) - E1(beta a))/L,  a = h (3/(4 pi))^(1/3)   (self_mode 1)
 * over the source set J and the target set T chosen by the adaptive
 * strategies of Section 3 (Eq. summationI, Eq. sourcepct, the Section 5
 * electric-field rule):
 *   J = { n : q[n] >= i_frac * max_n q }      (i_frac == 0: every cell)
 *   T = { n : |E|[n] >= e_applied + e_frac (max|E| - e_applied) },
 *       or { n : mask[n] != 0 }, or every cell.
 * Every threshold comparison is made in FP64 on the FP32 inputs.
 * The far field is approximated through the hierarchy of Section 2.4
 * (Eq. nearfar, Eq. s2l, Figure fmulloc); the near field is summed exactly.
 *
 * Grid: nx*ny*nz cells of edge h (cm); cell n = i + nx*(j + ny*k) (x fastest)
 * has centre origin + h*(i+1/2, j+1/2, k+1/2).  nx, ny, nz <= 1024.
 *
 * Conventions for every call:
 *  - Return value: SPH_OK (0) or a negative sph_status.  Nothing throws or
 *    aborts; sph_last_error() gives a one-line message for the last failure.
 *  - Pointers named *_dev are device pointers on the context's device; they
 *    are borrowed, never freed, and must stay valid until the work queued on
 *    the context's stream has finished.  Pointers named *_host are host memory.
 *  - All work is queued on the stream given to sph_create (NULL = legacy
 *    default stream).  eval_* calls may synchronise that stream internally
 *    (tree sizes are data dependent); they return after the result is queued.
 *  - The library's kernels are launched with programmatic stream serialization:
 *    each may be scheduled while the previous kernel of the stream drains, and
 *    waits at entry until that kernel (the caller's or the library's) has
 *    completed, so stream order holds as usual.  SPH_PDL=0 in the environment
 *    (read once per process) launches them in plain stream order.
 *  - A CUDA error poisons the context: every later call returns SPH_ECUDA.
 *  - Every spin-wait of the library's kernels is bounded.  The look-back of the selection (its
 *    one-pass form: SPH_SELECT_LOOKBACK=1, or grids without per-brick statistics) and of the
 *    device scan give up after a number of polls and report it (SPH_ETIMEOUT, or the flag of
 *    sph_select_noalloc); the context stays usable.  For tests, the environment can lower
 *    those limits and inject a failure: SPH_WAIT_LIMIT_SELECT=<polls> (read by sph_create
 *    and by every sph_select_noalloc call, as is SPH_SELECT_LOOKBACK), SPH_WAIT_LIMIT_SCAN=<polls> (read by every
 *    sph_scan_i32 call), SPH_FAULT=alloc[:k] (read by sph_create: the k-th device allocation of
 *    that context, default the first, fails with SPH_ENOMEM; later ones proceed).
 *  - One context per host thread; contexts are independent.
 */
#ifndef SPH_H
#define SPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sph_ctx sph_ctx;

typedef enum sph_status {
    SPH_OK = 0,
    SPH_EINVAL = -1,     /* bad argument (detected on the host before any work is queued) */
    SPH_ENOMEM = -2,     /* device allocation failed */
    SPH_ECUDA = -3,      /* CUDA runtime error (context is poisoned) */
    SPH_ESTATE = -4,     /* call order: grid / sources / targets / criteria not set */
    SPH_ECAPACITY = -5,  /* a size exceeds a fixed capacity of this call */
    SPH_ETIMEOUT = -6,   /* a bounded device wait gave up */
    SPH_EINTERNAL = -7
} sph_status;

/* Arithmetic of the far-field translation M2L (Section 2.4 far interactions). */
enum {
    SPH_M2L_F32 = 0,     /* FP32 SIMT */
    SPH_M2L_BF16X3 = 1   /* tensor cores: BF16 hi/lo split, 3 products, FP32 accumulate */
};

/* Far-field representation of a box (Section 2.4: artificial source points
 * with artificial intensities that reproduce its far interactions, Eq. s2l). */
enum {
    SPH_FAR_CHEBYSHEV = 0,  /* order^3 tensor Chebyshev nodes, intensities by anterpolation (default, order 5) */
    SPH_FAR_SURFACE = 1     /* equivalent / check surfaces of Figure fmulloc, order points per cube
                               edge, intensities by the least-squares solve of Eq. s2l (FP64 SVD) */
};

/* Per-call statistics (host struct, optional). */
typedef struct sph_stats {
    int64_t n_sources;         /* |J| */
    int64_t n_targets;         /* |T| */
    int32_t depth;             /* D: the grid is embedded in a 2^D cube of cells */
    int32_t max_level;         /* deepest level that holds a box */
    int64_t n_boxes;
    int64_t n_leaves;
    int64_t n_u, n_v, n_w, n_x;/* interaction-list pairs */
    /* GPU milliseconds per phase, from CUDA events on the context's stream (filled when
     * stats is non-NULL): selection; tree + lists; upward pass (P2M, M2M); grouping of the
     * V pairs by offset; M2L; L2L (+ P2L); table L2P; leaf kernel (near field, M2P and
     * the remaining L2P); whole eval. */
    float ms_select, ms_tree, ms_upward, ms_vpairs, ms_m2l, ms_l2l, ms_l2p, ms_near, ms_total;
    int64_t n_launches;        /* kernels launched by this eval (operator precompute excluded) */
    int32_t far_method, far_order;
    int32_t leaf_size;         /* leaf size of the tree (set_criteria's, or the autotuner's choice) */
    int32_t near_table;        /* 1 if the near field used the table form */
    int64_t n_w_skipped;       /* (target, W box) pairs skipped by strategy 3 (sph_set_skip_ratio) */
    int32_t l2lp_fused;        /* 1 if the deepest level's L2L and L2P ran as one kernel (leaves of edge 4) */
    float ms_l2lp;             /* its GPU milliseconds (inside ms_l2p), 0 if not fused */
    int32_t m2l_tiles;         /* tensor-core M2L form of this eval: 1 target-stationary tiles (dense V
                                  lists), 0 tiles of V pairs; chosen by V-pair density, or by timing both
                                  when the leaf size is autotuned (set_criteria leaf_size 0) */
} sph_stats;

/* Create a context on CUDA device `device`, queuing work on `cuda_stream`
 * (a cudaStream_t; NULL = default stream).  *out receives the handle. */
int sph_create(sph_ctx **out, int device, void *cuda_stream);
/* Release every device buffer the context owns.  NULL is accepted. */
void sph_destroy(sph_ctx *ctx);
/* Message for the last failed call on this context (never NULL). */
const char *sph_last_error(const sph_ctx *ctx);

/* Grid and gas (Section 4 uniform mesh; Eq. gfun coefficients).
 * nx, ny, nz in [1, 1024]; h > 0 (cm); pO2 > 0 (Torr);
 * 0 < chi_min < chi_max (cm^-1 Torr^-1).  origin_cm may be NULL (= 0,0,0);
 * it only shifts coordinates and does not change S_ph. */
int set_grid(sph_ctx *ctx, int nx, int ny, int nz, const double origin_cm[3], double h_cm,
             double pO2_torr, double chi_min, double chi_max);

/* Emission field q (float[nx*ny*nz], device, x fastest) and the scale that
 * turns it into I of Eq. Ifun: I = source_scale * q (source_scale > 0).
 * Cells with NaN q are never selected. */
int set_sources(sph_ctx *ctx, const float *q_dev, double source_scale);

/* Target rule input: |E| (float[nx*ny*nz], device) for the electric-field
 * rule, or an explicit mask (uint8[nx*ny*nz], device, nonzero = target).
 * At most one may be non-NULL; both NULL makes every cell a target. */
int set_targets(sph_ctx *ctx, const float *emag_dev, const uint8_t *mask_dev);

/* Adaptive criteria (Section 3) and method options.
 * i_frac in [0,1] (0: every cell is a source); e_frac in [0,1];
 * e_applied in the units of |E|; self_mode 0 (no self term) or 1 (ball);
 * leaf_size in [0, 4096]: the octree splits a box holding more sources or more
 * targets than this; 0 = autotune (the first eval of each problem class times the
 * candidates 32, 64, 128 and 512 and keeps the fastest for the life of the context);
 * m2l_precision one of SPH_M2L_*. */
int set_criteria(sph_ctx *ctx, double i_frac, double e_frac, double e_applied,
                 int self_mode, int leaf_size, int m2l_precision);

/* Far-field representation and its order (see SPH_FAR_*): Chebyshev order in
 * [2, 8] (p^3 nodes per box), surface order in [3, 10] (points per cube edge).
 * Default: SPH_FAR_CHEBYSHEV, 5.  Takes effect at the next eval. */
int sph_set_far_field(sph_ctx *ctx, int method, int order);

/* Near field (Eq. nearfar, the exact part): SPH_NEAR_EXP evaluates the kernel with its
 * exponentials for every source-target pair (default); SPH_NEAR_TABLE reads G for the integer
 * squared cell offsets below 4096 from a table built per evaluation with the same arithmetic
 * (uniform grids make every offset an integer); SPH_NEAR_AUTO times both on the first eval
 * of each problem class and keeps the faster.  Takes effect at the next eval. */
enum { SPH_NEAR_EXP = 0, SPH_NEAR_TABLE = 1, SPH_NEAR_AUTO = 2 };
int sph_set_near_field(sph_ctx *ctx, int mode);

/* Strategy 3 of Section 3 (third approach): after the far field, the leaf itself and the
 * leaves adjacent to it have been summed for a target, the non-adjacent near boxes (W list,
 * Chebyshev far field) are skipped for that target when their bounded contribution
 * G(d_min) * sum of their I_h is below r_s times that estimate (d_min: distance from the
 * target cell to the box's nearest cell).  r_s in [0, 1); 0 (default) turns it off; the paper
 * uses 1e-4 in its streamer simulations (Section 5).  Applies to leaves with at most 256
 * targets. */
int sph_set_skip_ratio(sph_ctx *ctx, double r_s);

/* Evaluate S_ph by the adaptive FMM into s_dev (float[nx*ny*nz], device):
 * S_ph at every target, 0 at every other cell.  stats may be NULL. */
int eval_sph(sph_ctx *ctx, float *s_dev, sph_stats *stats);

/* One snapshot of a batch: its own grid, gas, fields, thresholds and output. */
typedef struct sph_problem {
    int nx, ny, nz;                 /* [1, 1024] */
    double h_cm, pO2_torr;          /* > 0 */
    double chi_min, chi_max;        /* 0 < chi_min < chi_max */
    const float *q_dev;             /* float[nx*ny*nz], device */
    double source_scale;            /* > 0 */
    const float *emag_dev;          /* float[nx*ny*nz] or NULL */
    const uint8_t *mask_dev;        /* uint8[nx*ny*nz] or NULL (at most one of emag/mask) */
    double i_frac, e_frac, e_applied;
    float *s_dev;                   /* output float[nx*ny*nz], device; 0 at non-targets */
} sph_problem;

/* Evaluate n independent snapshots in one call (the paper evaluates S_ph twice per time step
 * of a streamer simulation, Section 5; a batch is many such evaluations).  Method options
 * (self term, leaf size or autotune, M2L arithmetic, far field) come from the context's
 * set_criteria / sph_set_far_field; the grid, fields and thresholds from each problem.  The
 * snapshots' phases are interleaved so the whole batch needs two host synchronisations, and their
 * FMM passes run concurrently on per-snapshot streams, captured into one CUDA graph.
 * Inputs must be ready on the context's stream; outputs are complete on it when the
 * queued work finishes.  stats (optional) sums counts over the batch; ms_total is the
 * batch's GPU time.  Each snapshot slot keeps its own buffers and operator cache. */
int eval_sph_batch(sph_ctx *ctx, int n, const sph_problem *problems, sph_stats *stats);

/* Same evaluation with host buffers: copies q (and |E| or the mask, as set
 * by the last set_targets call's kind: pass the matching host array, or NULL
 * for "every cell") to context-owned device memory, evaluates, and copies S
 * back to s_host.  Host pointers need not be pinned. */
int eval_sph_host(sph_ctx *ctx, const float *q_host, const float *emag_host,
                  const uint8_t *mask_host, float *s_host, sph_stats *stats);

/* Direct sum of Eq. summation over the same selected sets (no FMM):
 * fp64 == 0 writes float[nx*ny*nz] in FP32 arithmetic, fp64 == 1 writes
 * double[nx*ny*nz] in FP64 arithmetic.  0 at non-targets. */
int eval_direct(sph_ctx *ctx, int fp64, void *s_dev);

/* Selected sets of the last eval: canonical ascending linear indices.
 * Call with NULL arrays to get the counts; then with arrays of that size.
 * Synchronises the stream. */
int sph_get_selection(sph_ctx *ctx, int32_t *src_host, int64_t *n_src,
                      int32_t *trg_host, int64_t *n_trg);

/* Octree of the last eval.  Call with tree == NULL fields to read the counts
 * (n_boxes, n_u, n_v, n_w, n_x); then with arrays of those sizes.  Boxes are
 * ordered by (level, Morton key); pairs are (target box, source box).
 * Synchronises the stream. */
typedef struct sph_tree_view {
    int64_t n_boxes, n_u, n_v, n_w, n_x;
    int32_t depth;
    int32_t *level;        /* [n_boxes] */
    uint32_t *key;         /* [n_boxes] Morton key at its level: x bit 3b, y 3b+1, z 3b+2 */
    int32_t *src_begin, *src_end, *trg_begin, *trg_end;  /* [n_boxes] ranges in Morton-sorted points */
    int32_t *parent;       /* [n_boxes], -1 for the root */
    uint8_t *is_leaf;      /* [n_boxes] */
    int32_t *u_pairs, *v_pairs, *w_pairs, *x_pairs;      /* [2*n] (target box, source box) */
} sph_tree_view;
int sph_get_tree(sph_ctx *ctx, sph_tree_view *tree);

/* Selection without any device allocation (the paper has no counterpart: this is a
 * convenience of the library for callers that cannot allocate device memory while
 * they run -- e.g. an application that owns all device memory through its own
 * allocator or budget, or code running where an allocation would synchronise or is
 * forbidden).  It performs the same source / target selection as eval_sph (same
 * rules, same Morton-ordered output) but takes every output from the caller and
 * keeps its scratch in one fixed static device array inside the library.
 *   device, cuda_stream: CUDA device and stream (cudaStream_t, NULL = default);
 *   nx, ny, nz in [1, 512] (larger grids: SPH_ECAPACITY, nothing queued);
 *   q_dev, emag_dev / mask_dev, i_frac, e_frac, e_applied: as set_sources /
 *   set_targets / set_criteria (at most one of emag_dev, mask_dev non-NULL);
 *   outputs (device, each with room for nx*ny*nz entries): src_key_dev, src_pc_dev
 *   (packed i | j<<10 | k<<20), src_q_dev, trg_key_dev, trg_pc_dev, in Morton order;
 *   counts_dev: int32[3] receives (number of sources, number of targets, failure flag).
 * The work is queued on cuda_stream; results are valid once it completes and only if
 * counts_dev[2] is 0.  A non-zero counts_dev[2] means that a block of the selection gave up
 * waiting for its predecessors' counts (the condition eval_sph reports as SPH_ETIMEOUT):
 * the counts are then -1 or wrong and the outputs must not be used.  All calls
 * share the library's scratch array: calls that overlap on the GPU race and must be
 * serialised by the caller.  The first call for a device looks up the array's device
 * address; make it before any stream capture.  Never calls cudaMalloc or cudaFree. */
int sph_select_noalloc(int device, void *cuda_stream, int nx, int ny, int nz, const float *q_dev,
                       const float *emag_dev, const uint8_t *mask_dev, double i_frac, double e_frac,
                       double e_applied, uint32_t *src_key_dev, uint32_t *src_pc_dev, float *src_q_dev,
                       uint32_t *trg_key_dev, uint32_t *trg_pc_dev, int32_t *counts_dev);

/* Exclusive prefix sum of int32 counts: the building block that numbers the octree's boxes
 * (scan of the per-slot existence flags of Section 2.4's adaptive tree) and lays out the
 * interaction lists (scan of the per-box list lengths) -- the same one-launch device scan
 * the tree phase runs.  out_dev[i] = sum_{j<i} in_dev[j] (int32, wrapping), *total_dev =
 * sum of all n.  in_dev, out_dev: device int32[n], distinct; total_dev: device int32[1];
 * 0 <= n < 2^31.  Allocates its scratch and synchronises the stream.  SPH_ETIMEOUT if a
 * tile gave up waiting for its predecessors (the results are then not valid). */
int sph_scan_i32(int device, void *cuda_stream, int64_t n, const int32_t *in_dev, int32_t *out_dev,
                 int32_t *total_dev);

/* Measured throughput of the pipes that evaluate the kernel G (the paper has no counterpart:
 * these are the denominators of the library's near-field and direct-sum rooflines).  Runs
 * three short kernels on cuda_stream (FP32 fused multiply-add, MUFU ex2, MUFU rsqrt: eight
 * independent chains per thread, 8 CTAs of 256 threads per SM), times each with CUDA events
 * (best of three after one untimed launch) and synchronises the stream.  out_host: double[4]
 * receives FP32 flop/s (one FMA = 2 flop), ex2 results/s, rsqrt results/s and the number of
 * SMs.  The figures hold at the SM clock of the moment; allocates nothing. */
int sph_measure_pipe_peaks(int device, void *cuda_stream, double *out_host);

/* Library version string. */
const char *sph_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SPH_H */
