// Internal declarations shared by the libsph translation units (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "sph_common.cuh"

namespace sph {

// offset of level l inside the concatenated dense per-level arrays: (8^l - 1)/7
__host__ __device__ __forceinline__ int64_t dense_off(int l) { return ((1ll << (3 * l)) - 1) / 7; }

struct KParams64 {
    double alpha, bma, C, h, vol, scale, self_int;
};

// ---------------------------------------------------------------- selection
struct SelectArgs {
    int nx, ny, nz, D, brick_log2;
    const float *q, *emag;
    const uint8_t *mask;
    double i_frac, e_frac, e_app;
    unsigned *maxes;                 // [2]
    int *cnt_s, *cnt_t, *off_s, *off_t;   // [nbricks]
    int *totals;                     // [2] Ns, Nt
    uint32_t *src_key, *src_pc, *trg_key, *trg_pc;
    float *src_q;
};
int select_launch(const SelectArgs &A, cudaStream_t st);

// ---------------------------------------------------------------- direct sum
struct DirectArgs {
    const uint32_t *src_pc;
    const float *src_q;
    float wscale;
    int ns;
    const uint32_t *trg_pc;
    int nt;
    KParams kp;
    KParams64 kp64;
    int self_mode, nx, ny, fp64;
    void *out;
};
int direct_launch(const DirectArgs &A, cudaStream_t st);

// ---------------------------------------------------------------- tree
struct TreeDev {
    int *box_at;         // concatenated dense levels
    int *lvl_base, *lvl_count;   // [Lmax+1]
    int *b_level;
    uint32_t *b_key;
    int *b_sb, *b_se, *b_tb, *b_te, *b_parent;
    uint8_t *b_leaf;
};
struct TreeArgs {
    TreeDev T;
    int ns, nt, S, D, Lmax;
    const uint32_t *skey, *tkey;
    int *flag, *pos;     // dense scratch, 8^Lmax
    int4 *rng;           // dense scratch, 8^Lmax
    int *scan_tmp;
};
void tree_build_launch(const TreeArgs &A, cudaStream_t st);
size_t scan_tmp_ints(int n);
void scan_exclusive(const int *in, int *out, int n, int *total, int *tmp, cudaStream_t st);

struct ListDev {
    int *u_cnt, *v_cnt, *w_cnt, *x_cnt;     // [nboxes]
    int *u_off, *v_off, *w_off, *x_off;     // [nboxes+1]
    int *u_src, *v_src, *w_src, *x_src;
    short *v_oc;                            // offset code (ox+3) + 7(oy+3) + 49(oz+3)
};
void lists_count_launch(const TreeDev &T, const ListDev &L, int nboxes, int D, int Lmax, int *scan_tmp,
                        int *totals, cudaStream_t st);
void lists_fill_launch(const TreeDev &T, const ListDev &L, int nboxes, int D, int Lmax, const int *totals,
                       cudaStream_t st);

// ---------------------------------------------------------------- operators
// Surface radii in units of the box half-width.
constexpr double R_UE = 1.05, R_UC = 2.95, R_DC = 1.05, R_DE = 2.95;

struct OpsDev {
    // per level l (index l), FP32, transposed ([col][row]) so that threads over rows coalesce
    float *uc2e_t;    // [L][PP][PP]
    float *dc2e_t;    // [L][PP][PP]
    float *m2m_t;     // [L][8][PP][PP]  child (level l+1) ueq -> parent (level l) ueq
    float *l2l_t;     // [L][8][PP][PP]  parent (level l-1) deq -> child (level l) deq
    float *m2l_t;     // [L][316][PP][PP] source ueq -> target dcheck, [slot][j][i]
    uint16_t *m2l_bf; // [L][316][2][PP][PP] BF16 hi / lo, [slot][part][i][k] (row i = check point, K-major)
    short *slot_of_code;   // [343] -> 0..315 or -1
    float *surf;      // [152][4] unit surface points (x, y, z, 0)
    double *self_int; // [1]
};
struct OpsBuildArgs {
    int D, Lmax;
    double h, alpha, beta, eps;
    double *work;      // FP64 scratch
    OpsDev ops;
};
int ops_build(const OpsBuildArgs &A, cudaStream_t st);
size_t ops_work_doubles(int Lmax);

// ---------------------------------------------------------------- FMM passes
struct FmmDev {
    TreeDev T;
    ListDev L;
    OpsDev O;
    const uint32_t *src_pc, *trg_pc;
    const float *src_q;
    float wscale;
    KParams kp;
    int D, nx, ny, self_mode;
    float *ueq, *dchk, *deq;   // [nboxes][PP]
};
void fmm_upward_level(const FmmDev &F, int level, int box_begin, int box_count, cudaStream_t st);
void fmm_m2l_level(const FmmDev &F, int level, int box_begin, int box_count, int m2l_prec, cudaStream_t st);
void fmm_p2l_level(const FmmDev &F, int level, int box_begin, int box_count, cudaStream_t st);
void fmm_down_level(const FmmDev &F, int level, int box_begin, int box_count, cudaStream_t st);
void fmm_leaf(const FmmDev &F, int nboxes, int leaf_cap, float *out_dense, cudaStream_t st);

}  // namespace sph
