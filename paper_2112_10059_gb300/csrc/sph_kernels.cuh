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
// Polls of a look-back before a block gives up waiting for its predecessor (selection) or a
// tile for its predecessors (device scan) and reports it; the host may lower either (tests:
// 0 gives up at once, deterministically).
constexpr unsigned SELECT_WAIT_LIMIT = 1u << 22;
constexpr unsigned SCAN_WAIT_LIMIT = 1u << 20;
struct SelectArgs {
    int nx, ny, nz, D, brick_log2;
    const float *q, *emag;
    const uint8_t *mask;
    double i_frac, e_frac, e_app;
    unsigned *maxes;                 // [2]
    int *cnt_s, *cnt_t, *off_s, *off_t;   // [nbricks]
    int *totals;                     // [3] Ns, Nt, error flag (look-back gave up)
    int two_pass = 0;                // 1: the reference form (maxima alone, then count pass + scan + emit
                                     //    pass, every brick read twice)
    int lookback = 0;                // 1: one pass with a decoupled look-back even where per-brick
                                     //    statistics allow the count / scan / emit passes
    uint32_t *src_key, *src_pc, *trg_key;
    uint32_t *trg_pc = nullptr;      // optional: targets' packed cells (key_pc of trg_key)
    float *src_q;
    uint8_t *tmask = nullptr;        // optional [nx*ny*nz]: 1 where the cell is a target
    unsigned wait_limit = SELECT_WAIT_LIMIT;   // polls per look-back round before giving up
    // optional [nbricks] float4 scratch (16-byte aligned): per-brick statistics of the maxima
    // pass, with which the one-pass selection emits a uniform brick without reading it again;
    // nullptr: the maxima alone (k_grid_max) and every brick read
    float *bstat = nullptr;
    mutable int launched = 0;        // out: kernels select_launch queued
    bool zeroed = false;             // maxes[0..2) and totals[2] were cleared by zero_set_launch
};
// 1: queued, and off_t holds every brick's exclusive target offset (count / scan / emit form);
// 0: queued without per-brick offsets; -1: a launch failed
int select_launch(const SelectArgs &A, cudaStream_t st);

// ---------------------------------------------------------------- direct sum
struct DirectArgs {
    const uint32_t *src_pc;
    const float *src_q;
    float wscale;
    int ns;
    const uint32_t *trg_key;         // Morton keys of the targets (cells by key_pc)
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
    int *lvl_src;                // [Lmax+1] boxes holding sources per level (zeroed before the emit)
    int *lvl_leaf;               // [Lmax+1] leaves holding targets per level (lvl_src + 16,
                                 // zeroed with it)
    int *lvl_sleaf;              // [Lmax+1] leaves holding sources per level (lvl_src + 32, zeroed with it)
    int *b_level;
    uint32_t *b_key;
    int *b_sb, *b_se, *b_tb, *b_te, *b_parent;
    uint8_t *b_leaf;
    // near[s], slots of levels 0..Lmax-1: a source point, or a leaf holding sources, lies in
    // the 3x3x3 slots around s.  If not, every list of every child of s is empty.
    const uint8_t *near;
    // vsrc[s], every slot of every level: a box exists at s and holds sources
    const uint8_t *vsrc;
};
struct TreeArgs {
    TreeDev T;
    const int *ns_dev, *nt_dev;   // point counts (device: the selection's totals)
    int ncap;                     // upper bound of either count (cells of the grid)
    int S, D, Lmax;
    const uint32_t *skey, *tkey;
    int *flag, *pos;     // dense scratch over every level's slots, dense_off(Lmax + 1) (+1 for pos)
    int *rsb, *rse, *rtb, *rte;   // dense point ranges of every slot of every level
    uint8_t *occ, *near;          // dense over levels 0..Lmax-1: source occupancy and its 3x3x3 dilation
    uint8_t *vsrc;                // dense over levels 0..Lmax: box exists and holds sources
    int *scan_tmp;
    int *err = nullptr;           // bit 0 set if a scan's look-back gave up waiting
    // optional: the selection's exclusive offsets of each 16^3 brick's targets ([nbr], bricks
    // in Morton order, D >= 4): the target ranges then follow from them slot by slot (a
    // binary search only inside bricks that are partly selected) instead of from a pass over
    // the target keys
    const int *brick_off_t = nullptr;
    int nbr = 0;
    // the point ranges, the per-level source / leaf counts and the scan's state were cleared by
    // zero_set_launch before the evaluation (no clearing copies in the launch sequence)
    bool zeroed = false;
};
void tree_build_launch(const TreeArgs &A, cudaStream_t st);

// Up to 12 device ranges of 4-byte words cleared by one launch: the counters and look-back scan
// states that selection, tree build and list counts need cleared, in one kernel before the
// selection's first one instead of one clearing copy before each user.
struct ZeroSet {
    static constexpr int CAP = 12;
    int n = 0;
    int *p[CAP] = {};
    int64_t words[CAP] = {};
    bool add(int *q, int64_t w) {
        if (w <= 0) return true;
        if (!q || n >= CAP) return false;
        p[n] = q;
        words[n] = w;
        ++n;
        return true;
    }
};
void zero_set_launch(const ZeroSet &Z, cudaStream_t st);
// bytes of state a look-back scan of k arrays of length n clears before it runs (0: the
// single-CTA scan, which keeps no state)
size_t scan_state_bytes(int k, int n);
size_t scan_tmp_ints(int n);
void scan_exclusive(const int *in, int *out, int n, int *total, int *tmp, cudaStream_t st, int *err = nullptr,
                    unsigned wait_limit = SCAN_WAIT_LIMIT, bool state_zeroed = false);

struct ListDev {
    int *u_cnt, *v_cnt, *w_cnt, *x_cnt;     // [nboxes]
    int *u_off, *v_off, *w_off, *x_off;     // [nboxes+1]
    int *u_src, *v_src, *w_src, *x_src;
    short *v_oc;                            // offset code (ox+3) + 7(oy+3) + 49(oz+3)
    int *v_trg;                             // target box of each V entry
    int *heavy, *nheavy;                    // boxes that can have list entries ([nboxes]), their count
};
struct PairsDev;
// The V pairs are also counted per (level, offset) key by the count pass and bucketed by the
// fill pass (the grouping the M2L tiles read); `Pd` per-key arrays zeroed before the count.
// cap: slots of every level (upper bound of the box count, the length of the list count and
// offset arrays); nboxes_dev: the tree's box count on the device
// Values the host reads after its sync, written by the list layout kernel (the last kernel
// before that sync) into a mapped pinned buffer `dst` (device address; null: not written):
// dst[0..3) = sel[0..3) (selection totals), dst[8..40) = lvl[0..32) (level first boxes and
// counts), dst[64..112) = lvl[32..80) (boxes with sources, leaves with targets, leaves with
// sources per level), dst[43..48) = flag_tot[0..5) (scan flag, the four list totals).
struct ReadBack {
    int *dst = nullptr;
    const int *sel = nullptr, *lvl = nullptr, *flag_tot = nullptr;
};
// Returns true when the layout kernel was queued with R.dst (the read-backs are then in flight).
// zeroed: the heavy-box count and the scan's state were cleared by zero_set_launch
bool lists_count_launch(const TreeDev &T, const ListDev &L, const PairsDev &Pd, int cap, const int *nboxes_dev,
                        int D, int Lmax, int *scan_tmp, int *totals, int *err, const ReadBack &R, cudaStream_t st,
                        bool zeroed = false);
void lists_fill_launch(const TreeDev &T, const ListDev &L, const PairsDev &Pd, int nboxes, int D, int Lmax,
                       const int *totals, cudaStream_t st);

// ---------------------------------------------------------------- operators
// Far-field representation of a box (Section 2.4: artificial source points
// with artificial intensities reproduce the far interactions, Eq. s2l):
//   FAR_CHEB    : the artificial points are the p^3 tensor Chebyshev nodes of
//                 the box; intensities by Chebyshev anterpolation (default);
//   FAR_SURFACE : equivalent / check surfaces of Figure fmulloc (NP points
//                 per cube edge), intensities by the least-squares solve of
//                 Eq. s2l (FP64 truncated SVD).
enum FarMethod { FAR_CHEB = 0, FAR_SURFACE = 1 };
constexpr int MAXPAD = 512;          // largest padded state length (p <= 8, NP <= 10)
constexpr int NSLOT = 316;           // M2L offsets o in [-3,3]^3 \ [-1,1]^3

// Slot of a V offset (|o|_inf >= 2, components in [-3, 3]): its rank among those offsets in
// the order of the code (ox + 3) + 7 (oy + 3) + 49 (oz + 3), i.e. the code minus the number of
// adjacent offsets (components in {-1, 0, 1}) with a smaller code.
__host__ __device__ __forceinline__ int m2l_slot(int ox, int oy, int oz) {
    auto below = [](int v) { return v < -1 ? 0 : (v > 1 ? 3 : v + 1); };   // adjacent values < v
    const bool ny = oy >= -1 && oy <= 1, nz = oz >= -1 && oz <= 1;
    const int code = (ox + 3) + 7 * (oy + 3) + 49 * (oz + 3);
    return code - (9 * below(oz) + (nz ? 3 * below(oy) + (ny ? below(ox) : 0) : 0));
}
constexpr int ETAB_MAX_EDGE = 16;    // surface L2P tables for leaf boxes of edge <= 16 cells

// Surface radii in units of the box half-width: upward equivalent / check,
// downward check / equivalent.
struct Radii {
    double ue, uc, dc, de;
};
constexpr Radii RADII_DEFAULT = {1.05, 2.95, 1.05, 2.95};

__host__ __device__ __forceinline__ int far_n(int method, int order) {
    return method == FAR_CHEB ? order * order * order
                              : order * order * order - (order - 2) * (order - 2) * (order - 2);
}
__host__ __device__ __forceinline__ int pad16(int n) { return (n + 15) / 16 * 16; }

// State vectors (length n, rows padded to npad) per box:
//   FAR_CHEB:    u_B = anterpolated source weights at B's nodes,
//                d_B = far-field potential at B's nodes (interpolated to targets);
//   FAR_SURFACE: u_B = upward check potential, d_B = downward check potential
//                (every pseudo-inverse folded into the operators in FP64).
// Matrices are stored FP32 transposed ([col][row], npad x npad) so a CTA with
// one thread per output row reads them coalesced.
struct OpsDev {
    int method, order, n, npad;
    float *m2m_t;     // [L][8][npad][npad]  u_child(l+1, c) -> u_parent(l)
    float *l2l_t;     // [L][8][npad][npad]  d_parent(l-1) -> d_child(l, c)
    float *m2l_t;     // [L][316][npad][npad] u_A -> d_B (A at offset o from B)
    uint16_t *m2l_img;    // [L][316] BF16 hi / lo images of M2L for the tensor cores (npad == 128)
    uint16_t *l2l_img;    // [L][8]   BF16 hi / lo images of L2L
    uint16_t *m2m_img;    // [L][8]   BF16 hi / lo images of M2M
    float *e_tab;     // L2P tables per level: FAR_SURFACE [edge^3][npad] row-major (cells in linear order);
                      // FAR_CHEB [npad][edge^3] (cells in local Morton order)
    long long e_off[16];          // float offset of level l's table in e_tab, -1 if none
    uint16_t *l2p_img;            // FAR_CHEB: BF16 hi / lo images of the tables for the tensor-core L2P
    long long l2p_off[16];        // element offset of level l's images in l2p_img, -1 if none
    // FAR_CHEB, leaves of edge 4 at level D-2: images of the 8 composed tables E L2L_c (the L2L
    // from the parent into child c followed by the child's L2P), at this element offset in
    // l2p_img; -1 if not built
    long long l2pc_off;
    const double *uc64, *dc64;    // FAR_SURFACE FP64 UC2E_l / DC2E_l (row-major n x n), + l * pinv_stride
    long long pinv_stride;
    short *slot_of_code;  // [343] -> 0..315 or -1
    float *nodes;     // [npad][4] unit node positions: Chebyshev nodes in [-1,1]^3 or unit surface points
    float *cheb_t;    // [order] 1D Chebyshev nodes cos((2k+1) pi / (2p))
    double *self_int; // [1]
    Radii r;
};
struct OpsBuildArgs {
    int D, Lmax;
    double h, alpha, beta, eps;
    double *work;      // FP64 scratch; keeps UC2E_l / DC2E_l after the build (FAR_SURFACE)
    OpsDev ops;
};
int ops_build(const OpsBuildArgs &A, cudaStream_t st);
size_t ops_work_doubles(int method, int n, int Lmax);
size_t ops_etab_floats(int method, int npad, int D, int Lmax);
void ops_layout(int D, int Lmax, double *work, OpsDev &O);   // e_off, l2p_off, uc64, dc64, pinv_stride
size_t ops_l2p_img_elems(int D, int Lmax);                  // BF16 elements of every level's L2P images
                                                            // (and the composed L2L + L2P images)

// ---------------------------------------------------------------- FMM passes
struct FmmDev {
    TreeDev T;
    ListDev L;
    OpsDev O;
    const uint32_t *src_pc, *trg_key;   // targets' cells from their keys (key_pc)
    const float *src_q;
    int leaf_l2p_done;   // 1: k_leaf adds near-field terms only where a table L2P already wrote S
    int p2p_separate;    // 1: the U-list near field runs in k_p2p (after k_leaf), not in k_leaf
    int l2p_sep;         // 1: leaves without a table get their L2P from k_l2p_sep (before k_leaf)
    const uint8_t *tmask;   // [nx*ny*nz] 1 at targets (tensor-core L2P of partly selected leaves)
    const float *gtab;      // optional near-field table: g(d2) for integer squared offsets d2 < GTAB_N
    float r_s;              // strategy 3 (skip W boxes whose bounded share is below r_s S_est); 0 = off
    unsigned long long *skip_count;   // (target, W box) pairs skipped by strategy 3
    int *l2p_list = nullptr, *l2p_cnt = nullptr;   // per level (at lvl_base[l]): leaves with targets, [16] counts
    float wscale;
    KParams kp;
    double alpha, beta, C64;   // FP64 kernel constants for the FP64 evaluation paths
    int D, nx, ny, nz, self_mode;
    float *ueq, *dchk;   // [nboxes][PP]: upward / downward check potentials u_B, d_B
    // >= 0: the boxes from this one on (the deepest level, taken by the fused L2L + L2P) have
    // their d rows cleared by the work-list kernel only where they have V or X entries (the
    // others are never read); -1: every row cleared before the passes
    int d_sparse_from = -1;
    // optional [items][near_s] scratch: the near field sums into its leaf's slots (item i of the
    // class-walk order, target t - tb) instead of into the output, so that it can run beside the
    // far-field passes; fmm_near_add adds the slots into the output afterwards
    float *near_buf = nullptr;
    int near_s = 0;
};
// returns the number of kernels launched
int fmm_upward_level(const FmmDev &F, int level, int box_count, const int *list, const int *count, bool leaves_only,
                     cudaStream_t st);
// near-field leaves in classes by their number of kernel evaluations w: class c holds
// P2P_CLASS0 >> c <= w < P2P_CLASS0 >> (c - 1) (class 0: w >= P2P_CLASS0, the last: the rest)
constexpr int P2P_CLASSES = 6;
constexpr int64_t P2P_CLASS0 = 1 << 16;
// p2p_list: P2P_CLASSES lists of p2p_stride slots, p2p_cnt: their P2P_CLASSES counts
// own_list / own_cnt: the deepest-level leaves with targets and V or X entries (where
// F.d_sparse_from >= 0), for fmm_l2p_own
// w_list / w_cnt (optional): the near-field leaves with W entries, each as its slot in the class
// lists (class x p2p_stride + index in the class), for a launch of the W-list pass alone
void fmm_work_lists(const FmmDev &F, int nboxes, int *src_list, int *src_cnt, int *leaf_list, int *leaf_cnt,
                    int *p2p_list, int *p2p_cnt, int p2p_stride, int *own_list, int *own_cnt, cudaStream_t st,
                    int *w_list = nullptr, int *w_cnt = nullptr);
// near field over the U lists (pass 0) and W lists (pass 1) of the leaves in the class lists of
// p2p_list, passes [pass_lo, pass_hi); adds into out, or into F.near_buf where it is set (pass 0
// clears the leaf's slots; a launch of pass 1 alone must follow the one of pass 0).  At most
// per_sm CTAs per SM (grid-stride over the leaves).
// w_list / w_cnt (a launch of pass 1 alone): walk only those leaves (fmm_work_lists), with a
// grid of at most max_w CTAs
void fmm_p2p(const FmmDev &F, int nboxes, const int *p2p_list, const int *p2p_cnt, int stride, float *out,
             cudaStream_t st, int pass_lo = 0, int pass_hi = 2, int per_sm = 16, const int *w_list = nullptr,
             const int *w_cnt = nullptr, int max_w = 0);
// out[cell of t] += F.near_buf[slot of t] for every target of every leaf of those lists
// flags / flags_host (optional): flags[0..2) copied to the mapped host address flags_host once
// every earlier kernel of the stream has completed
void fmm_near_add(const FmmDev &F, int nboxes, const int *p2p_list, const int *p2p_cnt, int stride, float *out,
                  cudaStream_t st,
                  const int *flags = nullptr, int *flags_host = nullptr);
void fmm_m2l_level(const FmmDev &F, int level, int box_begin, int box_count, int m2l_prec, cudaStream_t st);
void fmm_p2l_level(const FmmDev &F, int level, int box_begin, int box_count, cudaStream_t st);
void fmm_down_level(const FmmDev &F, int level, int box_begin, int box_count, cudaStream_t st);
void fmm_leaf(const FmmDev &F, int nboxes, const int *list, const int *count, float *out_dense, cudaStream_t st);
// tensor-core L2P (FAR_CHEB, images present): writes S at the targets of the level's leaves
// L2L into the leaves of edge 4 at `level` fused with their L2P (tensor cores); every box at
// `level` must be a leaf (level == Lmax).  Replaces fmm_l2l_*_level(level) and the L2P of `level`.
void fmm_l2lp_tc_level(const FmmDev &F, int level, int parent_begin, int parent_count, float *out, int *err,
                       cudaStream_t st);
// the L2P of the own local terms of the leaves in list (count[0] <= max_count of them; leaves of
// edge 4 at `level`), added into out at their targets (FP32); the part of the deepest level's
// L2P that fmm_l2lp_tc_level leaves out
void fmm_l2p_own(const FmmDev &F, int level, const int *list, const int *count, int max_count, float *out,
                 cudaStream_t st);
// M2M of the split boxes with sources of `level` on the tensor cores: tiles of 64 boxes from
// the level's source list x one child slot per CTA, added into rows zeroed by the work lists
void fmm_m2m_tc_level(const FmmDev &F, int level, int box_count, const int *list, const int *count,
                      const uint16_t *images, int *err, cudaStream_t st);
void fmm_l2p_tc_level(const FmmDev &F, int level, int box_begin, int box_count, float *out, int *err,
                      cudaStream_t st);
__host__ __device__ int l2p_tile_n(int edge);
// separable L2P of the leaves with targets of one level: list / *count (device) from the work
// lists; box_count (host) bounds the count and sizes the launch
void fmm_l2p_sep_level(const FmmDev &F, int level, const int *list, const int *count, int box_count, float *out,
                       cudaStream_t st);
void fmm_init_attributes();
constexpr int GTAB_N = 4096;           // table of the scaled kernel for squared cell offsets 0 .. 4095
void fmm_near_table(const FmmDev &F, float *gtab, cudaStream_t st);
size_t l2p_image_elems(int edge);
void make_l2p_images(const float *etab, int edge, int n, uint16_t *img, cudaStream_t st);
void fmm_m2l_gemm_level(const FmmDev &F, int level, int box_begin, int box_count, cudaStream_t st);
// V pairs grouped by (level, offset slot): built once per tree, then one M2L launch for all levels.
struct PairsDev {
    int nkeys;            // (Lmax + 1) * 316
    int *cnt, *off;       // [nkeys], [nkeys + 1]
    int *cursor;          // [nkeys]
    int *tile_cnt, *tile_off;   // [nkeys], [nkeys + 1]
    int *trg, *src;       // [nV]
    int *total_tiles;     // [1]
    int *tile_key;        // [nV / 64 + nkeys]: key of every tile (one load instead of a search per CTA)
};
constexpr int VPAIR_TILE = 64;   // V pairs per M2L tile (the tensor-core tile's N)
void fmm_m2l_pairs(const FmmDev &F, const PairsDev &Pd, int nV, int m2l_prec, cudaStream_t st);
// tensor-core (tcgen05, BF16 x3) translations; require npad == 128
bool tc_supported(const OpsDev &O);
void tc_init_attributes();
size_t tc_image_elems(int count);
void make_images(const float *opT, int np, int count, uint16_t *img, cudaStream_t st);
void fmm_m2l_tc(const FmmDev &F, const PairsDev &Pd, int nV, const uint16_t *images, int *err, cudaStream_t st,
                bool pipelined = false,
                bool tile_loop = false, int *ticket = nullptr,   // ticket: a cleared counter (tile loop)
                int loop_ctas = 0);                              // > 0: CTAs of the tile loop (else 2 per SM)
// M2L of every level in target-stationary tiles (tensor cores): groups of up to 128 boxes of one
// level and octant, their V-list sources found by dense lookup (no pair list read)
struct MtLevels {
    int lmin, lmax;
    int gbase[18];      // first group of level l; gbase[lmax + 1] = number of groups
};
MtLevels m2l_tile_levels(int Lmax);
// groups: [number of groups] scratch; ngroups, counter: device ints zeroed before the call
void fmm_m2l_tiles(const FmmDev &F, const MtLevels &ML, int *groups, int *ngroups, int *counter,
                   const uint16_t *images, int *err, cudaStream_t st);
int sm_count();
void fmm_l2l_tc_level(const FmmDev &F, int level, int parent_begin, int parent_count, const uint16_t *images,
                      int *err, cudaStream_t st);
void fmm_l2l_tc8_level(const FmmDev &F, int level, int parent_begin, int parent_count, const uint16_t *images,
                       int *err, cudaStream_t st);
void fmm_l2l_gemm_level(const FmmDev &F, int level, int parent_begin, int parent_count, cudaStream_t st);
void fmm_l2p_gemm_level(const FmmDev &F, int level, int box_begin, int box_count, float *out, cudaStream_t st);

}  // namespace sph
