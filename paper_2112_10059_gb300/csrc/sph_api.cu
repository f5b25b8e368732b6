// C ABI of libsph (declared in include/sph.h): argument checks, context-owned
// device memory, the operator cache and the orchestration of one evaluation.
//
// One evaluation (eval_sph) queues, on the context's stream:
//   selection (Section 3)        -> Morton-ordered source / target points
//   octree + U/V/W/X lists       -> Section 2.4 hierarchy
//   operators (cached)           -> FP64 pseudo-inverses folded into FP32 translations
//   upward pass (P2M, M2M)       -> upward check potentials (Eq. s2l right-hand sides)
//   downward pass (M2L, P2L, L2L)-> downward check potentials
//   leaves (L2P, M2P, P2P)       -> S_ph at every target, 0 elsewhere
// Box and list counts are data dependent: the host reads them back three times
// (after selection, after the tree, after list counting) to size buffers and grids.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <map>
#include <vector>

#include "sph_kernels.cuh"
#include "nn_internal.h"
#include "nn_kernels.cuh"
#include "../../include/sph.h"
#include "../../include/sph_nn.h"

using namespace sph;

namespace {

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
};

}  // namespace

struct sph_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool poisoned = false;
    std::string err;
    // grid / gas
    bool grid_set = false;
    int nx = 0, ny = 0, nz = 0, D = 0;
    double origin[3] = {0, 0, 0};
    double h = 0, pO2 = 0, chi_min = 0, chi_max = 0, alpha = 0, beta = 0;
    // inputs
    bool src_set = false, trg_set = false, crit_set = false;
    const float *q = nullptr;
    double source_scale = 0;
    const float *emag = nullptr;
    const uint8_t *mask = nullptr;
    double i_frac = 0, e_frac = 0, e_app = 0;
    int self_mode = 1, leaf_size = 64, m2l_prec = SPH_M2L_BF16X3;
    int leaf_eff = 64;                // leaf size of the current tree (leaf_size, or the autotuner's choice)
    std::map<std::string, int> tune_cache;
    sph_ctx *tune_owner = nullptr;    // batch slots share their parent's autotuner cache
    // batches: one sub-context (own stream, buffers, operator cache) per snapshot slot
    std::vector<sph_ctx *> subs;
    bool own_stream = false;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<cudaEvent_t> events;
    bool batch_graph = true;
    bool eval_graph = true;             // single evaluations: FMM passes as one captured graph
    cudaGraphExec_t eval_gexec = nullptr;
    std::vector<uint8_t> gexec_sig;   // everything the captured passes depend on (empty: re-capture)
    int64_t gexec_launches = 0;       // kernels in that graph
    // surrogate evaluation: coarse and fine sub-contexts on this context's stream, buffers
    sph_ctx *sur_coarse = nullptr, *sur_fine = nullptr;
    DevBuf s_qc, s_Sc, s_y, s_Sp, s_x, s_Sf, s_mask, s_svox, s_err, s_pe, s_flags, s_counts;
    // results of the last eval
    int64_t ns = 0, nt = 0;
    int nboxes = 0, Lmax = 0;
    std::vector<int> lvl_count, lvl_base, lvl_src;   // boxes, first box, boxes with sources per level
    std::vector<int> lvl_leaf;                       // leaves with targets per level
    std::vector<int> lvl_sleaf;                      // leaves with sources per level
    int list_tot[4] = {0, 0, 0, 0};
    bool have_tree = false;
    int64_t launches = 0;   // kernels queued by the current eval (operator precompute excluded)
    bool translate_per_box = false;   // one CTA per box for M2L / L2L instead of the batched GEMMs
    bool tc_used = false;             // this eval ran the tensor-core translations
    bool l2l_eight = true;            // tensor-core L2L: all 8 children per CTA (else one child per CTA)
    int select_two_pass = 0;          // 1: the reference two-pass selection (maxima alone, every brick read twice)
    int select_lookback = 0;          // 1: one-pass look-back selection instead of count / scan / emit
    bool p2p_in_leaf = false;         // near field inside the leaf kernel (reference form)
    bool l2p_simt = false;            // FP32 SIMT L2P even when the tensor-core images exist
    bool l2p_tc_used = false;         // this eval ran the tensor-core L2P
    bool l2p_tc_tables = false;       // interpolation-table L2P (tensor cores) instead of the separable form
    bool m2l_pipe = false;            // tensor-core M2L as one persistent pipelined CTA per SM (measured slower)
    bool m2l_loop = true;             // tensor-core M2L as two persistent CTAs per SM looping over the tiles
    int m2l_loop_ctas = 0;            // > 0: that many CTAs for the tile loop instead (tests: many tiles per CTA)
    bool brick_offsets = false;       // the last selection left every 16^3 brick's target offset in b_off
    bool near_overlap = true;         // near field on a second stream beside the far-field passes
    int near_per_sm = 0;              // its U-list launch: CTAs per SM (0: by the estimate in fmm_queue)
    cudaStream_t near_stream = nullptr;
    cudaEvent_t near_fork = nullptr, near_join = nullptr, near_up = nullptr, near_l2l = nullptr;
    cudaEvent_t zero_fork = nullptr, zero_done = nullptr;   // the output's zero fill beside the tree build
    DevBuf b_nearbuf;                 // the near field's per-leaf sums (overlapped form)
    unsigned select_wait = SELECT_WAIT_LIMIT;   // look-back polls of the selection (SPH_WAIT_LIMIT_SELECT)
    int fault_alloc = 0;              // > 0: the fault_alloc-th allocation fails (SPH_FAULT=alloc[:k])
    int m2l_tiles = 2;                // tensor-core M2L in target-stationary tiles: 0 never (tiles of V
                                      // pairs), 1 always, 2 where the V lists are dense (>= 32 pairs per box)
    DevBuf b_mtg;                     // groups of the target-stationary M2L
    int m2l_form = -1;                // autotuned M2L form for this eval (-1: the density rule)
    bool m2l_tiles_used = false;      // the last eval ran the target-stationary M2L
    bool l2lp_fused = true;           // deepest level of edge-4 leaves: L2L and L2P in one tensor-core kernel
    bool l2lp_used = false;           // the last eval ran the fused kernel
    bool defer_sync = true;           // fixed leaf size: one host sync for selection, tree and list counts
    int list_cap = 0;                 // slots of every tree level: length of the list count / offset arrays
    int near_mode = SPH_NEAR_EXP;     // requested near-field form
    double r_s = 0.0;                 // strategy 3 ratio (0: off)
    DevBuf b_skip;
    bool near_table = false;          // resolved for the current evaluation
    DevBuf b_gtab;
    // buffers
    DevBuf b_maxes, b_cnt, b_off, b_tot, b_skey, b_spc, b_sq, b_tkey, b_tpc, b_bstat;
    DevBuf b_boxat, b_flag, b_pos, b_rng, b_scan, b_lvl;
    DevBuf b_level, b_key, b_sb, b_se, b_tb, b_te, b_parent, b_leaf;
    DevBuf b_lcnt, b_loff, b_usrc, b_vsrc, b_vocs, b_vtrg, b_wsrc, b_xsrc, b_pkeys, b_ppairs, b_heavy;
    DevBuf b_ueq, b_dchk;
    DevBuf o_work, o_etab, o_m2m, o_l2l, o_m2l, o_m2lbf, o_l2lbf, o_m2mbf, o_slot, o_surf, o_cheb, o_self;
    DevBuf b_err;                // device error flags of the tensor-core tiles
    DevBuf b_work;               // compact work lists: sources per level, leaves for the leaf and P2P kernels
    DevBuf b_tmask;              // [ncell] 1 at targets (written by the selection)
    DevBuf b_near;               // tree: source occupancy and its 3x3x3 dilation per dense slot
    DevBuf o_l2pimg;             // BF16 images of the L2P tables (tensor-core L2P)
    DevBuf h_q, h_e, h_m, h_s;   // device copies for eval_sph_host
    int *pinned = nullptr;       // small pinned host buffer for read-backs
    int *pinned_dev = nullptr;   // its device address (mapped), or null: read-backs then by copies
    bool chain_zeroed = false;   // chain_zero cleared the counters of the selection, tree and lists queued next
    // operator cache key
    bool ops_valid = false;
    int ops_D = -1, ops_L = -1;
    double ops_h = 0, ops_a = 0, ops_b = 0, ops_eps = 0;
    bool ops_bf = false;
    double self_int = 0;
    double pinv_eps = 1e-5;
    Radii radii = RADII_DEFAULT;
    Radii ops_r = {0, 0, 0, 0};
    int far_method = FAR_CHEB, far_order = 5;
    int ops_method = -1, ops_order = -1;
    int npad() const { return pad16(far_n(far_method, far_order)); }
};

namespace {

int fail(sph_ctx *c, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

int cuda_fail(sph_ctx *c, cudaError_t e, const char *where) {
    c->poisoned = true;
    return fail(c, SPH_ECUDA, "CUDA error in %s: %s", where, cudaGetErrorString(e));
}

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call);     \
    } while (0)

// Wait limit from the environment (tests lower it to make a bounded wait run out), else `dflt`.
unsigned env_limit(const char *name, unsigned dflt) {
    const char *e = getenv(name);
    if (!e || !*e) return dflt;
    char *end = nullptr;
    const unsigned long v = strtoul(e, &end, 10);
    return (end && *end == 0) ? (unsigned)v : dflt;
}

int ensure(sph_ctx *c, DevBuf &b, size_t bytes) {
    if (bytes <= b.cap && b.p) return SPH_OK;
    // injected failure (SPH_FAULT=alloc[:k] at context creation): the k-th allocation that
    // would call cudaMalloc fails as if the device were out of memory, then injection stops
    if (c->fault_alloc > 0 && --c->fault_alloc == 0)
        return fail(c, SPH_ENOMEM, "injected allocation failure (SPH_FAULT) for %zu bytes", bytes);
    if (b.p) {
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "stream sync before realloc");
        cudaFree(b.p);
        b.p = nullptr;
        b.cap = 0;
    }
    size_t want = std::max<size_t>(bytes, 256);
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return fail(c, SPH_ENOMEM, "cudaMalloc(%zu) failed: %s", want, cudaGetErrorString(e));
    }
    b.cap = want;
    return SPH_OK;
}

#define ENS(buf, bytes)                                  \
    do {                                                 \
        int r_ = ensure(c, (buf), (bytes));              \
        if (r_ != SPH_OK) return r_;                     \
    } while (0)

template <class T>
T *P(DevBuf &b) { return (T *)b.p; }

int depth_of(int nx, int ny, int nz) {
    int m = std::max(nx, std::max(ny, nz)), D = 0;
    while ((1 << D) < m) ++D;
    return D;
}

int check_ready(sph_ctx *c) {
    if (!c) return SPH_EINVAL;
    if (c->poisoned) return fail(c, SPH_ECUDA, "context poisoned by an earlier CUDA error");
    if (!c->grid_set) return fail(c, SPH_ESTATE, "set_grid has not been called");
    if (!c->src_set) return fail(c, SPH_ESTATE, "set_sources has not been called");
    if (!c->trg_set) return fail(c, SPH_ESTATE, "set_targets has not been called");
    if (!c->crit_set) return fail(c, SPH_ESTATE, "set_criteria has not been called");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    return SPH_OK;
}

KParams make_kp(const sph_ctx *c) {
    KParams k;
    memset(static_cast<void *>(&k), 0, sizeof k);
    const double log2e = 1.4426950408889634;
    double L = std::log(c->beta / c->alpha);
    k.a2 = (float)(c->alpha * log2e);
    k.b2 = (float)((c->beta - c->alpha) * log2e);
    k.bma = (float)(c->beta - c->alpha);
    k.C = (float)(1.0 / (4.0 * M_PI * L));
    k.h = (float)c->h;
    k.gself = (float)(c->self_int / (c->h * c->h * c->h));
    return k;
}

// Selection into Morton-ordered point arrays; reads back (Ns, Nt).
// ------------------------------------------------------------------ selection
// copy: read the totals back by a copy (else the list layout kernel writes them into the mapped
// read-back buffer before the host's sync)
int select_queue(sph_ctx *c, bool copy = true) {
    const int D = c->D;
    const int b = std::min(4, D);
    const int64_t nbr = 1ll << (3 * (D - b));
    const int64_t ncell = (int64_t)c->nx * c->ny * c->nz;
    ENS(c->b_maxes, 2 * sizeof(unsigned));
    ENS(c->b_cnt, 2 * nbr * sizeof(int));
    ENS(c->b_off, 2 * nbr * sizeof(int));
    ENS(c->b_tot, 16 * sizeof(int));
    ENS(c->b_skey, ncell * sizeof(uint32_t));
    ENS(c->b_spc, ncell * sizeof(uint32_t));
    ENS(c->b_sq, ncell * sizeof(float));
    ENS(c->b_tkey, ncell * sizeof(uint32_t));
    ENS(c->b_tmask, ncell);
    ENS(c->b_bstat, nbr * 4 * sizeof(float));
    SelectArgs A;
    A.nx = c->nx; A.ny = c->ny; A.nz = c->nz; A.D = D; A.brick_log2 = b;
    A.q = c->q; A.emag = c->emag; A.mask = c->mask;
    A.i_frac = c->i_frac; A.e_frac = c->e_frac; A.e_app = c->e_app;
    A.maxes = P<unsigned>(c->b_maxes);
    A.two_pass = c->select_two_pass;
    A.lookback = c->select_lookback;
    A.wait_limit = c->select_wait;
    A.cnt_s = P<int>(c->b_cnt); A.cnt_t = A.cnt_s + nbr;
    A.off_s = P<int>(c->b_off); A.off_t = A.off_s + nbr;
    A.totals = P<int>(c->b_tot);
    A.src_key = P<uint32_t>(c->b_skey); A.src_pc = P<uint32_t>(c->b_spc); A.src_q = P<float>(c->b_sq);
    A.trg_key = P<uint32_t>(c->b_tkey);   // targets' cells follow from their keys: no packed copy
    A.tmask = P<uint8_t>(c->b_tmask);
    A.bstat = P<float>(c->b_bstat);
    A.zeroed = c->chain_zeroed;
    const int sr = select_launch(A, c->stream);
    if (sr < 0) CK(cudaGetLastError());
    c->brick_offsets = sr == 1 && b == 4;
    c->launches += A.launched;
    if (copy) CK(cudaMemcpyAsync(c->pinned, A.totals, 3 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    return SPH_OK;
}

// after the stream has been synchronised
int select_read(sph_ctx *c) {
    if (c->pinned[0] < 0 || c->pinned[1] < 0 || (!c->select_two_pass && c->pinned[2] != 0))
        return fail(c, SPH_ETIMEOUT, "selection look-back gave up waiting for a preceding brick");
    c->ns = c->pinned[0];
    c->nt = c->pinned[1];
    return SPH_OK;
}

int run_select(sph_ctx *c) {
    int r = select_queue(c);
    if (r) return r;
    CK(cudaStreamSynchronize(c->stream));
    return select_read(c);
}

TreeDev tree_dev(sph_ctx *c) {
    TreeDev T;
    memset(static_cast<void *>(&T), 0, sizeof T);
    T.box_at = P<int>(c->b_boxat);
    T.lvl_base = P<int>(c->b_lvl);
    T.lvl_count = T.lvl_base + 16;
    T.lvl_src = T.lvl_base + 32;
    T.lvl_leaf = T.lvl_base + 48;
    T.lvl_sleaf = T.lvl_base + 64;
    T.b_level = P<int>(c->b_level);
    T.b_key = P<uint32_t>(c->b_key);
    T.b_sb = P<int>(c->b_sb); T.b_se = P<int>(c->b_se);
    T.b_tb = P<int>(c->b_tb); T.b_te = P<int>(c->b_te);
    T.b_parent = P<int>(c->b_parent);
    T.b_leaf = P<uint8_t>(c->b_leaf);
    T.near = c->Lmax >= 1 ? P<uint8_t>(c->b_near) + dense_off(c->Lmax + 1) : nullptr;
    T.vsrc = P<uint8_t>(c->b_near) + 2 * dense_off(c->Lmax + 1);
    return T;
}

ListDev list_dev(sph_ctx *c) {
    ListDev L;
    memset(static_cast<void *>(&L), 0, sizeof L);
    int nb = std::max(c->list_cap, 1);
    int *cnt = P<int>(c->b_lcnt), *off = P<int>(c->b_loff);
    L.u_cnt = cnt; L.v_cnt = cnt + nb; L.w_cnt = cnt + 2 * nb; L.x_cnt = cnt + 3 * nb;
    L.u_off = off; L.v_off = off + (nb + 1); L.w_off = off + 2 * (nb + 1); L.x_off = off + 3 * (nb + 1);
    L.u_src = P<int>(c->b_usrc); L.v_src = P<int>(c->b_vsrc); L.w_src = P<int>(c->b_wsrc);
    L.x_src = P<int>(c->b_xsrc);
    L.v_oc = P<short>(c->b_vocs);
    L.v_trg = P<int>(c->b_vtrg);
    L.heavy = P<int>(c->b_heavy);
    L.nheavy = P<int>(c->b_tot) + 8;
    return L;
}

// V pairs grouped by (level, offset) key: per-key arrays in b_pkeys (sized at the list count),
// the pairs and the tile -> key table in b_ppairs (sized at the list fill)
PairsDev pairs_dev(sph_ctx *c) {
    PairsDev Pd;
    memset(static_cast<void *>(&Pd), 0, sizeof Pd);
    const int nkeys = (c->Lmax + 1) * NSLOT;
    const int nV = std::max(c->list_tot[1], 1);
    int *pk = P<int>(c->b_pkeys);
    Pd.nkeys = nkeys;
    Pd.cnt = pk; Pd.off = pk + nkeys; Pd.cursor = pk + 2 * nkeys + 1;
    Pd.tile_cnt = pk + 3 * nkeys + 1; Pd.tile_off = pk + 4 * nkeys + 1;
    Pd.total_tiles = pk + 5 * nkeys + 2;
    int *pp = P<int>(c->b_ppairs);
    Pd.trg = pp; Pd.src = pp ? pp + nV : nullptr;
    Pd.tile_key = pp ? pp + 2 * (size_t)nV : nullptr;
    return Pd;
}

// ------------------------------------------------------------------ tree and lists
// pinned read-back slots: [0..3) selection totals, [8..40) level bases / counts,
// [43] scan give-up flag, [44..48) list totals, [48] and [49] tensor-core error flags,
// [64..64+Lmax] boxes with sources per level, [80..80+Lmax] leaves with targets per level,
// [96..96+Lmax] leaves with sources per level.
// The tree and the list counts read the selection's point counts and the tree's box count
// from device memory, so selection, tree and list counting need one host sync in all.
// deepest level: leaves of the effective leaf size hold at most 8^k cells
int lmax_of(const sph_ctx *c) {
    int k = 0;
    while (k < 4 && (1ll << (3 * (k + 1))) <= c->leaf_eff) ++k;
    return std::max(0, c->D - k);
}

// The scan scratch: the tree scan's region first, then the list scan's (separate look-back
// states, so that both can be cleared before the evaluation)
int64_t scan_list_off(int64_t dense_total) { return (int64_t)scan_tmp_ints((int)(4 * (dense_total + 1))); }
size_t scan_scratch_bytes(int64_t dense_total) {
    return (size_t)(scan_list_off(dense_total) + (int64_t)scan_tmp_ints((int)(dense_total + 1))) * sizeof(int) + 64;
}

int tree_queue(sph_ctx *c) {
    const int D = c->D;
    int S = c->leaf_eff;
    const int Lmax = lmax_of(c);
    c->Lmax = Lmax;
    const int64_t dense_total = dense_off(Lmax + 1);
    ENS(c->b_boxat, dense_total * sizeof(int));
    ENS(c->b_flag, dense_total * sizeof(int));
    ENS(c->b_pos, (dense_total + 1) * sizeof(int));
    ENS(c->b_rng, 4 * dense_total * sizeof(int));
    ENS(c->b_near, 3 * dense_total + 16);
    ENS(c->b_scan, scan_scratch_bytes(dense_total));
    ENS(c->b_lvl, 80 * sizeof(int));
    const int64_t cap = dense_total;   // every slot of every level could hold a box
    ENS(c->b_level, cap * sizeof(int));
    ENS(c->b_key, cap * sizeof(uint32_t));
    ENS(c->b_sb, cap * sizeof(int)); ENS(c->b_se, cap * sizeof(int));
    ENS(c->b_tb, cap * sizeof(int)); ENS(c->b_te, cap * sizeof(int));
    ENS(c->b_parent, cap * sizeof(int));
    ENS(c->b_leaf, cap);
    TreeArgs A;
    A.T = tree_dev(c);
    A.ns_dev = P<int>(c->b_tot); A.nt_dev = P<int>(c->b_tot) + 1;
    A.ncap = (int)std::min<int64_t>((int64_t)c->nx * c->ny * c->nz, INT32_MAX);
    A.S = S; A.D = D; A.Lmax = Lmax;
    c->list_cap = (int)dense_total;
    A.skey = P<uint32_t>(c->b_skey); A.tkey = P<uint32_t>(c->b_tkey);
    A.flag = P<int>(c->b_flag); A.pos = P<int>(c->b_pos);
    A.rsb = P<int>(c->b_rng); A.rse = A.rsb + dense_total; A.rtb = A.rse + dense_total; A.rte = A.rtb + dense_total;
    A.occ = P<uint8_t>(c->b_near); A.near = A.occ + dense_total; A.vsrc = A.occ + 2 * dense_total;
    A.scan_tmp = P<int>(c->b_scan);
    A.err = P<int>(c->b_tot) + 3;
    if (c->brick_offsets && D >= 4) {
        A.nbr = 1 << (3 * (D - 4));
        A.brick_off_t = P<int>(c->b_off) + A.nbr;       // off_t follows off_s (select_queue)
    }
    A.zeroed = c->chain_zeroed;
    if (!A.zeroed) CK(cudaMemsetAsync(A.err, 0, sizeof(int), c->stream));
    tree_build_launch(A, c->stream);
    // ranges (sources and targets in one launch), existence flags, scan, emit (with the source
    // occupancy), the occupancy's dilation
    c->launches += 1 + 3 + (Lmax >= 1 ? 1 : 0);
    CK(cudaGetLastError());
    if (!c->pinned_dev) {   // else written by the list layout kernel (lists_count_queue)
        CK(cudaMemcpyAsync(c->pinned + 8, A.T.lvl_base, 32 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaMemcpyAsync(c->pinned + 64, A.T.lvl_src, 48 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    }
    return SPH_OK;
}

// after tree_queue, no sync: the list counts over every slot (the box count stays on the
// device), their offsets, the V pairs per key; totals and the scans' flag read back
int lists_count_queue(sph_ctx *c) {
    const int Lmax = c->Lmax;
    const int cap = std::max(c->list_cap, 1);
    ENS(c->b_lcnt, 4 * (size_t)cap * sizeof(int));
    ENS(c->b_loff, 4 * (size_t)(cap + 1) * sizeof(int));
    ENS(c->b_heavy, (size_t)cap * sizeof(int));
    const int nkeys = (Lmax + 1) * NSLOT;
    ENS(c->b_pkeys, (5 * (size_t)nkeys + 10) * sizeof(int));
    if (!c->chain_zeroed) CK(cudaMemsetAsync(c->b_pkeys.p, 0, (5 * (size_t)nkeys + 10) * sizeof(int), c->stream));
    ENS(c->b_scan, scan_scratch_bytes(cap));
    ListDev L = list_dev(c);
    int *ltot = P<int>(c->b_tot) + 4;
    const int *nboxes_dev = P<int>(c->b_pos) + dense_off(Lmax + 1);   // the tree scan's total
    // the layout kernel writes the host's read-backs (selection totals, scan flag, list totals,
    // level arrays) into the mapped buffer
    ReadBack R{};
    R.dst = c->pinned_dev;
    R.sel = P<int>(c->b_tot);
    R.flag_tot = ltot - 1;
    R.lvl = tree_dev(c).lvl_base;
    const bool rb = lists_count_launch(tree_dev(c), L, pairs_dev(c), c->list_cap, nboxes_dev, c->D, Lmax,
                                       P<int>(c->b_scan) + scan_list_off(cap), ltot, ltot - 1, R, c->stream,
                                       c->chain_zeroed);
    c->chain_zeroed = false;
    c->launches += 4;   // classify, count, list scan, lists / pairs layout
    CK(cudaGetLastError());
    if (!rb) {
        CK(cudaMemcpyAsync(c->pinned, R.sel, 3 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaMemcpyAsync(c->pinned + 8, R.lvl, 32 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaMemcpyAsync(c->pinned + 64, R.lvl + 32, 48 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaMemcpyAsync(c->pinned + 43, ltot - 1, 5 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    }
    return SPH_OK;
}

// Before the deferred selection, tree build and list counts: one kernel clears every counter
// and look-back state they need cleared (the selection's maxima and look-back flag, the tree
// scans' flag, the per-level source and leaf counts, the slots' source ranges, the heavy-box
// count, the V-pair key counts and both scans' states) instead of a clearing copy before each
// user, which would stand between two kernels of the launch sequence.
int chain_zero(sph_ctx *c) {
    c->chain_zeroed = false;
    const int Lmax = lmax_of(c);
    const int64_t dense_total = dense_off(Lmax + 1);
    const int nkeys = (Lmax + 1) * NSLOT;
    ENS(c->b_maxes, 2 * sizeof(unsigned));
    ENS(c->b_tot, 16 * sizeof(int));
    ENS(c->b_rng, 4 * dense_total * sizeof(int));
    ENS(c->b_scan, scan_scratch_bytes(dense_total));
    ENS(c->b_lvl, 80 * sizeof(int));
    ENS(c->b_pkeys, (5 * (size_t)nkeys + 10) * sizeof(int));
    ZeroSet Z;
    const bool ok =
        Z.add(P<int>(c->b_maxes), 2) && Z.add(P<int>(c->b_tot) + 2, 2) && Z.add(P<int>(c->b_tot) + 8, 1) &&
        Z.add(P<int>(c->b_rng), 2 * dense_total) && Z.add(P<int>(c->b_lvl) + 32, 48) &&
        Z.add(P<int>(c->b_scan), (int64_t)(scan_state_bytes(1, (int)dense_total) / sizeof(int))) &&
        Z.add(P<int>(c->b_scan) + scan_list_off(dense_total),
              (int64_t)(scan_state_bytes(4, (int)dense_total) / sizeof(int))) &&
        Z.add(P<int>(c->b_pkeys), 5 * (int64_t)nkeys + 10);
    if (!ok) return SPH_OK;   // each user then clears its own
    zero_set_launch(Z, c->stream);
    CK(cudaGetLastError());
    c->launches += 1;
    c->chain_zeroed = true;
    return SPH_OK;
}

// after the sync: level counts -> box count (the scans' flag covers the tree and the list counts)
int tree_levels_read(sph_ctx *c) {
    const int Lmax = c->Lmax;
    if (c->pinned[43] != 0) return fail(c, SPH_ETIMEOUT, "a tree or list scan gave up waiting for a preceding tile");
    c->lvl_count.assign(Lmax + 1, 0);
    c->lvl_base.assign(Lmax + 1, 0);
    c->lvl_src.assign(Lmax + 1, 0);
    c->lvl_leaf.assign(Lmax + 1, 0);
    c->lvl_sleaf.assign(Lmax + 1, 0);
    int64_t tot = 0;
    for (int l = 0; l <= Lmax; ++l) {
        c->lvl_src[l] = c->pinned[64 + l];
        c->lvl_leaf[l] = c->pinned[80 + l];
        c->lvl_sleaf[l] = c->pinned[96 + l];
        c->lvl_count[l] = c->pinned[8 + 16 + l];
        if (c->lvl_src[l] < 0 || c->lvl_src[l] > c->pinned[8 + 16 + l] || c->lvl_leaf[l] < 0 ||
            c->lvl_leaf[l] > c->pinned[8 + 16 + l] || c->lvl_sleaf[l] < 0 || c->lvl_sleaf[l] > c->lvl_src[l])
            return fail(c, SPH_ETIMEOUT, "inconsistent level counts from the tree build");
        if (c->lvl_count[l] < 0) return fail(c, SPH_ETIMEOUT, "inconsistent level counts from the tree build");
        c->lvl_base[l] = (int)tot;
        tot += c->lvl_count[l];
    }
    if (tot > dense_off(Lmax + 1)) return fail(c, SPH_ETIMEOUT, "inconsistent level counts from the tree build");
    c->nboxes = (int)tot;
    return SPH_OK;
}

// after a sync: list totals -> buffers; queue the list fill
int lists_fill(sph_ctx *c) {
    if (c->pinned[43] != 0) return fail(c, SPH_ETIMEOUT, "a list scan gave up waiting for a preceding tile");
    for (int i = 0; i < 4; ++i) c->list_tot[i] = c->pinned[44 + i];
    ENS(c->b_usrc, std::max(1, c->list_tot[0]) * sizeof(int));
    ENS(c->b_vsrc, std::max(1, c->list_tot[1]) * sizeof(int));
    ENS(c->b_vocs, std::max(1, c->list_tot[1]) * sizeof(short));
    ENS(c->b_vtrg, std::max(1, c->list_tot[1]) * sizeof(int));
    ENS(c->b_wsrc, std::max(1, c->list_tot[2]) * sizeof(int));
    ENS(c->b_xsrc, std::max(1, c->list_tot[3]) * sizeof(int));
    {
        const size_t nV = std::max(1, c->list_tot[1]), nkeys = (size_t)(c->Lmax + 1) * NSLOT;
        ENS(c->b_ppairs, (2 * nV + nV / 64 + nkeys + 1) * sizeof(int));
    }
    ListDev L = list_dev(c);
    int *ltot = P<int>(c->b_tot) + 4;
    lists_fill_launch(tree_dev(c), L, pairs_dev(c), c->nboxes, c->D, c->Lmax, ltot, c->stream);
    if (c->nboxes > 0) c->launches += 1;   // fill (with the tiles' keys)
    CK(cudaGetLastError());
    c->have_tree = true;
    return SPH_OK;
}

int run_tree(sph_ctx *c) {
    int r = tree_queue(c);
    if (!r) r = lists_count_queue(c);
    if (r) return r;
    CK(cudaStreamSynchronize(c->stream));
    r = tree_levels_read(c);
    if (r) return r;
    return lists_fill(c);
}

void fill_ops(sph_ctx *c, OpsDev &O, int D, int L, bool bf) {
    O.method = c->far_method;
    O.order = c->far_order;
    O.n = far_n(c->far_method, c->far_order);
    O.npad = pad16(O.n);
    O.e_tab = P<float>(c->o_etab);
    O.r = c->radii;
    O.m2m_t = P<float>(c->o_m2m); O.l2l_t = P<float>(c->o_l2l);
    O.m2l_t = P<float>(c->o_m2l);
    const bool img = bf && O.npad == 128;
    O.m2l_img = img ? P<uint16_t>(c->o_m2lbf) : nullptr;
    O.l2l_img = img ? P<uint16_t>(c->o_l2lbf) : nullptr;
    O.m2m_img = (img && c->far_method == FAR_CHEB) ? P<uint16_t>(c->o_m2mbf) : nullptr;
    O.l2p_img = (img && c->far_method == FAR_CHEB) ? P<uint16_t>(c->o_l2pimg) : nullptr;
    O.slot_of_code = P<short>(c->o_slot);
    O.nodes = P<float>(c->o_surf);
    O.cheb_t = P<float>(c->o_cheb);
    O.self_int = P<double>(c->o_self);
    ops_layout(D, L, P<double>(c->o_work), O);
}

int run_ops(sph_ctx *c) {
    bool want_bf = c->m2l_prec == SPH_M2L_BF16X3;
    if (c->ops_valid && c->ops_D == c->D && c->ops_L >= c->Lmax && c->ops_h == c->h && c->ops_a == c->alpha &&
        c->ops_b == c->beta && c->ops_eps == c->pinv_eps && (c->ops_bf || !want_bf) &&
        c->ops_method == c->far_method && c->ops_order == c->far_order &&
        c->ops_r.ue == c->radii.ue && c->ops_r.uc == c->radii.uc && c->ops_r.dc == c->radii.dc &&
        c->ops_r.de == c->radii.de)
        return SPH_OK;
    const int L = c->Lmax;
    const int n = far_n(c->far_method, c->far_order), np = pad16(n);
    const size_t PP2 = (size_t)np * np;
    ENS(c->o_work, ops_work_doubles(c->far_method, n, L) * sizeof(double));
    ENS(c->o_etab, ops_etab_floats(c->far_method, np, c->D, L) * sizeof(float));
    ENS(c->o_m2m, (L + 1) * 8 * PP2 * sizeof(float));
    ENS(c->o_l2l, (L + 1) * 8 * PP2 * sizeof(float));
    ENS(c->o_m2l, (L + 1) * 316 * PP2 * sizeof(float));
    if (want_bf && np == 128) {
        ENS(c->o_m2lbf, tc_image_elems((L + 1) * 316) * sizeof(uint16_t));
        ENS(c->o_l2lbf, tc_image_elems((L + 1) * 8) * sizeof(uint16_t));
        if (c->far_method == FAR_CHEB) ENS(c->o_m2mbf, tc_image_elems((L + 1) * 8) * sizeof(uint16_t));
        if (c->far_method == FAR_CHEB) ENS(c->o_l2pimg, (ops_l2p_img_elems(c->D, L) + 64) * sizeof(uint16_t));
    }
    ENS(c->o_slot, 343 * sizeof(short));
    ENS(c->o_surf, (size_t)np * 4 * sizeof(float));
    ENS(c->o_cheb, 16 * sizeof(float));
    ENS(c->o_self, 4 * sizeof(double));
    OpsBuildArgs A;
    A.D = c->D; A.Lmax = L; A.h = c->h; A.alpha = c->alpha; A.beta = c->beta; A.eps = c->pinv_eps;
    A.work = P<double>(c->o_work);
    fill_ops(c, A.ops, c->D, L, want_bf);
    if (ops_build(A, c->stream) != 0) CK(cudaGetLastError());
    double si = 0;
    CK(cudaMemcpyAsync(&si, A.ops.self_int, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->self_int = si;
    c->ops_valid = true;
    c->ops_D = c->D; c->ops_L = L; c->ops_h = c->h; c->ops_a = c->alpha; c->ops_b = c->beta;
    c->ops_eps = c->pinv_eps;
    c->ops_bf = want_bf;
    c->ops_r = c->radii;
    c->ops_method = c->far_method;
    c->ops_order = c->far_order;
    return SPH_OK;
}

OpsDev ops_dev(sph_ctx *c) {
    OpsDev O;
    memset(static_cast<void *>(&O), 0, sizeof O);
    fill_ops(c, O, c->ops_D, c->ops_L, c->ops_bf);
    O.r = c->ops_r;
    return O;
}

struct PhaseTimer {
    cudaEvent_t ev[16];
    bool on = false;
    int n = 0;
    void start(bool enable, cudaStream_t st) {
        on = enable;
        if (!on) return;
        for (auto &e : ev) cudaEventCreate(&e);
        n = 0;
        mark(st);
    }
    void mark(cudaStream_t st) {
        if (on && n < 16) {
            rec[n] = true;
            cudaEventRecord(ev[n++], st);
        }
    }
    void mark_at(int k, cudaStream_t st) {   // record event k (events between may stay unrecorded)
        if (on && k < 16) {
            // inside a graph capture the record must become an event-record node of the graph
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            cudaStreamIsCapturing(st, &cs);
            if (cs == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(ev[k], st, cudaEventRecordExternal);
            else cudaEventRecord(ev[k], st);
            rec[k] = true;
            n = std::max(n, k + 1);
        }
    }
    bool rec[16] = {};
    float ms(int a, int b) {     // 0 unless both events were recorded in this eval
        float m = 0;
        if (on && a < 16 && b < 16 && rec[a] && rec[b]) cudaEventElapsedTime(&m, ev[a], ev[b]);
        return m;
    }
    ~PhaseTimer() {
        if (on)
            for (auto &e : ev) cudaEventDestroy(e);
    }
};

// ------------------------------------------------------------------ FMM passes
struct PassState {
    FmmDev F;
    int *w_src = nullptr, *w_leaf = nullptr, *w_p2p = nullptr, *w_cnt = nullptr, *w_own = nullptr, *w_wl = nullptr;
    PairsDev Pd;
    int *err = nullptr;
    bool tc = false;
    MtLevels ML;                 // target-stationary M2L: groups per level
    int *mt_groups = nullptr;    // [groups] scratch of that M2L
    bool fused = false;          // the last L2L and the L2P of the deepest level in one kernel
};

// the last L2L and the L2P of the deepest level fused (every box there a leaf of edge 4)
bool l2lp_fusable(const sph_ctx *c, const PassState &S) {
    const FmmDev &F = S.F;
    return S.tc && c->l2lp_fused && F.leaf_l2p_done && F.O.l2p_img != nullptr && !c->l2p_simt &&
           F.O.l2pc_off >= 0 && c->Lmax >= 3 && c->Lmax == c->D - 2 && F.O.l2p_off[c->Lmax] >= 0;
}

// Every buffer the passes need (so that fmm_queue allocates nothing and can be captured).
int fmm_prepare(sph_ctx *c, PassState &S) {
    const int nb = c->nboxes;
    const size_t vb = (size_t)std::max(nb, 1) * c->npad() * sizeof(float);
    ENS(c->b_ueq, vb);
    ENS(c->b_dchk, vb);
    ENS(c->b_work, ((5 + P2P_CLASSES) * (size_t)std::max(nb, 1) + 64) * sizeof(int));
    ENS(c->b_err, 16 * sizeof(int));
    FmmDev &F = S.F;
    F.T = tree_dev(c);
    F.L = list_dev(c);
    F.O = ops_dev(c);
    F.src_pc = P<uint32_t>(c->b_spc);
    F.trg_key = P<uint32_t>(c->b_tkey);
    F.src_q = P<float>(c->b_sq);
    F.wscale = (float)(c->source_scale * c->h * c->h * c->h);
    F.kp = make_kp(c);
    F.D = c->D; F.nx = c->nx; F.ny = c->ny; F.nz = c->nz; F.self_mode = c->self_mode;
    F.ueq = P<float>(c->b_ueq); F.dchk = P<float>(c->b_dchk);
    F.alpha = c->alpha; F.beta = c->beta; F.C64 = 1.0 / (4.0 * M_PI * std::log(c->beta / c->alpha));
    F.leaf_l2p_done = (!c->translate_per_box && F.O.method == FAR_CHEB) ? 1 : 0;
    F.p2p_separate = c->p2p_in_leaf ? 0 : 1;
    F.l2p_sep = (F.leaf_l2p_done && F.O.method == FAR_CHEB && !c->l2p_simt) ? 1 : 0;
    F.tmask = P<uint8_t>(c->b_tmask);
    F.gtab = nullptr;
    F.r_s = (float)c->r_s;
    ENS(c->b_skip, 2 * sizeof(unsigned long long));
    F.skip_count = P<unsigned long long>(c->b_skip);
    if (c->near_table && F.p2p_separate) {
        ENS(c->b_gtab, GTAB_N * sizeof(float));
        F.gtab = P<float>(c->b_gtab);
    }
    S.w_src = P<int>(c->b_work);
    S.w_leaf = S.w_src + std::max(nb, 1);
    S.w_p2p = S.w_leaf + std::max(nb, 1);                   // P2P_CLASSES lists of max(nb, 1) slots
    S.w_cnt = S.w_p2p + P2P_CLASSES * std::max(nb, 1);
    F.l2p_list = S.w_cnt + 64;                  // [nb], per level at lvl_base[l]
    S.w_own = F.l2p_list + std::max(nb, 1);     // [nb]: deepest-level leaves with V / X entries, count w_cnt[62]
    S.w_wl = S.w_own + std::max(nb, 1);         // [nb]: near-field leaves with W entries, count w_cnt[39]
    F.l2p_cnt = S.w_cnt + 40;                   // [16]
    S.Pd = pairs_dev(c);
    S.err = P<int>(c->b_err);
    S.tc = c->m2l_prec == SPH_M2L_BF16X3 && F.O.m2l_img != nullptr && !c->translate_per_box;
    // the near field beside the far-field passes (from the end of the upward pass, whose
    // equivalent densities its W-list part reads): its sums go to per-leaf slots and are added
    // into the output after the L2P.  Strategy 3 reads the L2P's far field, so it keeps the
    // near field after the L2P.
    if (F.p2p_separate && c->near_overlap && c->r_s == 0.0) {
        int64_t leaves = 0;
        for (int l = 0; l <= c->Lmax; ++l) leaves += c->lvl_leaf[l];
        ENS(c->b_nearbuf, (size_t)std::max<int64_t>(leaves, 1) * c->leaf_eff * sizeof(float));
        F.near_buf = P<float>(c->b_nearbuf);
        F.near_s = c->leaf_eff;
        if (!c->near_stream) CK(cudaStreamCreateWithFlags(&c->near_stream, cudaStreamNonBlocking));
        if (!c->near_fork) CK(cudaEventCreateWithFlags(&c->near_fork, cudaEventDisableTiming));
        if (!c->near_join) CK(cudaEventCreateWithFlags(&c->near_join, cudaEventDisableTiming));
        if (!c->near_up) CK(cudaEventCreateWithFlags(&c->near_up, cudaEventDisableTiming));
        if (!c->near_l2l) CK(cudaEventCreateWithFlags(&c->near_l2l, cudaEventDisableTiming));
    }
    // the fused deepest level reads only the d rows of leaves with V or X entries: the rows of
    // that level are then cleared one by one by the work lists, the levels above by a memset
    S.fused = l2lp_fusable(c, S);
    F.d_sparse_from = S.fused && c->lvl_count[c->Lmax - 1] > 0 ? c->lvl_base[c->Lmax] : -1;
    S.ML = m2l_tile_levels(c->Lmax);
    if (S.tc && c->m2l_tiles) {
        ENS(c->b_mtg, (size_t)std::max(1, S.ML.gbase[S.ML.lmax + 1]) * sizeof(int));
        S.mt_groups = P<int>(c->b_mtg);
    }
    tc_init_attributes();
    fmm_init_attributes();
    return SPH_OK;
}

// The M2L form: target-stationary tiles pay a round per (group, offset) whatever the number of
// pairs in it, so they are taken where the lists are dense (uniform trees), the tiles of V pairs
// elsewhere (an autotuned choice overrides the density rule).
bool m2l_target_tiles(const sph_ctx *c, const PassState &S) {
    const int64_t nV = c->list_tot[1], nb = c->nboxes;
    return S.tc && (c->m2l_tiles == 1 ||
                    (c->m2l_tiles == 2 && (c->m2l_form >= 0 ? c->m2l_form == 1 : nV >= 32 * nb)));
}

// CTAs per SM of the overlapped near field's U-list launch.  Where the far-field chain is the
// longer of the two, 6 (measured best at the 256^3 headline) leave slots to its kernels; where
// the near field is the longer one (every cell a source: the uniform 128^3 tree), it gets the
// whole machine (16; measured best there).  Estimates from the list totals: near-field
// evaluations at most U entries x leaf size^2 at 1.6e12/s; far field a fixed 150 us plus the
// M2L at its measured cost per V pair (0.45 ns in pair tiles, 0.19 ns in target tiles).
int near_cap(const sph_ctx *c, const PassState &S) {
    if (c->near_per_sm > 0) return c->near_per_sm;
    const double s = c->leaf_eff;
    const double near_us = (double)c->list_tot[0] * s * s / 1.6e6;
    const double far_us = 150.0 + (double)c->list_tot[1] * (m2l_target_tiles(c, S) ? 0.19e-3 : 0.45e-3);
    return near_us > far_us ? 16 : 6;
}

// Queue the passes on c->stream: memsets and kernels only (no allocation, no sync).
int fmm_queue(sph_ctx *c, PassState &S, float *out, PhaseTimer *tm) {
    FmmDev &F = S.F;
    const int nb = c->nboxes;
    const size_t vb = (size_t)std::max(nb, 1) * c->npad() * sizeof(float);
    const size_t db = F.d_sparse_from >= 0 ? (size_t)F.d_sparse_from * c->npad() * sizeof(float) : vb;
    // one clearing kernel: the downward states (rows the M2L, P2L and L2L add into), the work
    // list counters, the tensor-core tiles' flags ([0] M2M / M2L / L2L, [1] L2P) and the near
    // field's skip count
    {
        ZeroSet Z;
        const bool ok = Z.add(P<int>(c->b_dchk), (int64_t)(db / sizeof(int))) && Z.add(S.w_cnt, 64) &&
                        Z.add(S.err, 2) && Z.add(reinterpret_cast<int *>(F.skip_count), 2);
        if (!ok) return fail(c, SPH_EINVAL, "internal: clearing set overflow");
        zero_set_launch(Z, c->stream);
        ++c->launches;
    }
    // the tiles' flags reach the host through the near-field add (the last kernel), written into
    // the mapped read-back buffer, where that kernel runs; else by copies
    const bool err_mapped = c->pinned_dev && F.near_buf && nb > 0;
    fmm_work_lists(F, nb, S.w_src, S.w_cnt, S.w_leaf, S.w_cnt + 32, S.w_p2p, S.w_cnt + 56, std::max(nb, 1),
                   S.w_own, S.w_cnt + 62, c->stream, S.w_wl, S.w_cnt + 39);
    c->launches += nb > 0;
    const bool near_fork = F.near_buf && nb > 0;
    if (near_fork) {
        // fork: the near field's U-list part on its own stream from here (it needs the work
        // lists), beside the upward and far-field passes; its W-list part (M2P, which reads the
        // upward pass's equivalent densities) after the upward pass; joined before its sums are
        // added into the output
        CK(cudaEventRecord(c->near_fork, c->stream));
        CK(cudaStreamWaitEvent(c->near_stream, c->near_fork, 0));
        if (F.gtab) {
            fmm_near_table(F, const_cast<float *>(F.gtab), c->near_stream);
            ++c->launches;
        }
        if (tm) tm->mark_at(12, c->near_stream);
        fmm_p2p(F, nb, S.w_p2p, S.w_cnt + 56, std::max(nb, 1), out, c->near_stream, 0, 1, near_cap(c, S));
        ++c->launches;
        if (tm) tm->mark_at(14, c->near_stream);
    }
    if (tm) tm->mark_at(3, c->stream);
    // P2M of the leaves (and, without the tensor-core images, M2M) box by box; with them the
    // split boxes' M2M in tiles on the tensor cores (their rows zeroed by the work lists)
    const bool m2m_tc = S.tc && F.O.m2m_img != nullptr;
    for (int l = c->Lmax; l >= 2; --l) {
        // launch sizes from the number of boxes with sources (the kernels read the exact count);
        // with the tensor-core M2M the box-by-box kernel takes the leaves alone (P2M), and
        // neither kernel is launched on a level without its kind of box
        if (!m2m_tc || c->lvl_sleaf[l] > 0)
            c->launches += fmm_upward_level(F, l, c->lvl_src[l], S.w_src + c->lvl_base[l], S.w_cnt + l, m2m_tc,
                                            c->stream);
        if (m2m_tc && l < c->Lmax && c->lvl_src[l] > c->lvl_sleaf[l]) {
            fmm_m2m_tc_level(F, l, c->lvl_src[l], S.w_src + c->lvl_base[l], S.w_cnt + l, F.O.m2m_img, S.err,
                             c->stream);
            ++c->launches;
        }
    }
    if (tm) tm->mark_at(4, c->stream);
    if (near_fork) {
        CK(cudaEventRecord(c->near_up, c->stream));
        CK(cudaStreamWaitEvent(c->near_stream, c->near_up, 0));
        if (tm) tm->mark_at(15, c->near_stream);
        if (c->list_tot[2] > 0 && F.O.method == FAR_CHEB) {
            // only the leaves with W entries (at most one per W entry)
            fmm_p2p(F, nb, S.w_p2p, S.w_cnt + 56, std::max(nb, 1), out, c->near_stream, 1, 2, 16, S.w_wl,
                    S.w_cnt + 39, c->list_tot[2]);
            ++c->launches;
        }
        if (tm) tm->mark_at(13, c->near_stream);
    }
    const bool fused = S.fused;
    c->l2lp_used = fused && c->lvl_count[c->Lmax - 1] > 0;
    if (c->translate_per_box) {
        if (tm) { tm->mark_at(5, c->stream); tm->mark_at(6, c->stream); }
        for (int l = 2; l <= c->Lmax; ++l) {
            fmm_m2l_level(F, l, c->lvl_base[l], c->lvl_count[l], c->m2l_prec, c->stream);
            c->launches += c->lvl_count[l] > 0;
            if (c->list_tot[3] > 0) {
                fmm_p2l_level(F, l, c->lvl_base[l], c->lvl_count[l], c->stream);
                c->launches += c->lvl_count[l] > 0;
            }
            fmm_down_level(F, l, c->lvl_base[l], c->lvl_count[l], c->stream);
            c->launches += l >= 3 && c->lvl_count[l] > 0;
        }
    } else {
        // every M2L (all levels) and P2L first, then L2L top-down: d_child += L2L d_parent
        // needs the parent's d complete, which holds once the level above is done.
        const int nV = c->list_tot[1];
        // (the V pairs were grouped by key with the lists)
        if (tm) tm->mark_at(5, c->stream);
        const bool tiles = m2l_target_tiles(c, S);
        c->m2l_tiles_used = tiles;
        if (tiles) {
            // w_cnt[36]: number of groups, w_cnt[37]: the work counter (zeroed with the others)
            if (nV > 0) {
                fmm_m2l_tiles(F, S.ML, S.mt_groups, S.w_cnt + 36, S.w_cnt + 37, F.O.m2l_img, S.err, c->stream);
                c->launches += 2;
            }
        } else if (S.tc) {
            fmm_m2l_tc(F, S.Pd, nV, F.O.m2l_img, S.err, c->stream, c->m2l_pipe, c->m2l_loop, S.w_cnt + 38,
                       c->m2l_loop_ctas);
            c->launches += nV > 0;
        } else {
            fmm_m2l_pairs(F, S.Pd, nV, c->m2l_prec, c->stream);
            c->launches += nV > 0;
        }
        if (tm) tm->mark_at(6, c->stream);
        for (int l = 2; l <= c->Lmax; ++l)
            if (c->list_tot[3] > 0) {
                fmm_p2l_level(F, l, c->lvl_base[l], c->lvl_count[l], c->stream);
                c->launches += c->lvl_count[l] > 0;
            }
        for (int l = 3; l <= c->Lmax - (fused ? 1 : 0); ++l) {
            // 8 children per CTA where that still gives every SM a CTA; one child per CTA (8x the
            // CTAs, 1/8 of the serial work each) for the small upper levels
            const bool few = (c->lvl_count[l - 1] + 63) / 64 < 152;
            if (S.tc && c->l2l_eight && !few)
                fmm_l2l_tc8_level(F, l, c->lvl_base[l - 1], c->lvl_count[l - 1], F.O.l2l_img, S.err, c->stream);
            else if (S.tc)
                fmm_l2l_tc_level(F, l, c->lvl_base[l - 1], c->lvl_count[l - 1], F.O.l2l_img, S.err, c->stream);
            else fmm_l2l_gemm_level(F, l, c->lvl_base[l - 1], c->lvl_count[l - 1], c->stream);
            c->launches += c->lvl_count[l - 1] > 0;
        }
        if (S.tc && !err_mapped) CK(cudaMemcpyAsync(c->pinned + 48, S.err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        c->tc_used = S.tc;
    }
    if (tm) tm->mark_at(7, c->stream);
    if (F.leaf_l2p_done) {
        // default: the interpolation table on the tensor cores for leaves of edge 4 (the bulk of
        // a fine tree; measured faster there), the tensor-product (separable) form elsewhere.
        // SPH_L2P_TC=1: tables on the tensor cores at every level; SPH_L2P_SIMT=1: FP32 tables.
        const bool l2p_tc = S.tc && F.O.l2p_img != nullptr && !c->l2p_simt;
        const bool sep_all = F.l2p_sep && !c->l2p_tc_tables;
        // with the near field on its own stream and a fused deepest level, the separable L2P of
        // the coarser leaves (other leaves than the fused kernel's) joins the near stream once the
        // L2L passes are done, beside the fused kernel
        cudaStream_t sep_st = c->stream;
        if (near_fork && fused) {
            CK(cudaEventRecord(c->near_l2l, c->stream));
            CK(cudaStreamWaitEvent(c->near_stream, c->near_l2l, 0));
            sep_st = c->near_stream;
        }
        for (int l = 2; l <= c->Lmax; ++l) {
            if (fused && l == c->Lmax) {
                if (c->lvl_count[l - 1] > 0) {
                    if (tm) tm->mark_at(10, c->stream);
                    fmm_l2lp_tc_level(F, l, c->lvl_base[l - 1], c->lvl_count[l - 1], out, S.err + 1, c->stream);
                    if (tm) tm->mark_at(11, c->stream);
                    ++c->launches;
                    if (c->list_tot[1] + c->list_tot[3] > 0) {
                        // the own local terms of the leaves with V or X entries
                        fmm_l2p_own(F, l, S.w_own, S.w_cnt + 62, c->lvl_count[l], out, c->stream);
                        ++c->launches;
                    }
                }
                continue;
            }
            // only levels that hold leaves with targets (counted by the tree build) get a launch;
            // the separable form's launch is sized by that count
            if (c->lvl_count[l] == 0 || c->lvl_leaf[l] == 0) continue;
            const bool tc_here = l2p_tc && (c->l2p_tc_tables || (1 << (c->D - l)) == 4);
            if (sep_all && !tc_here) {
                fmm_l2p_sep_level(F, l, F.l2p_list + c->lvl_base[l], F.l2p_cnt + l, c->lvl_leaf[l], out, sep_st);
                ++c->launches;
            } else if (F.O.e_off[l] >= 0) {
                if (tc_here) fmm_l2p_tc_level(F, l, c->lvl_base[l], c->lvl_count[l], out, S.err + 1, c->stream);
                else fmm_l2p_gemm_level(F, l, c->lvl_base[l], c->lvl_count[l], out, c->stream);
                ++c->launches;
            } else if (F.l2p_sep) {
                fmm_l2p_sep_level(F, l, F.l2p_list + c->lvl_base[l], F.l2p_cnt + l, c->lvl_leaf[l], out, c->stream);
                ++c->launches;
            }
        }
        if (l2p_tc && !err_mapped)
            CK(cudaMemcpyAsync(c->pinned + 49, S.err + 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        c->l2p_tc_used = l2p_tc;
    }
    if (near_fork) CK(cudaEventRecord(c->near_join, c->near_stream));
    if (tm) tm->mark_at(8, c->stream);
    // the leaf kernel has work only where a leaf's L2P or near field is not taken by the kernels
    // above: with the Chebyshev far field, the separable L2P and the separate near field that is
    // the leaves of levels 0 and 1
    const bool leaf_taken = F.leaf_l2p_done && F.O.method == FAR_CHEB && F.l2p_sep && F.p2p_separate;
    if (!leaf_taken || c->lvl_leaf[0] + (c->Lmax >= 1 ? c->lvl_leaf[1] : 0) > 0) {
        fmm_leaf(F, nb, S.w_leaf, S.w_cnt + 32, out, c->stream);
        c->launches += nb > 0;
    }
    if (F.near_buf) {
        if (nb > 0) {
            CK(cudaStreamWaitEvent(c->stream, c->near_join, 0));
            fmm_near_add(F, nb, S.w_p2p, S.w_cnt + 56, std::max(nb, 1), out, c->stream,
                         err_mapped ? S.err : nullptr, err_mapped ? c->pinned_dev + 48 : nullptr);
            ++c->launches;
        }
    } else if (F.p2p_separate) {
        CK(cudaMemsetAsync(F.skip_count, 0, sizeof(unsigned long long), c->stream));
        if (F.gtab) {
            fmm_near_table(F, const_cast<float *>(F.gtab), c->stream);
            ++c->launches;
        }
        fmm_p2p(F, nb, S.w_p2p, S.w_cnt + 56, std::max(nb, 1), out, c->stream);
        c->launches += nb > 0;
    }
    if (tm) tm->mark_at(9, c->stream);
    CK(cudaGetLastError());
    return SPH_OK;
}

// Surfaces a timeout recorded by the previous eval's tensor-core tiles (read back after its sync).
int check_previous_tc(sph_ctx *c) {
    const int code = (c->tc_used ? c->pinned[48] : 0) | (c->l2p_tc_used ? c->pinned[49] : 0);
    c->tc_used = false;
    c->l2p_tc_used = false;
    if (code != 0)
        return fail(c, SPH_ETIMEOUT, "a tensor-core tile of the previous eval gave up waiting (code %d)", code);
    return SPH_OK;
}

void fill_stats(sph_ctx *c, sph_stats *stats, PhaseTimer *tm) {
    memset(stats, 0, sizeof *stats);
    stats->n_sources = c->ns;
    stats->n_targets = c->nt;
    stats->depth = c->D;
    int ml = 0;
    for (int l = 0; l < (int)c->lvl_count.size(); ++l)
        if (c->lvl_count[l] > 0) ml = l;
    stats->max_level = ml;
    stats->n_boxes = c->nboxes;
    stats->n_u = c->list_tot[0]; stats->n_v = c->list_tot[1];
    stats->n_w = c->list_tot[2]; stats->n_x = c->list_tot[3];
    if (tm) {
        stats->ms_select = tm->ms(0, 1);
        stats->ms_tree = tm->ms(1, 2);
        stats->ms_upward = tm->ms(3, 4);
        stats->ms_vpairs = tm->ms(4, 5);
        stats->ms_m2l = tm->ms(5, 6);
        stats->ms_l2l = tm->ms(6, 7);
        stats->ms_l2p = tm->ms(7, 8);
        // overlapped near field: its U-list and W-list launches themselves
        stats->ms_near = tm->rec[12] ? tm->ms(12, 14) + tm->ms(15, 13) : tm->ms(8, 9);
        stats->ms_total = tm->ms(0, 9);
        stats->ms_l2lp = tm->ms(10, 11);
    }
    stats->n_launches = c->launches;
    stats->far_method = c->far_method;
    stats->far_order = c->far_order;
    stats->leaf_size = c->leaf_eff;
    stats->near_table = c->near_table ? 1 : 0;
    stats->l2lp_fused = c->l2lp_used ? 1 : 0;
    stats->m2l_tiles = c->m2l_tiles_used ? 1 : 0;
    if (c->b_skip.p) {
        unsigned long long k = 0;
        if (cudaMemcpy(&k, c->b_skip.p, sizeof k, cudaMemcpyDeviceToHost) == cudaSuccess) stats->n_w_skipped = (int64_t)k;
        else cudaGetLastError();
    }
}

// The context's capture stream, at the device's highest stream priority: where the near field
// runs beside the far-field passes on a stream of default priority, the CTAs of the far-field
// chain (the longer one) are scheduled first whenever both wait for a slot.
cudaError_t make_capture_stream(cudaStream_t *s) {
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
        cudaGetLastError();
        greatest = 0;
    }
    return cudaStreamCreateWithPriority(s, cudaStreamNonBlocking, greatest);
}

// The passes queued as one CUDA graph: captured on the context's private capture stream (the
// caller's stream may be the legacy default stream, which cannot be captured) and launched on
// the caller's stream; the executable is updated in place while the topology repeats.
// Everything fmm_queue reads, as bytes: the pass state (zero-filled before it was built, so
// its padding compares equal), the level and list sizes, the output and the path switches.
std::vector<uint8_t> graph_signature(const sph_ctx *c, const PassState &S, const float *out) {
    std::vector<uint8_t> v;
    auto put = [&](const void *p, size_t n) {
        const uint8_t *b = static_cast<const uint8_t *>(p);
        v.insert(v.end(), b, b + n);
    };
    put(&S, sizeof S);
    put(c->lvl_count.data(), c->lvl_count.size() * sizeof(int));
    put(c->lvl_base.data(), c->lvl_base.size() * sizeof(int));
    put(c->lvl_src.data(), c->lvl_src.size() * sizeof(int));
    put(c->lvl_leaf.data(), c->lvl_leaf.size() * sizeof(int));
    put(c->lvl_sleaf.data(), c->lvl_sleaf.size() * sizeof(int));
    put(c->list_tot, sizeof c->list_tot);
    const int64_t sc[] = {c->nboxes, c->Lmax, c->D, c->m2l_prec, c->translate_per_box, c->l2l_eight, c->l2p_simt,
                          c->l2p_tc_tables, c->m2l_pipe, c->m2l_loop, c->m2l_loop_ctas, c->l2lp_fused, c->m2l_tiles, c->m2l_form,
                          (int64_t)reinterpret_cast<uintptr_t>(out)};
    put(sc, sizeof sc);
    return v;
}

int fmm_queue_graph(sph_ctx *c, PassState &S, float *out, PhaseTimer *tm) {
    if (!c->cap_stream) CK(make_capture_stream(&c->cap_stream));
    // the same passes with the same arguments as the last captured graph (and no phase events
    // to record): launch that executable again instead of capturing an identical one
    const bool timed = tm && tm->on;   // phase events are recorded inside the graph
    std::vector<uint8_t> sig;
    if (!timed) sig = graph_signature(c, S, out);
    if (!timed && c->eval_gexec && sig == c->gexec_sig) {
        c->launches += c->gexec_launches;
        CK(cudaGraphLaunch(c->eval_gexec, c->stream));
        return SPH_OK;
    }
    c->gexec_sig.clear();
    const int64_t launches0 = c->launches;
    cudaStream_t user = c->stream;
    c->stream = c->cap_stream;
    cudaError_t eb = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    int r = eb == cudaSuccess ? fmm_queue(c, S, out, tm) : SPH_ECUDA;
    cudaGraph_t g = nullptr;
    cudaError_t ee = eb == cudaSuccess ? cudaStreamEndCapture(c->cap_stream, &g) : eb;
    c->stream = user;
    if (r || ee != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return r ? r : cuda_fail(c, ee, "capture of the FMM passes");
    }
    bool updated = false;
    if (c->eval_gexec) {
        cudaGraphExecUpdateResultInfo info;
        updated = cudaGraphExecUpdate(c->eval_gexec, g, &info) == cudaSuccess;
        if (!updated) {
            cudaGetLastError();
            cudaGraphExecDestroy(c->eval_gexec);
            c->eval_gexec = nullptr;
        }
    }
    cudaError_t ei = updated ? cudaSuccess : cudaGraphInstantiate(&c->eval_gexec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
        c->eval_gexec = nullptr;
        return cuda_fail(c, ei, "cudaGraphInstantiate (FMM passes)");
    }
    c->gexec_launches = c->launches - launches0;
    c->gexec_sig = std::move(sig);
    CK(cudaGraphLaunch(c->eval_gexec, c->stream));
    return SPH_OK;
}

// tree + operators + passes for the current selection (used by eval and by the autotuner)
// the passes after the tree: operators, pass state, FMM passes (graph)
int fmm_after_tree(sph_ctx *c, float *out, PhaseTimer *tm) {
    if (tm) tm->mark_at(2, c->stream);
    int r = run_ops(c);
    if (r) return r;
    PassState S;
    memset(static_cast<void *>(&S), 0, sizeof S);   // padding included: the graph signature compares bytes
    r = fmm_prepare(c, S);
    if (r) return r;
    return c->eval_graph ? fmm_queue_graph(c, S, out, tm) : fmm_queue(c, S, out, tm);
}

int fmm_after_select(sph_ctx *c, float *out, PhaseTimer *tm) {
    int r = run_tree(c);
    if (r) return r;
    return fmm_after_tree(c, out, tm);
}

// Problem class of the autotuner's cache: grid shape, far-field form and arithmetic, and the
// selected set sizes and kernel decay length on a log2 scale (the quantities that move the
// near/far balance); snapshots of one class share the measured leaf size.
std::string tune_key(const sph_ctx *c) {
    auto lg = [](double v) { return v > 0 ? (int)std::lround(std::log2(v)) : -99; };
    char buf[256];
    snprintf(buf, sizeof buf, "%d,%d,%d|%d,%d,%d|%d,%d|%d", c->nx, c->ny, c->nz, c->far_method, c->far_order,
             c->m2l_prec, lg((double)c->ns), lg((double)c->nt), lg(2.0 * c->beta * c->h));
    return buf;
}

// Leaf size by measurement: each candidate's tree, lists and passes are timed with CUDA
// events on the context's stream (the operator build is excluded: it is cached); the
// fastest is kept per problem class (tune_key) for the life of the context.
int autotune_leaf(sph_ctx *c, float *out) {
    const std::string key = tune_key(c);
    std::map<std::string, int> &cache = c->tune_owner ? c->tune_owner->tune_cache : c->tune_cache;
    auto it = cache.find(key);
    if (it != cache.end()) {
        c->leaf_eff = it->second;
        return SPH_OK;
    }
    static const int cands[] = {32, 64, 128, 512};
    float best_ms = 1e30f;
    int best = 64;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const size_t out_bytes = sizeof(float) * (size_t)c->nx * c->ny * c->nz;
    for (int S : cands) {
        c->leaf_eff = S;
        int r = fmm_after_select(c, out, nullptr);   // builds and caches this candidate's operators
        if (r) { cudaEventDestroy(e0); cudaEventDestroy(e1); return r; }
        float tot = 0.f;
        for (int rep = 0; rep < 2; ++rep) {
            CK(cudaEventRecord(e0, c->stream));
            r = fmm_after_select(c, out, nullptr);
            if (r) { cudaEventDestroy(e0); cudaEventDestroy(e1); return r; }
            CK(cudaEventRecord(e1, c->stream));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            tot += ms;
        }
        if (tot < best_ms) { best_ms = tot; best = S; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // the trial passes accumulated into out: clear it for the real evaluation
    CK(cudaMemsetAsync(out, 0, out_bytes, c->stream));
    cache[key] = best;
    c->leaf_eff = best;
    return SPH_OK;
}

// Near-field form for this evaluation: fixed, or (SPH_NEAR_AUTO) the faster of the two,
// timed like the leaf size and cached per problem class.
int resolve_near(sph_ctx *c, float *out) {
    if (c->near_mode != SPH_NEAR_AUTO) {
        c->near_table = c->near_mode == SPH_NEAR_TABLE;
        return SPH_OK;
    }
    const std::string key = tune_key(c) + "|near|" + std::to_string(c->leaf_eff);
    std::map<std::string, int> &cache = c->tune_owner ? c->tune_owner->tune_cache : c->tune_cache;
    auto it = cache.find(key);
    if (it != cache.end()) {
        c->near_table = it->second != 0;
        return SPH_OK;
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 1e30f;
    int choice = 0;
    for (int table = 0; table < 2; ++table) {
        c->near_table = table != 0;
        int r = fmm_after_select(c, out, nullptr);
        float tot = 0.f;
        for (int rep = 0; rep < 2 && !r; ++rep) {
            CK(cudaEventRecord(e0, c->stream));
            r = fmm_after_select(c, out, nullptr);
            CK(cudaEventRecord(e1, c->stream));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            tot += ms;
        }
        if (r) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return r;
        }
        if (tot < best) {
            best = tot;
            choice = table;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(cudaMemsetAsync(out, 0, sizeof(float) * (size_t)c->nx * c->ny * c->nz, c->stream));
    cache[key] = choice;
    c->near_table = choice != 0;
    return SPH_OK;
}

// Tensor-core M2L form for this evaluation when the leaf size is autotuned (set_criteria
// leaf_size 0) and the form is left to the library: the faster of the tiles of V pairs and the
// target-stationary tiles, timed like the leaf size over the FMM passes and cached per problem
// class, leaf size and near-field form.  Otherwise the density rule of fmm_queue decides.
int fmm_after_select(sph_ctx *c, float *out, PhaseTimer *tm);
int resolve_m2l(sph_ctx *c, float *out) {
    c->m2l_form = -1;
    if (c->leaf_size != 0 || c->m2l_tiles != 2 || c->m2l_prec != SPH_M2L_BF16X3) return SPH_OK;
    const std::string key = tune_key(c) + "|m2l|" + std::to_string(c->leaf_eff) + "|" + std::to_string(c->near_table);
    std::map<std::string, int> &cache = c->tune_owner ? c->tune_owner->tune_cache : c->tune_cache;
    auto it = cache.find(key);
    if (it != cache.end()) {
        c->m2l_form = it->second;
        return SPH_OK;
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 1e30f;
    int choice = 0;
    for (int form = 0; form < 2; ++form) {
        c->m2l_form = form;
        int r = fmm_after_select(c, out, nullptr);
        float tot = 0.f;
        for (int rep = 0; rep < 2 && !r; ++rep) {
            CK(cudaEventRecord(e0, c->stream));
            r = fmm_after_select(c, out, nullptr);
            CK(cudaEventRecord(e1, c->stream));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            tot += ms;
        }
        if (r) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return r;
        }
        if (tot < best) {
            best = tot;
            choice = form;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(cudaMemsetAsync(out, 0, sizeof(float) * (size_t)c->nx * c->ny * c->nz, c->stream));
    cache[key] = choice;
    c->m2l_form = choice;
    return SPH_OK;
}


int run_fmm(sph_ctx *c, float *out, sph_stats *stats) {
    PhaseTimer tm;
    tm.start(stats != nullptr, c->stream);
    c->launches = 0;
    c->chain_zeroed = false;
    c->m2l_form = -1;                 // the density rule unless the autotuner picks the form below
    int r = check_previous_tc(c);
    if (r) return r;
    if (c->defer_sync && c->leaf_size != 0 && c->near_mode != SPH_NEAR_AUTO) {
        // fixed leaf size: selection, tree and list counts queued back to back, one sync
        c->leaf_eff = c->leaf_size;
        r = chain_zero(c);
        if (r) return r;
        r = select_queue(c, false);
        if (r) {
            c->chain_zeroed = false;
            return r;
        }
        tm.mark_at(1, c->stream);
        // the output's zero fill (an HBM-bound pass) runs on the side stream beside the tree build
        // and list counts (latency-bound passes); the context's stream takes it back before the sync
        const bool zero_side = c->near_overlap && (int64_t)c->nx * c->ny * c->nz > 0;
        if (zero_side) {
            if (!c->near_stream) CK(cudaStreamCreateWithFlags(&c->near_stream, cudaStreamNonBlocking));
            if (!c->zero_fork) CK(cudaEventCreateWithFlags(&c->zero_fork, cudaEventDisableTiming));
            if (!c->zero_done) CK(cudaEventCreateWithFlags(&c->zero_done, cudaEventDisableTiming));
            CK(cudaEventRecord(c->zero_fork, c->stream));
            CK(cudaStreamWaitEvent(c->near_stream, c->zero_fork, 0));
            CK(cudaMemsetAsync(out, 0, sizeof(float) * (size_t)c->nx * c->ny * c->nz, c->near_stream));
            CK(cudaEventRecord(c->zero_done, c->near_stream));
        } else if ((int64_t)c->nx * c->ny * c->nz > 0) {
            CK(cudaMemsetAsync(out, 0, sizeof(float) * (size_t)c->nx * c->ny * c->nz, c->stream));
        }
        c->leaf_eff = c->leaf_size;
        r = resolve_near(c, out);
        if (!r) r = tree_queue(c);
        if (!r) r = lists_count_queue(c);
        c->chain_zeroed = false;   // consumed (or abandoned on an error) by the three above
        if (zero_side) CK(cudaStreamWaitEvent(c->stream, c->zero_done, 0));
        if (r) return r;
        CK(cudaStreamSynchronize(c->stream));
        r = select_read(c);
        if (r) return r;
        if (c->nt == 0) {
            c->have_tree = false;
            if (stats) {
                memset(stats, 0, sizeof *stats);
                stats->n_sources = c->ns;
                stats->depth = c->D;
                stats->n_launches = c->launches;
            }
            return SPH_OK;
        }
        r = tree_levels_read(c);
        if (!r) r = lists_fill(c);
        if (!r) r = fmm_after_tree(c, out, &tm);
        if (r) return r;
        if (stats) {
            CK(cudaStreamSynchronize(c->stream));
            if ((c->tc_used && c->pinned[48] != 0) || (c->l2p_tc_used && c->pinned[49] != 0))
                return fail(c, SPH_ETIMEOUT, "a tensor-core tile gave up waiting (code %d)",
                            c->pinned[48] | c->pinned[49]);
            fill_stats(c, stats, &tm);
        }
        return SPH_OK;
    }
    r = run_select(c);
    if (r) return r;
    tm.mark_at(1, c->stream);
    if ((int64_t)c->nx * c->ny * c->nz > 0) {
        CK(cudaMemsetAsync(out, 0, sizeof(float) * (size_t)c->nx * c->ny * c->nz, c->stream));
    }
    if (c->nt == 0) {
        c->have_tree = false;
        if (stats) {
            memset(stats, 0, sizeof *stats);
            stats->n_sources = c->ns;
            stats->depth = c->D;
            stats->n_launches = c->launches;
        }
        return SPH_OK;
    }
    if (c->leaf_size == 0) {
        r = autotune_leaf(c, out);
        if (r) return r;
    } else {
        c->leaf_eff = c->leaf_size;
    }
    r = resolve_near(c, out);
    if (r) return r;
    r = resolve_m2l(c, out);
    if (r) return r;
    r = fmm_after_select(c, out, &tm);
    if (r) return r;
    if (stats) {
        CK(cudaStreamSynchronize(c->stream));
        if ((c->tc_used && c->pinned[48] != 0) || (c->l2p_tc_used && c->pinned[49] != 0))
            return fail(c, SPH_ETIMEOUT, "a tensor-core tile gave up waiting (code %d)",
                        c->pinned[48] | c->pinned[49]);
        fill_stats(c, stats, &tm);
    }
    return SPH_OK;
}

// The context's read-back buffer: 128 ints of pinned host memory, mapped into the device's
// address space so that the last kernel before a host sync can write what the host reads
// there (no copy operations in the stream); without a device address the read-backs are copies.
bool alloc_pinned(sph_ctx *c) {
    if (cudaHostAlloc(reinterpret_cast<void **>(&c->pinned), 128 * sizeof(int), cudaHostAllocMapped) != cudaSuccess) {
        cudaGetLastError();
        c->pinned = nullptr;
        return false;
    }
    void *d = nullptr;
    if (cudaHostGetDevicePointer(&d, c->pinned, 0) == cudaSuccess) {
        c->pinned_dev = static_cast<int *>(d);
    } else {
        cudaGetLastError();
        c->pinned_dev = nullptr;
    }
    return true;
}

// A sub-context of `parent`: its own stream (batch slots) or the parent's (shared_stream).
sph_ctx *make_sub(sph_ctx *parent, bool shared_stream = false) {
    sph_ctx *c = new (std::nothrow) sph_ctx();
    if (!c) return nullptr;
    c->device = parent->device;
    c->tune_owner = parent;
    if (shared_stream) {
        c->stream = parent->stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete c;
            return nullptr;
        }
        c->own_stream = true;
    }
    if (!alloc_pinned(c)) {
        cudaGetLastError();
        if (c->own_stream) cudaStreamDestroy(c->stream);
        delete c;
        return nullptr;
    }
    return c;
}

int configure_sub(sph_ctx *sub, const sph_ctx *parent, const sph_problem &p) {
    if (p.nx < 1 || p.ny < 1 || p.nz < 1 || p.nx > 1024 || p.ny > 1024 || p.nz > 1024) return SPH_EINVAL;
    if (!(p.h_cm > 0) || !(p.pO2_torr > 0) || !(p.chi_min > 0) || !(p.chi_max > p.chi_min)) return SPH_EINVAL;
    if (!p.q_dev || !p.s_dev || !(p.source_scale > 0)) return SPH_EINVAL;
    if (p.emag_dev && p.mask_dev) return SPH_EINVAL;
    if (!(p.i_frac >= 0 && p.i_frac <= 1) || !(p.e_frac >= 0 && p.e_frac <= 1)) return SPH_EINVAL;
    sub->nx = p.nx; sub->ny = p.ny; sub->nz = p.nz;
    sub->D = depth_of(p.nx, p.ny, p.nz);
    sub->h = p.h_cm; sub->pO2 = p.pO2_torr; sub->chi_min = p.chi_min; sub->chi_max = p.chi_max;
    sub->alpha = p.chi_min * p.pO2_torr;
    sub->beta = p.chi_max * p.pO2_torr;
    sub->grid_set = true;
    sub->q = p.q_dev; sub->source_scale = p.source_scale; sub->src_set = true;
    sub->emag = p.emag_dev; sub->mask = p.mask_dev; sub->trg_set = true;
    sub->i_frac = p.i_frac; sub->e_frac = p.e_frac; sub->e_app = p.e_applied;
    sub->self_mode = parent->self_mode; sub->leaf_size = parent->leaf_size; sub->m2l_prec = parent->m2l_prec;
    sub->crit_set = true;
    sub->far_method = parent->far_method; sub->far_order = parent->far_order;
    sub->radii = parent->radii; sub->pinv_eps = parent->pinv_eps;
    sub->translate_per_box = parent->translate_per_box; sub->l2l_eight = parent->l2l_eight;
    sub->select_two_pass = parent->select_two_pass;
    sub->select_lookback = parent->select_lookback;
    sub->p2p_in_leaf = parent->p2p_in_leaf;
    sub->l2p_simt = parent->l2p_simt;
    sub->l2p_tc_tables = parent->l2p_tc_tables;
    sub->m2l_pipe = parent->m2l_pipe;
    sub->m2l_loop = parent->m2l_loop;
    sub->m2l_loop_ctas = parent->m2l_loop_ctas;
    sub->near_overlap = parent->near_overlap;
    sub->near_per_sm = parent->near_per_sm;
    sub->l2lp_fused = parent->l2lp_fused;
    sub->m2l_tiles = parent->m2l_tiles;
    sub->defer_sync = parent->defer_sync;
    sub->near_mode = parent->near_mode;
    sub->r_s = parent->r_s;
    sub->launches = 0;
    return SPH_OK;
}

int sub_fail(sph_ctx *c, sph_ctx *sub, int code, int i) {
    return fail(c, code, "snapshot %d: %s", i, sub->err.c_str());
}

cudaEvent_t batch_event(sph_ctx *c, size_t k) {
    while (c->events.size() <= k) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
        c->events.push_back(e);
    }
    return c->events[k];
}

int run_batch(sph_ctx *c, int n, const sph_problem *probs, sph_stats *stats) {
    while ((int)c->subs.size() < n) {
        sph_ctx *sub = make_sub(c);
        if (!sub) return fail(c, SPH_ENOMEM, "cannot create the context of batch slot %d", (int)c->subs.size());
        c->subs.push_back(sub);
    }
    for (int i = 0; i < n; ++i) {
        int r = configure_sub(c->subs[i], c, probs[i]);
        if (r) return fail(c, r, "snapshot %d: invalid problem", i);
    }
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (stats) {
        CK(cudaEventCreate(&t0));
        CK(cudaEventCreate(&t1));
        CK(cudaEventRecord(t0, c->stream));
    }
    // fork: the snapshots' streams wait for the inputs queued on the context's stream
    cudaEvent_t fork = batch_event(c, 0);
    if (!fork) return fail(c, SPH_ECUDA, "event creation failed");
    CK(cudaEventRecord(fork, c->stream));
    for (int i = 0; i < n; ++i) CK(cudaStreamWaitEvent(c->subs[i]->stream, fork, 0));
    // phase 1: selection of every snapshot, one synchronisation
    for (int i = 0; i < n; ++i) {
        sph_ctx *sub = c->subs[i];
        int r = check_previous_tc(sub);
        if (!r) r = select_queue(sub);
        if (r) return sub_fail(c, sub, r, i);
        size_t cells = (size_t)sub->nx * sub->ny * sub->nz;
        CK(cudaMemsetAsync(probs[i].s_dev, 0, cells * sizeof(float), sub->stream));
    }
    for (int i = 0; i < n; ++i) {
        sph_ctx *sub = c->subs[i];
        CK(cudaStreamSynchronize(sub->stream));
        int r = select_read(sub);
        if (r) return sub_fail(c, sub, r, i);
    }
    // leaf sizes (autotuned shapes run their candidates here, once per shape)
    std::vector<int> live;
    for (int i = 0; i < n; ++i) {
        sph_ctx *sub = c->subs[i];
        if (sub->nt == 0) { sub->have_tree = false; continue; }
        live.push_back(i);
        if (sub->leaf_size == 0) {
            int r = autotune_leaf(sub, probs[i].s_dev);
            if (r) return sub_fail(c, sub, r, i);
        } else {
            sub->leaf_eff = sub->leaf_size;
        }
        {
            int r = resolve_near(sub, probs[i].s_dev);
            if (!r) r = resolve_m2l(sub, probs[i].s_dev);
            if (r) return sub_fail(c, sub, r, i);
        }
    }
    // phases 2-3: trees and list counts, then list fills -- one more synchronisation
    for (int i : live) {
        int r = tree_queue(c->subs[i]);
        if (!r) r = lists_count_queue(c->subs[i]);
        if (r) return sub_fail(c, c->subs[i], r, i);
    }
    for (int i : live) {
        CK(cudaStreamSynchronize(c->subs[i]->stream));
        int r = tree_levels_read(c->subs[i]);
        if (!r) r = lists_fill(c->subs[i]);
        if (!r) r = run_ops(c->subs[i]);
        if (r) return sub_fail(c, c->subs[i], r, i);
    }
    std::vector<PassState> ps(n);
    for (int i : live) {
        int r = fmm_prepare(c->subs[i], ps[i]);
        if (r) return sub_fail(c, c->subs[i], r, i);
    }
    // phase 4: the FMM passes of every snapshot, concurrently, as one graph
    bool graph = c->batch_graph && !live.empty();
    if (graph) {
        if (!c->cap_stream) CK(make_capture_stream(&c->cap_stream));
        CK(cudaStreamSynchronize(c->cap_stream));
        // the capture stream starts after the context's stream and every snapshot's pending work
        cudaEvent_t pre = batch_event(c, 1);
        CK(cudaEventRecord(pre, c->stream));
        CK(cudaStreamWaitEvent(c->cap_stream, pre, 0));
        for (size_t k = 0; k < live.size(); ++k) {
            cudaEvent_t e = batch_event(c, 2 + k);
            CK(cudaEventRecord(e, c->subs[live[k]]->stream));
            CK(cudaStreamWaitEvent(c->cap_stream, e, 0));
        }
        CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
        cudaEvent_t cf = batch_event(c, 2 + live.size());
        int r = SPH_OK;
        if (cudaEventRecord(cf, c->cap_stream) != cudaSuccess) r = SPH_ECUDA;
        for (size_t k = 0; k < live.size() && !r; ++k) {
            sph_ctx *sub = c->subs[live[k]];
            if (cudaStreamWaitEvent(sub->stream, cf, 0) != cudaSuccess) { r = SPH_ECUDA; break; }
            r = fmm_queue(sub, ps[live[k]], probs[live[k]].s_dev, nullptr);
            cudaEvent_t j = batch_event(c, 3 + live.size() + k);
            if (!r && (cudaEventRecord(j, sub->stream) != cudaSuccess ||
                       cudaStreamWaitEvent(c->cap_stream, j, 0) != cudaSuccess))
                r = SPH_ECUDA;
        }
        cudaGraph_t g = nullptr;
        cudaError_t ee = cudaStreamEndCapture(c->cap_stream, &g);
        if (r || ee != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return fail(c, SPH_ECUDA, "batch graph capture failed");
        }
        // same topology as the previous batch (the usual case): update the executable in place
        bool updated = false;
        if (c->gexec) {
            cudaGraphExecUpdateResultInfo info;
            updated = cudaGraphExecUpdate(c->gexec, g, &info) == cudaSuccess;
            if (!updated) {
                cudaGetLastError();
                cudaGraphExecDestroy(c->gexec);
                c->gexec = nullptr;
            }
        }
        cudaError_t ei = updated ? cudaSuccess : cudaGraphInstantiate(&c->gexec, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            c->gexec = nullptr;
            return cuda_fail(c, ei, "cudaGraphInstantiate");
        }
        CK(cudaGraphLaunch(c->gexec, c->cap_stream));
        cudaEvent_t done = batch_event(c, 3 + 2 * live.size());
        CK(cudaEventRecord(done, c->cap_stream));
        CK(cudaStreamWaitEvent(c->stream, done, 0));
    } else {
        for (int i : live) {
            int r = fmm_queue(c->subs[i], ps[i], probs[i].s_dev, nullptr);
            if (r) return sub_fail(c, c->subs[i], r, i);
        }
    }
    // join every snapshot stream back into the context's stream
    for (int i = 0; i < n; ++i) {
        cudaEvent_t e = batch_event(c, 4 + 2 * live.size() + i);
        CK(cudaEventRecord(e, c->subs[i]->stream));
        CK(cudaStreamWaitEvent(c->stream, e, 0));
    }
    if (stats) {
        CK(cudaEventRecord(t1, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        memset(stats, 0, sizeof *stats);
        for (int i = 0; i < n; ++i) {
            sph_ctx *sub = c->subs[i];
            if ((sub->tc_used && sub->pinned[48] != 0) || (sub->l2p_tc_used && sub->pinned[49] != 0))
                return fail(c, SPH_ETIMEOUT, "snapshot %d: a tensor-core tile gave up waiting", i);
            stats->n_sources += sub->ns;
            stats->n_targets += sub->nt;
            stats->n_boxes += sub->nboxes;
            stats->n_u += sub->list_tot[0]; stats->n_v += sub->list_tot[1];
            stats->n_w += sub->list_tot[2]; stats->n_x += sub->list_tot[3];
            stats->n_launches += sub->launches;
            stats->depth = std::max(stats->depth, sub->D);
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t0, t1);
        stats->ms_total = ms;
        stats->far_method = c->far_method;
        stats->far_order = c->far_order;
        stats->leaf_size = c->leaf_size;
        cudaEventDestroy(t0);
        cudaEventDestroy(t1);
    }
    return SPH_OK;
}

int run_surrogate(sph_ctx *c, sph_nn *net, int factor, double tol, int samples, uint64_t seed, int use_net,
                  float *out, sph_surrogate_stats *st) {
    const int D = nn::net_edge(net);
    int lgD = 0;
    while ((1 << lgD) < D) ++lgD;
    if (D < nn::JUDGE_BLOCK || (1 << lgD) != D) return fail(c, SPH_EINVAL, "network edge must be a power of two >= 8");
    if (c->nx != c->ny || c->nx != c->nz || c->nx != factor * D)
        return fail(c, SPH_EINVAL, "grid must be cubic with edge factor * %d", D);
    const int n = c->nx;
    const size_t nf = (size_t)n * n * n, nc = (size_t)D * D * D;
    const int nbl = (D / nn::JUDGE_BLOCK) * (D / nn::JUDGE_BLOCK) * (D / nn::JUDGE_BLOCK);
    ENS(c->s_qc, nc * sizeof(float));
    ENS(c->s_Sc, nc * sizeof(float));
    ENS(c->s_y, 2 * nc * sizeof(float));
    ENS(c->s_Sp, nc * sizeof(float));
    ENS(c->s_x, 16 * nc * sizeof(uint16_t));
    ENS(c->s_Sf, nf * sizeof(float));
    ENS(c->s_mask, nf);
    ENS(c->s_svox, (size_t)nbl * samples * sizeof(int));
    ENS(c->s_err, nbl * sizeof(float));
    ENS(c->s_pe, nbl * sizeof(float));
    ENS(c->s_flags, nbl * sizeof(int));
    ENS(c->s_counts, 4 * sizeof(unsigned));
    if (!c->sur_coarse) c->sur_coarse = make_sub(c, true);
    if (!c->sur_fine) c->sur_fine = make_sub(c, true);
    if (!c->sur_coarse || !c->sur_fine) return fail(c, SPH_ENOMEM, "cannot create the surrogate's sub-contexts");
    cudaStream_t s = c->stream;
    cudaEvent_t ev[5];
    for (auto &e : ev) CK(cudaEventCreate(&e));
    struct EvGuard {
        cudaEvent_t *e;
        ~EvGuard() {
            for (int i = 0; i < 5; ++i) cudaEventDestroy(e[i]);
        }
    } guard{ev};
    CK(cudaEventRecord(ev[0], s));
    // 1. coarse FMM on the pooled source
    nn::pool_avg_f32(c->q, n, factor, P<float>(c->s_qc), s);
    sph_problem pc;
    pc.nx = pc.ny = pc.nz = D;
    pc.h_cm = c->h * factor; pc.pO2_torr = c->pO2; pc.chi_min = c->chi_min; pc.chi_max = c->chi_max;
    pc.q_dev = P<float>(c->s_qc); pc.source_scale = c->source_scale;
    pc.emag_dev = nullptr; pc.mask_dev = nullptr;
    pc.i_frac = c->i_frac; pc.e_frac = 0; pc.e_applied = 0;
    pc.s_dev = P<float>(c->s_Sc);
    int r = configure_sub(c->sur_coarse, c, pc);
    if (!r) r = run_fmm(c->sur_coarse, P<float>(c->s_Sc), nullptr);
    if (r) return fail(c, r, "coarse FMM: %s", c->sur_coarse->err.c_str());
    CK(cudaEventRecord(ev[1], s));
    // 2. network
    if (use_net) {
        cudaStream_t ns = nn::net_stream(net);
        if (ns != s) {
            CK(cudaStreamWaitEvent(ns, ev[1], 0));
        }
        r = sph_nn_make_inputs(net, n, factor, c->q, c->emag, P<float>(c->s_Sc), P<uint16_t>(c->s_x));
        if (!r) r = sph_nn_forward(net, 1, P<uint16_t>(c->s_x), P<float>(c->s_y));
        if (r) return fail(c, r, "network: %s", nn::net_error(net));
        if (ns != s) {
            CK(cudaEventRecord(ev[2], ns));
            CK(cudaStreamWaitEvent(s, ev[2], 0));
        }
        nn::block_pred_err(P<float>(c->s_y), lgD, P<float>(c->s_pe), s);
    }
    nn::apply_residual(P<float>(c->s_Sc), P<float>(c->s_y), use_net, P<float>(c->s_Sp), nc, s);
    CK(cudaEventRecord(ev[2], s));
    // 3. judge: the FMM at the sampled voxels' fine cells
    nn::judge_mask(lgD, factor, seed, samples, P<uint8_t>(c->s_mask), P<int>(c->s_svox), s);
    sph_problem pf = pc;
    pf.nx = pf.ny = pf.nz = n;
    pf.h_cm = c->h;
    pf.q_dev = c->q;
    pf.mask_dev = P<uint8_t>(c->s_mask);
    pf.s_dev = P<float>(c->s_Sf);
    r = configure_sub(c->sur_fine, c, pf);
    if (!r) r = run_fmm(c->sur_fine, P<float>(c->s_Sf), nullptr);
    if (r) return fail(c, r, "judge FMM: %s", c->sur_fine->err.c_str());
    const int64_t judge_nt = c->sur_fine->nt;
    nn::judge_err(P<float>(c->s_Sf), P<float>(c->s_Sp), P<int>(c->s_svox), lgD, factor, samples,
                  P<float>(c->s_err), s);
    nn::fallback_flags(P<float>(c->s_err), P<float>(c->s_pe), use_net, (float)tol, nbl, P<int>(c->s_flags),
                       P<unsigned>(c->s_counts), s);
    CK(cudaEventRecord(ev[3], s));
    // 4. fallback: every fine cell of the failing blocks
    nn::fallback_mask(P<int>(c->s_flags), lgD, factor, P<uint8_t>(c->s_mask), s);
    r = run_fmm(c->sur_fine, P<float>(c->s_Sf), nullptr);
    if (r) return fail(c, r, "fallback FMM: %s", c->sur_fine->err.c_str());
    const int64_t fb_nt = c->sur_fine->nt;
    nn::combine(P<float>(c->s_Sp), P<float>(c->s_Sf), P<int>(c->s_flags), lgD, factor, out, s);
    CK(cudaEventRecord(ev[4], s));
    unsigned cnt[4];
    CK(cudaMemcpyAsync(cnt, c->s_counts.p, sizeof cnt, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
    if (st) {
        memset(st, 0, sizeof *st);
        st->n_blocks = nbl;
        st->n_fallback = (int)cnt[0];
        st->n_judged_fail = (int)cnt[1];
        st->n_predicted_fail = (int)cnt[2];
        float mx;
        memcpy(&mx, &cnt[3], sizeof mx);
        st->judged_max_err = mx;
        st->n_judge_targets = judge_nt;
        st->n_fallback_targets = fb_nt;
        cudaEventElapsedTime(&st->ms_coarse, ev[0], ev[1]);
        cudaEventElapsedTime(&st->ms_net, ev[1], ev[2]);
        cudaEventElapsedTime(&st->ms_judge, ev[2], ev[3]);
        cudaEventElapsedTime(&st->ms_fallback, ev[3], ev[4]);
        cudaEventElapsedTime(&st->ms_total, ev[0], ev[4]);
    }
    return SPH_OK;
}

}  // namespace

extern "C" {

int eval_sph_surrogate(sph_ctx *c, sph_nn *net, int factor, double tol, int samples_per_block, uint64_t seed,
                       int use_net, float *out, sph_surrogate_stats *stats) {
    if (!c) return SPH_EINVAL;
    if (c->poisoned) return fail(c, SPH_ECUDA, "context poisoned by an earlier CUDA error");
    if (!net || !out || factor < 1 || !(tol > 0) || samples_per_block < 1 || samples_per_block > 64)
        return fail(c, SPH_EINVAL, "bad surrogate arguments");
    if (!c->grid_set || !c->src_set || !c->crit_set) return fail(c, SPH_ESTATE, "grid, sources and criteria must be set");
    CK(cudaSetDevice(c->device));
    return run_surrogate(c, net, factor, tol, samples_per_block, seed, use_net ? 1 : 0, out, stats);
}


int sph_scan_i32(int device, void *cuda_stream, int64_t n, const int32_t *in_dev, int32_t *out_dev,
                 int32_t *total_dev) {
    if (n < 0 || n > INT32_MAX || !total_dev || (n > 0 && (!in_dev || !out_dev))) return SPH_EINVAL;
    if (n > 0 && in_dev == out_dev) return SPH_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return SPH_ECUDA;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    const size_t nt = scan_tmp_ints((int)n);
    int *tmp = nullptr;
    if (cudaMalloc(&tmp, (nt + 2) * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return SPH_ENOMEM;
    }
    int *err = tmp + nt;
    int herr = 0;
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        scan_exclusive(in_dev, out_dev, (int)n, total_dev, tmp, st, err,
                       env_limit("SPH_WAIT_LIMIT_SCAN", SCAN_WAIT_LIMIT));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(tmp);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SPH_ECUDA;
    }
    return herr ? SPH_ETIMEOUT : SPH_OK;
}

const char *sph_version(void) { return "libsph 0.1 (sm_103a)"; }

int sph_create(sph_ctx **out, int device, void *cuda_stream) {
    if (!out) return SPH_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return SPH_EINVAL;
    }
    sph_ctx *c = new (std::nothrow) sph_ctx();
    if (!c) return SPH_ENOMEM;
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    if (cudaSetDevice(device) != cudaSuccess || !alloc_pinned(c)) {
        cudaGetLastError();
        delete c;
        return SPH_ECUDA;
    }
    if (const char *e = getenv("SPH_PINV_EPS")) c->pinv_eps = atof(e);
    if (const char *e = getenv("SPH_TRANSLATE_PER_BOX")) c->translate_per_box = atoi(e) != 0;
    if (const char *e = getenv("SPH_L2L_ONE_CHILD")) c->l2l_eight = atoi(e) == 0;
    if (const char *e = getenv("SPH_SELECT_TWO_PASS")) c->select_two_pass = atoi(e) != 0;
    if (const char *e = getenv("SPH_SELECT_LOOKBACK")) c->select_lookback = atoi(e) != 0;
    if (const char *e = getenv("SPH_P2P_IN_LEAF")) c->p2p_in_leaf = atoi(e) != 0;
    if (const char *e = getenv("SPH_L2P_SIMT")) c->l2p_simt = atoi(e) != 0;
    if (const char *e = getenv("SPH_L2P_TC")) c->l2p_tc_tables = atoi(e) != 0;
    if (const char *e = getenv("SPH_M2L_PIPE")) c->m2l_pipe = atoi(e) != 0;
    if (const char *e = getenv("SPH_M2L_LOOP")) c->m2l_loop = atoi(e) != 0;
    if (const char *e = getenv("SPH_M2L_LOOP_CTAS")) c->m2l_loop_ctas = std::max(0, atoi(e));
    if (const char *e = getenv("SPH_NEAR_OVERLAP")) c->near_overlap = atoi(e) != 0;
    if (const char *e = getenv("SPH_NEAR_PER_SM")) c->near_per_sm = std::max(1, atoi(e));
    if (const char *e = getenv("SPH_L2LP_FUSED")) c->l2lp_fused = atoi(e) != 0;
    if (const char *e = getenv("SPH_M2L_TILES")) c->m2l_tiles = atoi(e);
    c->select_wait = env_limit("SPH_WAIT_LIMIT_SELECT", SELECT_WAIT_LIMIT);
    if (const char *e = getenv("SPH_FAULT")) {
        if (strncmp(e, "alloc", 5) == 0) c->fault_alloc = e[5] == ':' ? std::max(1, atoi(e + 6)) : 1;
    }
    if (const char *e = getenv("SPH_DEFER_SYNC")) c->defer_sync = atoi(e) != 0;
    if (const char *e = getenv("SPH_BATCH_GRAPH")) c->batch_graph = atoi(e) != 0;
    if (const char *e = getenv("SPH_EVAL_GRAPH")) c->eval_graph = atoi(e) != 0;
    if (const char *e = getenv("SPH_FAR")) {
        int m, o;
        if (sscanf(e, "%d,%d", &m, &o) == 2) { c->far_method = m; c->far_order = o; }
    }
    if (const char *e = getenv("SPH_RADII")) {
        Radii r;
        if (sscanf(e, "%lf,%lf,%lf,%lf", &r.ue, &r.uc, &r.dc, &r.de) == 4) c->radii = r;
    }
    *out = c;
    return SPH_OK;
}

void sph_destroy(sph_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->cap_stream) cudaStreamSynchronize(c->cap_stream);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->eval_gexec) cudaGraphExecDestroy(c->eval_gexec);
    for (cudaEvent_t e : c->events) cudaEventDestroy(e);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->near_stream) {
        cudaStreamSynchronize(c->near_stream);
        cudaStreamDestroy(c->near_stream);
    }
    if (c->near_fork) cudaEventDestroy(c->near_fork);
    if (c->near_join) cudaEventDestroy(c->near_join);
    if (c->near_up) cudaEventDestroy(c->near_up);
    if (c->near_l2l) cudaEventDestroy(c->near_l2l);
    if (c->zero_fork) cudaEventDestroy(c->zero_fork);
    if (c->zero_done) cudaEventDestroy(c->zero_done);
    for (sph_ctx *sub : c->subs) sph_destroy(sub);
    c->subs.clear();
    if (c->sur_coarse) sph_destroy(c->sur_coarse);
    if (c->sur_fine) sph_destroy(c->sur_fine);
    DevBuf *all[] = {&c->b_maxes, &c->b_bstat, &c->b_cnt, &c->b_off, &c->b_tot, &c->b_skey, &c->b_spc, &c->b_sq, &c->b_tkey,
                     &c->b_tpc, &c->b_boxat, &c->b_flag, &c->b_pos, &c->b_rng, &c->b_scan, &c->b_lvl,
                     &c->b_level, &c->b_key, &c->b_sb, &c->b_se, &c->b_tb, &c->b_te, &c->b_parent, &c->b_leaf,
                     &c->b_lcnt, &c->b_loff, &c->b_usrc, &c->b_vsrc, &c->b_vocs, &c->b_vtrg, &c->b_wsrc, &c->b_xsrc, &c->b_pkeys, &c->b_ppairs, &c->b_heavy,
                     &c->b_ueq, &c->b_dchk, &c->o_work, &c->o_etab, &c->o_m2m, &c->o_l2l,
                     &c->o_m2l, &c->o_m2lbf, &c->o_l2lbf, &c->o_m2mbf, &c->b_err, &c->b_work, &c->b_mtg, &c->b_nearbuf, &c->o_slot, &c->o_surf, &c->o_cheb, &c->o_self, &c->h_q, &c->h_e, &c->h_m,
                     &c->h_s, &c->b_tmask, &c->b_near, &c->b_gtab, &c->b_skip, &c->o_l2pimg, &c->s_qc, &c->s_Sc, &c->s_y, &c->s_Sp, &c->s_x, &c->s_Sf,
                     &c->s_mask, &c->s_svox, &c->s_err, &c->s_pe, &c->s_flags, &c->s_counts};
    for (DevBuf *b : all)
        if (b->p) cudaFree(b->p);
    if (c->pinned) cudaFreeHost(c->pinned);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char *sph_last_error(const sph_ctx *c) { return c ? c->err.c_str() : "null context"; }

int set_grid(sph_ctx *c, int nx, int ny, int nz, const double origin_cm[3], double h_cm, double pO2_torr,
             double chi_min, double chi_max) {
    if (!c) return SPH_EINVAL;
    if (nx < 1 || ny < 1 || nz < 1 || nx > 1024 || ny > 1024 || nz > 1024)
        return fail(c, SPH_EINVAL, "grid dimensions must be in [1, 1024], got %d x %d x %d", nx, ny, nz);
    if (!(h_cm > 0) || !std::isfinite(h_cm)) return fail(c, SPH_EINVAL, "h must be positive and finite");
    if (!(pO2_torr > 0) || !std::isfinite(pO2_torr)) return fail(c, SPH_EINVAL, "pO2 must be positive");
    if (!(chi_min > 0) || !(chi_max > chi_min) || !std::isfinite(chi_max))
        return fail(c, SPH_EINVAL, "need 0 < chi_min < chi_max");
    c->nx = nx; c->ny = ny; c->nz = nz;
    c->D = depth_of(nx, ny, nz);
    for (int i = 0; i < 3; ++i) c->origin[i] = origin_cm ? origin_cm[i] : 0.0;
    c->h = h_cm; c->pO2 = pO2_torr; c->chi_min = chi_min; c->chi_max = chi_max;
    c->alpha = chi_min * pO2_torr;
    c->beta = chi_max * pO2_torr;
    c->grid_set = true;
    c->have_tree = false;
    return SPH_OK;
}

int set_sources(sph_ctx *c, const float *q_dev, double source_scale) {
    if (!c) return SPH_EINVAL;
    if (!q_dev) return fail(c, SPH_EINVAL, "q_dev is NULL");
    if (!(source_scale > 0) || !std::isfinite(source_scale))
        return fail(c, SPH_EINVAL, "source_scale must be positive and finite");
    c->q = q_dev;
    c->source_scale = source_scale;
    c->src_set = true;
    return SPH_OK;
}

int set_targets(sph_ctx *c, const float *emag_dev, const uint8_t *mask_dev) {
    if (!c) return SPH_EINVAL;
    if (emag_dev && mask_dev) return fail(c, SPH_EINVAL, "give |E| or a mask, not both");
    c->emag = emag_dev;
    c->mask = mask_dev;
    c->trg_set = true;
    return SPH_OK;
}

int sph_set_far_field(sph_ctx *c, int method, int order) {
    if (!c) return SPH_EINVAL;
    if (method == SPH_FAR_CHEBYSHEV) {
        if (order < 2 || order > 8) return fail(c, SPH_EINVAL, "Chebyshev order must be in [2, 8]");
        c->far_method = FAR_CHEB;
    } else if (method == SPH_FAR_SURFACE) {
        if (order < 3 || order > 10) return fail(c, SPH_EINVAL, "surface points per edge must be in [3, 10]");
        c->far_method = FAR_SURFACE;
    } else {
        return fail(c, SPH_EINVAL, "unknown far-field method %d", method);
    }
    c->far_order = order;
    return SPH_OK;
}

int set_criteria(sph_ctx *c, double i_frac, double e_frac, double e_applied, int self_mode, int leaf_size,
                 int m2l_precision) {
    if (!c) return SPH_EINVAL;
    if (!(i_frac >= 0 && i_frac <= 1)) return fail(c, SPH_EINVAL, "i_frac must be in [0, 1]");
    if (!(e_frac >= 0 && e_frac <= 1)) return fail(c, SPH_EINVAL, "e_frac must be in [0, 1]");
    if (!std::isfinite(e_applied)) return fail(c, SPH_EINVAL, "e_applied must be finite");
    if (self_mode != 0 && self_mode != 1) return fail(c, SPH_EINVAL, "self_mode must be 0 or 1");
    if (leaf_size < 0 || leaf_size > 4096) return fail(c, SPH_EINVAL, "leaf_size must be in [0, 4096] (0: autotune)");
    if (m2l_precision != SPH_M2L_F32 && m2l_precision != SPH_M2L_BF16X3)
        return fail(c, SPH_EINVAL, "unknown m2l_precision %d", m2l_precision);
    c->i_frac = i_frac; c->e_frac = e_frac; c->e_app = e_applied;
    c->self_mode = self_mode; c->leaf_size = leaf_size; c->m2l_prec = m2l_precision;
    c->crit_set = true;
    return SPH_OK;
}

int eval_sph(sph_ctx *c, float *s_dev, sph_stats *stats) {
    int r = check_ready(c);
    if (r) return r;
    if (!s_dev) return fail(c, SPH_EINVAL, "s_dev is NULL");
    return run_fmm(c, s_dev, stats);
}

int sph_set_skip_ratio(sph_ctx *c, double r_s) {
    if (!c) return SPH_EINVAL;
    if (!(r_s >= 0.0 && r_s < 1.0)) return fail(c, SPH_EINVAL, "r_s must be in [0, 1)");
    c->r_s = r_s;
    return SPH_OK;
}

int sph_set_near_field(sph_ctx *c, int mode) {
    if (!c) return SPH_EINVAL;
    if (mode != SPH_NEAR_EXP && mode != SPH_NEAR_TABLE && mode != SPH_NEAR_AUTO)
        return fail(c, SPH_EINVAL, "near-field mode must be SPH_NEAR_EXP, SPH_NEAR_TABLE or SPH_NEAR_AUTO");
    c->near_mode = mode;
    return SPH_OK;
}

int eval_sph_batch(sph_ctx *c, int n, const sph_problem *problems, sph_stats *stats) {
    if (!c) return SPH_EINVAL;
    if (c->poisoned) return fail(c, SPH_ECUDA, "context poisoned by an earlier CUDA error");
    if (n < 0 || (n > 0 && !problems)) return fail(c, SPH_EINVAL, "bad batch");
    if (!c->crit_set) return fail(c, SPH_ESTATE, "set_criteria has not been called");
    if (n == 0) {
        if (stats) memset(stats, 0, sizeof *stats);
        return SPH_OK;
    }
    CK(cudaSetDevice(c->device));
    return run_batch(c, n, problems, stats);
}

int eval_sph_host(sph_ctx *c, const float *q_host, const float *emag_host, const uint8_t *mask_host,
                  float *s_host, sph_stats *stats) {
    if (!c) return SPH_EINVAL;
    if (!q_host || !s_host) return fail(c, SPH_EINVAL, "q_host and s_host must be non-NULL");
    if (emag_host && mask_host) return fail(c, SPH_EINVAL, "give |E| or a mask, not both");
    if (!c->grid_set) return fail(c, SPH_ESTATE, "set_grid has not been called");
    if (!c->crit_set) return fail(c, SPH_ESTATE, "set_criteria has not been called");
    if (c->source_scale <= 0) return fail(c, SPH_ESTATE, "set_sources has not been called (source_scale)");
    if (c->poisoned) return fail(c, SPH_ECUDA, "context poisoned by an earlier CUDA error");
    CK(cudaSetDevice(c->device));
    const size_t n = (size_t)c->nx * c->ny * c->nz;
    ENS(c->h_q, n * sizeof(float));
    ENS(c->h_s, n * sizeof(float));
    CK(cudaMemcpyAsync(c->h_q.p, q_host, n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    const float *e = nullptr;
    const uint8_t *m = nullptr;
    if (emag_host) {
        ENS(c->h_e, n * sizeof(float));
        CK(cudaMemcpyAsync(c->h_e.p, emag_host, n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        e = P<float>(c->h_e);
    } else if (mask_host) {
        ENS(c->h_m, n);
        CK(cudaMemcpyAsync(c->h_m.p, mask_host, n, cudaMemcpyHostToDevice, c->stream));
        m = P<uint8_t>(c->h_m);
    }
    c->q = P<float>(c->h_q);
    c->src_set = true;
    c->emag = e;
    c->mask = m;
    c->trg_set = true;
    int r = run_fmm(c, P<float>(c->h_s), stats);
    if (r) return r;
    CK(cudaMemcpyAsync(s_host, c->h_s.p, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return SPH_OK;
}

int eval_direct(sph_ctx *c, int fp64, void *s_dev) {
    int r = check_ready(c);
    if (r) return r;
    if (!s_dev) return fail(c, SPH_EINVAL, "s_dev is NULL");
    if (fp64 != 0 && fp64 != 1) return fail(c, SPH_EINVAL, "fp64 must be 0 or 1");
    r = run_select(c);
    if (r) return r;
    // the self term needs the ball integral: computed with the operators' precompute
    const size_t n = (size_t)c->nx * c->ny * c->nz;
    CK(cudaMemsetAsync(s_dev, 0, n * (fp64 ? sizeof(double) : sizeof(float)), c->stream));
    if (!c->ops_valid || c->ops_h != c->h || c->ops_a != c->alpha || c->ops_b != c->beta) {
        c->Lmax = 0;   // only the self integral is needed
        r = run_ops(c);
        if (r) return r;
    }
    DirectArgs A;
    A.src_pc = P<uint32_t>(c->b_spc);
    A.src_q = P<float>(c->b_sq);
    A.wscale = (float)(c->source_scale * c->h * c->h * c->h);
    A.ns = (int)c->ns;
    A.trg_key = P<uint32_t>(c->b_tkey);
    A.nt = (int)c->nt;
    A.kp = make_kp(c);
    double L = std::log(c->beta / c->alpha);
    A.kp64.alpha = c->alpha; A.kp64.bma = c->beta - c->alpha; A.kp64.C = 1.0 / (4.0 * M_PI * L);
    A.kp64.h = c->h; A.kp64.vol = c->h * c->h * c->h; A.kp64.scale = c->source_scale;
    A.kp64.self_int = c->self_int;
    A.self_mode = c->self_mode; A.nx = c->nx; A.ny = c->ny; A.fp64 = fp64;
    A.out = s_dev;
    if (direct_launch(A, c->stream) != 0) CK(cudaGetLastError());
    return SPH_OK;
}

int sph_get_selection(sph_ctx *c, int32_t *src_host, int64_t *n_src, int32_t *trg_host, int64_t *n_trg) {
    if (!c) return SPH_EINVAL;
    if (c->poisoned) return fail(c, SPH_ECUDA, "context poisoned");
    if (n_src) *n_src = c->ns;
    if (n_trg) *n_trg = c->nt;
    if (!src_host && !trg_host) return SPH_OK;
    CK(cudaStreamSynchronize(c->stream));
    // packed cells (sources) or Morton keys (targets, whose cells follow from the key)
    auto fetch = [&](DevBuf &pcb, int64_t n, int32_t *dst, bool keys) -> int {
        std::vector<uint32_t> pc(n);
        if (n) {
            cudaError_t e = cudaMemcpy(pc.data(), pcb.p, n * sizeof(uint32_t), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_fail(c, e, "selection read-back");
        }
        for (int64_t i = 0; i < n; ++i) {
            const uint32_t p = keys ? key_pc(pc[i]) : pc[i];
            dst[i] = pc_i(p) + c->nx * (pc_j(p) + c->ny * pc_k(p));
        }
        std::sort(dst, dst + n);
        return SPH_OK;
    };
    if (src_host) { int r = fetch(c->b_spc, c->ns, src_host, false); if (r) return r; }
    if (trg_host) { int r = fetch(c->b_tkey, c->nt, trg_host, true); if (r) return r; }
    return SPH_OK;
}

int sph_get_tree(sph_ctx *c, sph_tree_view *tv) {
    if (!c || !tv) return SPH_EINVAL;
    if (c->poisoned) return fail(c, SPH_ECUDA, "context poisoned");
    if (!c->have_tree) return fail(c, SPH_ESTATE, "no tree: run eval_sph first");
    tv->n_boxes = c->nboxes;
    tv->n_u = c->list_tot[0]; tv->n_v = c->list_tot[1]; tv->n_w = c->list_tot[2]; tv->n_x = c->list_tot[3];
    tv->depth = c->D;
    if (!tv->level) return SPH_OK;
    CK(cudaStreamSynchronize(c->stream));
    const int nb = c->nboxes;
    auto get = [&](void *dst, DevBuf &b, size_t bytes) -> int {
        if (!dst || !bytes) return SPH_OK;
        cudaError_t e = cudaMemcpy(dst, b.p, bytes, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(c, e, "tree read-back");
        return SPH_OK;
    };
    int r = 0;
    if ((r = get(tv->level, c->b_level, nb * sizeof(int)))) return r;
    if ((r = get(tv->key, c->b_key, nb * sizeof(uint32_t)))) return r;
    if ((r = get(tv->src_begin, c->b_sb, nb * sizeof(int)))) return r;
    if ((r = get(tv->src_end, c->b_se, nb * sizeof(int)))) return r;
    if ((r = get(tv->trg_begin, c->b_tb, nb * sizeof(int)))) return r;
    if ((r = get(tv->trg_end, c->b_te, nb * sizeof(int)))) return r;
    if ((r = get(tv->parent, c->b_parent, nb * sizeof(int)))) return r;
    if ((r = get(tv->is_leaf, c->b_leaf, nb))) return r;
    ListDev L = list_dev(c);
    std::vector<int> off((size_t)nb + 1), src;
    auto pairs = [&](const int *doff, const int *dsrc, int tot, int32_t *dst) -> int {
        if (!dst) return SPH_OK;
        cudaError_t e = cudaMemcpy(off.data(), doff, (nb + 1) * sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(c, e, "list read-back");
        src.resize(std::max(tot, 1));
        if (tot) {
            e = cudaMemcpy(src.data(), dsrc, tot * sizeof(int), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_fail(c, e, "list read-back");
        }
        std::vector<std::pair<int, int>> pr;
        pr.reserve(tot);
        for (int b = 0; b < nb; ++b)
            for (int k = off[b]; k < off[b + 1]; ++k) pr.emplace_back(b, src[k]);
        std::sort(pr.begin(), pr.end());
        for (size_t k = 0; k < pr.size(); ++k) {
            dst[2 * k] = pr[k].first;
            dst[2 * k + 1] = pr[k].second;
        }
        return SPH_OK;
    };
    if ((r = pairs(L.u_off, L.u_src, c->list_tot[0], tv->u_pairs))) return r;
    if ((r = pairs(L.v_off, L.v_src, c->list_tot[1], tv->v_pairs))) return r;
    if ((r = pairs(L.w_off, L.w_src, c->list_tot[2], tv->w_pairs))) return r;
    if ((r = pairs(L.x_off, L.x_src, c->list_tot[3], tv->x_pairs))) return r;
    return SPH_OK;
}

}  // extern "C"
