// Morton octree over the selected points and its interaction lists (Section 2.4: leaves
// bounded in point count, the near / far split of Eq. nearfar, the recursive far-field
// hierarchy).
//
// Build: the grid is embedded in a 2^D cube of cells.  Level l has a dense array
// box_at[l][key] (8^l entries, -1 = no box), so every neighbour lookup is one load.
//   k_tree_ranges : one pass over the Morton-sorted keys gives every dense slot of every
//                   level its [begin, end) point range (sources and targets);
//   k_tree_exists : a slot holds a box iff it has points and its parent was split;
//   scan          : exclusive scan of the existence flags -> canonical index
//                   (boxes ordered by (level, key));
//   k_tree_emit_all : the compact box records, box_at and the per-slot source flag.
// A box splits iff it holds more than S sources or more than S targets and its
// level is below D.  All of it is integer arithmetic, so the tree is
// bit-identical to the oracle's.
//
// Lists (per target-side box B, pairs (B, A)):
//   U: B leaf, A leaf with sources, adjacent (touching or overlapping closed cubes);
//   V: same level >= 2, parents adjacent, A not adjacent to B; offset code kept;
//   W: B leaf, A finer with sources, parent(A) adjacent to B, A not adjacent;
//   X: A leaf with sources, coarser than B, A adjacent to parent(B), not to B.
// k_lists_classify + k_lists_warp<false> count, one scan gives the four CSR offset arrays,
// k_lists_warp<true> fills.
#include <algorithm>

#include "sph_kernels.cuh"

namespace sph {

// ------------------------------------------------------------ device-wide scan
// One launch per scan (up to four arrays of the same length at once, blockIdx.y).  A CTA
// scans a tile of SCAN_TILE ints staged through shared memory; tiles find their offset by
// decoupled look-back in ticket order (state word: 2-bit status | 32-bit value), or, for
// short arrays, one CTA per array walks every tile with a running carry.
constexpr int SCAN_PER = 8;
constexpr int SCAN_T = 256, SCAN_TILE = SCAN_T * SCAN_PER;          // look-back tiles (2048 ints)
constexpr int SCAN_ST = 1024, SCAN_STILE = SCAN_ST * SCAN_PER;      // the one-CTA form's tiles
constexpr int SCAN_SMALL = 4 * SCAN_STILE;         // one CTA per array up to this length
constexpr unsigned long long ST_AGG = 1ull << 62, ST_INC = 2ull << 62;

struct ScanSet {
    const int *in[4];
    int *out[4];
    int *total[4];
};

__device__ __forceinline__ int spad(int i) { return i + (i >> 5); }

// Exclusive scan of one tile of NT * SCAN_PER ints staged through shared memory: returns the
// tile's sum (every thread), leaves the thread's exclusive prefix in *pre and its SCAN_PER
// elements in v.  ws: [32] shared.
template <int NT>
__device__ __forceinline__ int tile_scan(const int *__restrict__ in, int base, int n, int *sh, int *ws,
                                         int (&v)[SCAN_PER], int *pre) {
    constexpr int NW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
#pragma unroll
    for (int u = 0; u < SCAN_PER; ++u) {
        const int i = u * NT + tid;
        sh[spad(i)] = base + i < n ? in[base + i] : 0;
    }
    __syncthreads();
    int s = 0;
#pragma unroll
    for (int u = 0; u < SCAN_PER; ++u) {
        v[u] = sh[spad(tid * SCAN_PER + u)];
        s += v[u];
    }
    int inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) ws[w] = inc;
    __syncthreads();
    if (w == 0) {
        int t = lane < NW ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < NW) ws[lane] = t;
    }
    __syncthreads();
    *pre = (w ? ws[w - 1] : 0) + inc - s;
    return ws[NW - 1];
}

// The tile's exclusive prefixes (offset x added) written back through shared memory, coalesced.
template <int NT>
__device__ __forceinline__ void tile_store(int *__restrict__ out, int base, int n, int *sh, const int (&v)[SCAN_PER],
                                           int x) {
    const int tid = threadIdx.x;
    __syncthreads();
#pragma unroll
    for (int u = 0; u < SCAN_PER; ++u) {
        sh[spad(tid * SCAN_PER + u)] = x;
        x += v[u];
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < SCAN_PER; ++u) {
        const int i = u * NT + tid;
        if (base + i < n) out[base + i] = sh[spad(i)];
    }
}

__global__ void __launch_bounds__(SCAN_ST) k_scan_small(ScanSet S, int n) {
    pdl_enter();
    __shared__ int sh[SCAN_STILE + SCAN_STILE / 32];
    __shared__ int ws[32];
    const int a = blockIdx.y;
    int carry = 0;
    for (int base = 0; base < n; base += SCAN_STILE) {
        int v[SCAN_PER], pre;
        const int sum = tile_scan<SCAN_ST>(S.in[a], base, n, sh, ws, v, &pre);
        tile_store<SCAN_ST>(S.out[a], base, n, sh, v, carry + pre);
        carry += sum;
        __syncthreads();      // ws / sh are reused by the next tile
    }
    if (threadIdx.x == 0) *S.total[a] = carry;
}

// state: per array ntiles + 1 words (the last one is the ticket), zeroed before the launch.
// A tile that gives up waiting for a predecessor counts it as zero (its prefixes stay in
// [0, true prefix], so indices derived from them stay in bounds) and sets bit 0 of *err.
__global__ void __launch_bounds__(SCAN_T) k_scan_onepass(ScanSet S, int n, int ntiles,
                                                         unsigned long long *__restrict__ state, int *err,
                                                         unsigned wait_limit) {
    pdl_enter();
    __shared__ int sh[SCAN_TILE + SCAN_TILE / 32];
    __shared__ int ws[32];
    __shared__ int s_tile, s_pre;
    const int a = blockIdx.y, tid = threadIdx.x;
    unsigned long long *st = state + (size_t)a * (ntiles + 1);
    if (tid == 0) s_tile = (int)atomicAdd(st + ntiles, 1ull);
    __syncthreads();
    const int tile = s_tile, base = tile * SCAN_TILE;
    int v[SCAN_PER], pre;
    const int sum = tile_scan<SCAN_T>(S.in[a], base, n, sh, ws, v, &pre);
    if (tid < 32) {
        if (tid == 0) atomicExch(st + tile, (tile == 0 ? ST_INC : ST_AGG) | (unsigned)sum);
        __syncwarp();
        // warp 0 walks back 32 predecessors at a time; the nearest inclusive state ends the walk
        unsigned run = 0;
        bool gave_up = false;
        for (int j = tile - 1; j >= 0; j -= 32) {
            const int idx = j - tid;
            unsigned long long w = ST_INC;   // before tile 0: an inclusive zero
            unsigned k = 0;
            for (; k < wait_limit; ++k) {
                if (idx >= 0) w = *((volatile unsigned long long *)(st + idx));
                if (__all_sync(0xffffffffu, (w >> 62) != 0)) break;
                __nanosleep(32);
            }
            if (k == wait_limit) {
                gave_up = true;
                break;
            }
            const unsigned inc_mask = __ballot_sync(0xffffffffu, (w >> 62) == 2);
            const int stop = inc_mask ? __ffs(inc_mask) - 1 : 31;
            unsigned c = (tid <= stop && idx >= 0) ? (unsigned)w : 0u;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
            run += c;
            if (inc_mask) break;
        }
        if (tid == 0) {
            if (gave_up && err) atomicOr(err, 1);
            if (tile > 0) atomicExch(st + tile, ST_INC | (unsigned)(run + (unsigned)sum));
            s_pre = (int)run;
            if (tile == ntiles - 1) *S.total[a] = (int)run + sum;
        }
    }
    __syncthreads();
    tile_store<SCAN_T>(S.out[a], base, n, sh, v, s_pre + pre);
}

size_t scan_tmp_ints(int n) {
    const int ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    return 2 * 4 * ((size_t)ntiles + 1) + 16;
}

// out_k[i] = sum_{j<i} in_k[j]; *total_k = sum (device), for k <= 4 arrays of length n.
// tmp: scan_tmp_ints(n) ints, 8-byte aligned; err (optional): bit 0 set if a look-back gave up.
size_t scan_state_bytes(int k, int n) {
    if (n <= SCAN_SMALL) return 0;
    const int ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    return sizeof(unsigned long long) * (size_t)k * (size_t)(ntiles + 1);
}

__global__ void __launch_bounds__(256) k_zero_set(ZeroSet Z) {
    pdl_enter();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int s = 0; s < Z.n; ++s)
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Z.words[s]; i += stride) Z.p[s][i] = 0;
}

void zero_set_launch(const ZeroSet &Z, cudaStream_t st) {
    int64_t mx = 0;
    for (int s = 0; s < Z.n; ++s) mx = std::max(mx, Z.words[s]);
    if (mx <= 0) return;
    const int grid = (int)std::min<int64_t>((mx + 255) / 256, 152 * 4);
    launch_pdl(k_zero_set, grid, 256, 0, st, Z);
}

// state_zeroed: the look-back state (scan_state_bytes(k, n) at tmp) is already clear
void scan_exclusive_multi(const ScanSet &S, int k, int n, int *tmp, int *err, cudaStream_t st,
                          unsigned wait_limit = SCAN_WAIT_LIMIT, bool state_zeroed = false) {
    if (n <= 0) {
        for (int a = 0; a < k; ++a) cudaMemsetAsync(S.total[a], 0, sizeof(int), st);
        return;
    }
    if (n <= SCAN_SMALL) {
        launch_pdl(k_scan_small, dim3(1, k), SCAN_ST, 0, st, S, n);
        return;
    }
    const int ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    unsigned long long *state = reinterpret_cast<unsigned long long *>(tmp);
    if (!state_zeroed) cudaMemsetAsync(state, 0, sizeof(unsigned long long) * k * (ntiles + 1), st);
    launch_pdl(k_scan_onepass, dim3(ntiles, k), SCAN_T, 0, st, S, n, ntiles, state, err, wait_limit);
}

void scan_exclusive(const int *in, int *out, int n, int *total, int *tmp, cudaStream_t st, int *err,
                    unsigned wait_limit, bool state_zeroed) {
    ScanSet S{};
    S.in[0] = in;
    S.out[0] = out;
    S.total[0] = total;
    scan_exclusive_multi(S, 1, n, tmp, err, st, wait_limit, state_zeroed);
}

// ------------------------------------------------------------ tree build
__device__ __forceinline__ int lower_bound_u32(const uint32_t *a, int lo, int hi, uint32_t v) {
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Point ranges of every dense slot of every level in one pass over the Morton-sorted keys:
// point i opens the range of its slot at level l when point i-1 lies in another slot of
// that level, and closes it when point i+1 does.  Untouched slots keep [0, 0).
// Eight keys per thread (two 16-byte loads), neighbours through warp shuffles.  A key whose
// finest slot (level Lmax) matches both neighbours' -- all but about one in 8^(D-Lmax) --
// costs a few integer operations; the boundary writes are queued in shared memory and
// carried out by the whole block, so that no warp runs them one lane at a time.
constexpr int RANGE_PER = 8, RANGE_T = 256;

// Target ranges from the selection's per-brick offsets (bricks of 16^3 cells, Morton order,
// brick b's targets at [boff[b], boff[b + 1]) of the key array, boff[nbr] = nt): a slot of a
// level at or above the bricks' (D - 4) spans whole bricks; a finer slot lies inside one brick,
// whose keys are (b << 12) | local index -- consecutive where every cell is a target, found by
// two binary searches over the brick's keys otherwise.  One thread per dense slot.
__device__ __forceinline__ void slot_range_from_bricks(int64_t s, int Lmax, int D, const int *__restrict__ boff,
                                                       int nbr, int nt, const uint32_t *__restrict__ key,
                                                       int &tb, int &te) {
    int l = 0;
    while (l < Lmax && s >= dense_off(l + 1)) ++l;
    const uint32_t m = (uint32_t)(s - dense_off(l));
    auto off = [&](uint32_t b) { return b < (uint32_t)nbr ? boff[b] : nt; };
    if (l <= D - 4) {
        const int sh = 3 * (D - 4 - l);
        tb = off(m << sh);
        te = off((m + 1) << sh);
        return;
    }
    const int sh = 3 * (D - l);
    const uint32_t k0 = m << sh, b = k0 >> 12;
    const int ob = off(b), oe = off(b + 1);
    if (oe - ob == 4096) {
        tb = ob + (int)(k0 & 4095u);
        te = tb + (1 << sh);
        return;
    }
    int lo = ob, hi = oe;                                   // first key >= k0
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (key[mid] < k0) lo = mid + 1; else hi = mid;
    }
    tb = lo;
    hi = oe;                                                // first key >= k0 + 8^(D-l)
    const uint32_t k1 = k0 + (1u << sh);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (key[mid] < k1) lo = mid + 1; else hi = mid;
    }
    te = lo;
}

// One launch for both point sets: blocks [0, gs) take the sources (grid-stride over gs blocks),
// the others the targets -- by a pass over the keys, or (boff != nullptr) slot by slot from the
// selection's per-brick offsets.
__global__ void __launch_bounds__(RANGE_T) k_tree_ranges(const int *__restrict__ ns_dev, const uint32_t *__restrict__ skey,
                                                         int *__restrict__ sbeg, int *__restrict__ send, int gs,
                                                         const int *__restrict__ nt_dev, const uint32_t *__restrict__ tkey,
                                                         int *__restrict__ tbeg, int *__restrict__ tend, int D, int Lmax,
                                                         const int *__restrict__ boff, int nbr, int64_t nslot) {
    pdl_enter();
    const bool src = (int)blockIdx.x < gs;
    if (!src && boff) {
        const int64_t s = (int64_t)(blockIdx.x - gs) * blockDim.x + threadIdx.x;
        if (s >= nslot) return;
        const int nt = max(*nt_dev, 0);
        int tb, te;
        slot_range_from_bricks(s, Lmax, D, boff, nbr, nt, tkey, tb, te);
        tbeg[s] = tb;
        tend[s] = te;
        return;
    }
    const int bid = src ? (int)blockIdx.x : (int)blockIdx.x - gs, nblk = src ? gs : (int)gridDim.x - gs;
    const int *n_dev = src ? ns_dev : nt_dev;
    const uint32_t *key = src ? skey : tkey;
    int *beg = src ? sbeg : tbeg, *end = src ? send : tend;
    __shared__ uint32_t task_key[2 * RANGE_PER * RANGE_T];
    __shared__ int task_val[2 * RANGE_PER * RANGE_T];
    __shared__ uint8_t task_lvl[2 * RANGE_PER * RANGE_T];   // first level | 0x80 for an end
    __shared__ int ntask;
    const int n = *n_dev;                 // a negative count (failed selection) reads as none
    const int lane = threadIdx.x & 31;
    const int fine = 3 * (D - Lmax);
    // two keys fall in different slots of level l iff their highest differing bit b (0-based)
    // satisfies b >= 3 (D - l), i.e. for every l >= D - b / 3
    auto first_level = [&](uint32_t x, uint32_t o) { return max(0, D - (31 - __clz(x ^ o)) / 3); };
    // grid-stride over chunks of RANGE_T * RANGE_PER keys (uniform across the block); point
    // counts stay below 2^30 (grids of at most 1024^3 cells), so int indices do not overflow
    for (int base = bid * RANGE_T * RANGE_PER; base < n; base += nblk * RANGE_T * RANGE_PER) {
        const int i0 = base + threadIdx.x * RANGE_PER;
        if (threadIdx.x == 0) ntask = 0;
        uint32_t k[RANGE_PER];
        if (i0 + RANGE_PER <= n) {
            const uint4 v0 = *reinterpret_cast<const uint4 *>(key + i0);
            const uint4 v1 = *reinterpret_cast<const uint4 *>(key + i0 + 4);
            k[0] = v0.x; k[1] = v0.y; k[2] = v0.z; k[3] = v0.w;
            k[4] = v1.x; k[5] = v1.y; k[6] = v1.z; k[7] = v1.w;
        } else {
#pragma unroll
            for (int u = 0; u < RANGE_PER; ++u) k[u] = i0 + u < n ? key[i0 + u] : 0u;
        }
        // every lane takes part in the shuffles; lanes past the end only supply values nobody uses
        uint32_t prev = __shfl_up_sync(0xffffffffu, k[RANGE_PER - 1], 1);
        uint32_t next = __shfl_down_sync(0xffffffffu, k[0], 1);
        if (lane == 0) prev = (i0 > 0 && i0 - 1 < n) ? key[i0 - 1] : 0u;
        if (lane == 31) next = (i0 + RANGE_PER < n) ? key[i0 + RANGE_PER] : 0u;
        __syncthreads();
#pragma unroll
        for (int u = 0; u < RANGE_PER; ++u) {
            const int i = i0 + u;
            if (i >= n) break;
            const uint32_t p = u == 0 ? prev : k[u - 1];
            const uint32_t q = u == RANGE_PER - 1 ? next : k[u + 1];
            if (i == 0 || ((k[u] ^ p) >> fine) != 0) {
                const int s = atomicAdd(&ntask, 1);
                task_key[s] = k[u];
                task_val[s] = i;
                task_lvl[s] = (uint8_t)(i == 0 ? 0 : first_level(k[u], p));
            }
            if (i + 1 == n || ((k[u] ^ q) >> fine) != 0) {
                const int s = atomicAdd(&ntask, 1);
                task_key[s] = k[u];
                task_val[s] = i + 1;
                task_lvl[s] = (uint8_t)(0x80 | (i + 1 == n ? 0 : first_level(k[u], q)));
            }
        }
        __syncthreads();
        for (int s = threadIdx.x; s < ntask; s += RANGE_T) {
            const uint32_t kk = task_key[s];
            const int val = task_val[s];
            const int l0 = task_lvl[s] & 0x7f;
            int *out = (task_lvl[s] & 0x80) ? end : beg;
            int64_t off = dense_off(l0);
            for (int l = l0; l <= Lmax; ++l, off = 8 * off + 1) out[off + (kk >> (3 * (D - l)))] = val;
        }
        __syncthreads();                      // the task queue is reused by the next chunk
    }
}

__device__ __forceinline__ int level_of_slot(int64_t s, int Lmax) {
    int l = 0;
    while (l < Lmax && s >= dense_off(l + 1)) ++l;
    return l;
}

// A slot holds a box iff it has points and its parent was split (ns > S or nt > S at a
// level < D).  Point counts only shrink from parent to child, so a split parent implies
// that every ancestor was split as well.
__global__ void k_tree_exists(int64_t nslot, int Lmax, int D, int S, const int *__restrict__ rsb,
                              const int *__restrict__ rse, const int *__restrict__ rtb, const int *__restrict__ rte,
                              int *__restrict__ flag) {
    pdl_enter();
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nslot) return;
    const int l = level_of_slot(s, Lmax);
    const int ns = rse[s] - rsb[s], nt = rte[s] - rtb[s];
    bool ex = ns + nt > 0;
    if (ex && l > 0) {
        const int64_t ps = dense_off(l - 1) + ((s - dense_off(l)) >> 3);
        const int pns = rse[ps] - rsb[ps], pnt = rte[ps] - rtb[ps];
        ex = (l - 1 < D) && (pns > S || pnt > S);
    }
    flag[s] = ex ? 1 : 0;
}

// Boxes in (level, key) order: box index = exclusive scan of the existence flags.
__global__ void __launch_bounds__(256) k_tree_emit_all(TreeDev T, int64_t nslot, int Lmax, int D, int S,
                                                      const int *__restrict__ flag, const int *__restrict__ pos,
                                                      const int *__restrict__ rsb, const int *__restrict__ rse,
                                                      const int *__restrict__ rtb, const int *__restrict__ rte,
                                                      const int *__restrict__ total, const uint32_t *__restrict__ skey,
                                                      const int *__restrict__ ns_dev, const uint32_t *__restrict__ tkey,
                                                      const int *__restrict__ nt_dev, uint8_t *__restrict__ vsrc,
                                                      uint8_t *__restrict__ occ, int64_t npar) {
    pdl_enter();
    // per-level counts of the block's boxes with sources and leaves with targets, added into
    // the level tables once per block and level (the same few counters for every block)
    __shared__ int s_src[16], s_leaf[16], s_sleaf[16];
    if (threadIdx.x < 16) {
        s_src[threadIdx.x] = 0;
        s_leaf[threadIdx.x] = 0;
        s_sleaf[threadIdx.x] = 0;
    }
    __syncthreads();
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (occ && s < npar) {
        // occ[s], levels 0..Lmax-1: the slot's region holds a source point, or lies inside a leaf
        // that holds sources (the deepest existing box over the slot, found from the existence
        // flags and point ranges)
        uint8_t o = rse[s] > rsb[s];
        if (!o) {
            int l = level_of_slot(s, Lmax);
            int64_t m = s - dense_off(l);
            for (; l >= 0; --l, m >>= 3) {
                const int64_t a = dense_off(l) + m;
                if (flag[a]) {
                    const int ns = rse[a] - rsb[a], nt = rte[a] - rtb[a];
                    o = !(l < D && (ns > S || nt > S)) && ns > 0;
                    break;
                }
            }
        }
        occ[s] = o;
    }
    if (s <= Lmax) {       // level table (threads 0..Lmax)
        const int l = (int)s;
        const int b0 = pos[dense_off(l)];
        const int b1 = l < Lmax ? pos[dense_off(l + 1)] : *total;
        T.lvl_base[l] = b0;
        T.lvl_count[l] = b1 - b0;
    }
    if (s < nslot && !flag[s]) {
        T.box_at[s] = -1;
        vsrc[s] = 0;
    } else if (s < nslot) {
        const int l = level_of_slot(s, Lmax);
        const int64_t m = s - dense_off(l);
        const int idx = pos[s];
        T.box_at[s] = idx;
        int sb = rsb[s], se = rse[s], tb = rtb[s], te = rte[s];
        // an empty range starts where the slot's first key would be inserted
        const uint32_t lo = (uint32_t)m << (3 * (D - l));
        if (se == sb) sb = se = lower_bound_u32(skey, 0, max(*ns_dev, 0), lo);
        if (te == tb) tb = te = lower_bound_u32(tkey, 0, max(*nt_dev, 0), lo);
        T.b_level[idx] = l;
        T.b_key[idx] = (uint32_t)m;
        T.b_sb[idx] = sb; T.b_se[idx] = se;
        T.b_tb[idx] = tb; T.b_te[idx] = te;
        T.b_parent[idx] = l > 0 ? pos[dense_off(l - 1) + (m >> 3)] : -1;
        const bool leaf = !(l < D && (se - sb > S || te - tb > S));
        T.b_leaf[idx] = leaf;
        vsrc[s] = se > sb;
        if (se > sb) atomicAdd(s_src + l, 1);
        if (leaf && te > tb) atomicAdd(s_leaf + l, 1);
        if (leaf && se > sb) atomicAdd(s_sleaf + l, 1);
    }
    __syncthreads();
    if (threadIdx.x < 16) {
        if (s_src[threadIdx.x]) atomicAdd(T.lvl_src + threadIdx.x, s_src[threadIdx.x]);
        if (s_leaf[threadIdx.x]) atomicAdd(T.lvl_leaf + threadIdx.x, s_leaf[threadIdx.x]);
        if (s_sleaf[threadIdx.x]) atomicAdd(T.lvl_sleaf + threadIdx.x, s_sleaf[threadIdx.x]);
    }
}

__global__ void k_src_near(int64_t nslot, int Lmax, const uint8_t *__restrict__ occ, uint8_t *__restrict__ near) {
    pdl_enter();
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nslot) return;
    const int l = level_of_slot(s, Lmax);
    const uint32_t m = (uint32_t)(s - dense_off(l));
    uint32_t x, y, z;
    demorton3(m, x, y, z);
    const int n = 1 << l;
    uint8_t v = 0;
    for (int dz = -1; dz <= 1 && !v; ++dz)
        for (int dy = -1; dy <= 1 && !v; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int qx = (int)x + dx, qy = (int)y + dy, qz = (int)z + dz;
                if (qx < 0 || qy < 0 || qz < 0 || qx >= n || qy >= n || qz >= n) continue;
                if (occ[dense_off(l) + morton3(qx, qy, qz)]) {
                    v = 1;
                    break;
                }
            }
    near[s] = v;
}

void tree_build_launch(const TreeArgs &A, cudaStream_t st) {
    const int64_t nslot = dense_off(A.Lmax + 1);
    if (A.zeroed) {
        // the source ranges were cleared before the evaluation (zero_set_launch); the target
        // ranges too need clearing unless the brick offsets write every slot's
        if (!A.brick_off_t) {
            cudaMemsetAsync(A.rtb, 0, nslot * sizeof(int), st);
            cudaMemsetAsync(A.rte, 0, nslot * sizeof(int), st);
        }
    } else if (A.brick_off_t) {
        // the target ranges of every slot are written from the brick offsets
        cudaMemsetAsync(A.rsb, 0, nslot * sizeof(int), st);
        cudaMemsetAsync(A.rse, 0, nslot * sizeof(int), st);
    } else if (A.rse == A.rsb + nslot && A.rtb == A.rse + nslot && A.rte == A.rtb + nslot) {
        cudaMemsetAsync(A.rsb, 0, 4 * nslot * sizeof(int), st);
    } else {
        cudaMemsetAsync(A.rsb, 0, nslot * sizeof(int), st);
        cudaMemsetAsync(A.rse, 0, nslot * sizeof(int), st);
        cudaMemsetAsync(A.rtb, 0, nslot * sizeof(int), st);
        cudaMemsetAsync(A.rte, 0, nslot * sizeof(int), st);
    }
    constexpr int RB = RANGE_T * RANGE_PER;
    // targets: enough blocks for every possible point (blocks past the actual count exit at
    // once); sources, usually far fewer: a grid-stride loop over 8 blocks per SM
    const int rg = (int)std::min<int64_t>(((int64_t)A.ncap + RB - 1) / RB, 1 << 20);
    const int gs = std::max(std::min(rg, 152 * 8), 1);
    const int gt = A.brick_off_t ? (int)((nslot + RANGE_T - 1) / RANGE_T) : std::max(rg, 1);
    launch_pdl(k_tree_ranges, gs + gt, RANGE_T, 0, st, A.ns_dev, A.skey, A.rsb, A.rse, gs, A.nt_dev,
               A.tkey, A.rtb, A.rte, A.D, A.Lmax, A.brick_off_t, A.nbr, nslot);
    const int grid = (int)((nslot + 255) / 256);
    if (!A.zeroed) cudaMemsetAsync(A.T.lvl_src, 0, 48 * sizeof(int), st);   // lvl_src, lvl_leaf and lvl_sleaf
    launch_pdl(k_tree_exists, grid, 256, 0, st, nslot, A.Lmax, A.D, A.S, A.rsb, A.rse, A.rtb, A.rte, A.flag);
    int *total = A.pos + nslot;
    scan_exclusive(A.flag, A.pos, (int)nslot, total, A.scan_tmp, st, A.err, SCAN_WAIT_LIMIT, A.zeroed);
    const int64_t npar = dense_off(A.Lmax);        // slots of levels 0..Lmax-1
    launch_pdl(k_tree_emit_all, grid, 256, 0, st, A.T, nslot, A.Lmax, A.D, A.S, A.flag, A.pos, A.rsb, A.rse, A.rtb,
                                          A.rte, total, A.skey, A.ns_dev, A.tkey, A.nt_dev, A.vsrc,
                                          (npar > 0 && A.near) ? A.occ : nullptr, npar);
    if (npar > 0 && A.occ && A.near) {
        const int g2 = (int)((npar + 255) / 256);
        launch_pdl(k_src_near, g2, 256, 0, st, npar, A.Lmax - 1, A.occ, A.near);
    }
}

// ------------------------------------------------------------ interaction lists
struct BoxGeom {
    int level;
    int x, y, z;   // coordinates at its level
};

__device__ __forceinline__ BoxGeom geom_of(const TreeDev &T, int b) {
    BoxGeom g;
    g.level = T.b_level[b];
    uint32_t x, y, z;
    demorton3(T.b_key[b], x, y, z);
    g.x = (int)x; g.y = (int)y; g.z = (int)z;
    return g;
}

// closed cubes touch or overlap (cell units, depth D)
__device__ __forceinline__ bool adjacent(const BoxGeom &a, const BoxGeom &b, int D) {
    int sa = 1 << (D - a.level), sb = 1 << (D - b.level);
    int ax = a.x * sa, ay = a.y * sa, az = a.z * sa;
    int bx = b.x * sb, by = b.y * sb, bz = b.z * sb;
    return ax <= bx + sb && bx <= ax + sa && ay <= by + sb && by <= ay + sa && az <= bz + sb && bz <= az + sa;
}


// Lists in two steps.  k_lists_classify (thread per box) finds the boxes that can have an
// entry -- targets, and sources somewhere around the parent -- and queues them (any order:
// every box writes only its own CSR range); the others get empty lists.  k_lists_warp
// then takes one queued box per warp: the 27 neighbour slots of U / W and of X one per
// lane, the 216 V candidates 32 at a time, entries placed in slot order by warp prefix
// sums, so every list comes out exactly as a serial walk of the slots would write it.
__global__ void k_lists_classify(TreeDev T, ListDev L, int cap, const int *__restrict__ nboxes_dev) {
    pdl_enter();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= cap) return;
    bool heavy = false;
    if (b < *nboxes_dev && T.b_te[b] > T.b_tb[b]) {
        const int l = T.b_level[b];
        // nothing with sources anywhere around the parent: every list is empty
        heavy = !(l >= 1 && T.near && !T.near[dense_off(l - 1) + (T.b_key[b] >> 3)]);
    }
    if (heavy) {
        L.heavy[atomicAdd(L.nheavy, 1)] = b;
    } else {
        L.u_cnt[b] = 0; L.v_cnt[b] = 0; L.w_cnt[b] = 0; L.x_cnt[b] = 0;
    }
}

// Descendants of a split colleague A of leaf B: adjacent leaves with sources join U, the
// first non-adjacent boxes with sources join W (depth first, children in key order).
template <bool FILL>
__device__ __noinline__ void lists_descend(const TreeDev &T, const ListDev &L, const BoxGeom &B, int D, int A,
                                           int pu, int pw, int &cu, int &cw) {
    int stk[128];
    int sp = 0;
    const uint32_t ck = T.b_key[A] << 3;
    for (int c = 0; c < 8; ++c) {
        const int C = T.box_at[dense_off(B.level + 1) + ck + c];
        if (C >= 0) stk[sp++] = C;
    }
    while (sp > 0) {
        const int Dn = stk[--sp];
        const BoxGeom G = geom_of(T, Dn);
        const bool hs = T.b_se[Dn] > T.b_sb[Dn];
        if (adjacent(G, B, D)) {
            if (T.b_leaf[Dn]) {
                if (hs) {
                    if (FILL) L.u_src[pu + cu] = Dn;
                    ++cu;
                }
            } else if (sp + 8 <= 128) {
                const uint32_t k2 = T.b_key[Dn] << 3;
                for (int c = 0; c < 8; ++c) {
                    const int C = T.box_at[dense_off(G.level + 1) + k2 + c];
                    if (C >= 0) stk[sp++] = C;
                }
            }
        } else if (hs) {
            if (FILL) L.w_src[pw + cw] = Dn;
            ++cw;
        }
    }
}

// Deepest existing box over slot (qx, qy, qz) of level lq, searched from level lq - 1 up;
// its index if it is a leaf with sources, else -1.
__device__ __forceinline__ int coarse_leaf_src(const TreeDev &T, int lq, int qx, int qy, int qz) {
    for (int m = lq - 1; m >= 0; --m) {
        const int sh = lq - m;
        const int64_t sl = dense_off(m) + morton3(qx >> sh, qy >> sh, qz >> sh);
        const int Am = T.box_at[sl];
        if (Am >= 0) return (T.vsrc[sl] && T.b_leaf[Am]) ? Am : -1;
    }
    return -1;
}

// After the list counts and their scan (one CTA of 1024 threads): the closing offsets of the four
// lists (entry nboxes: the list's total), the V pairs' key offsets (exclusive scan of the per-key
// counts; entry nkeys: the number of pairs) and their tiles of VPAIR_TILE pairs per key (counts,
// exclusive offsets; entry nkeys: the number of tiles).  The key of every tile is written by the
// list fill, once the pair buffer has its size.
__global__ void __launch_bounds__(1024) k_lists_layout(ListDev L, PairsDev Pd, const int *__restrict__ nboxes_dev,
                                                       const int *__restrict__ totals, ReadBack R) {
    pdl_enter();
    // the host's read-backs, straight into its mapped buffer (every producer has completed)
    if (R.dst) {
        const int tid = threadIdx.x;
        if (tid < 3) R.dst[tid] = R.sel[tid];
        else if (tid >= 32 && tid < 64) R.dst[8 + tid - 32] = R.lvl[tid - 32];
        else if (tid >= 64 && tid < 112) R.dst[tid] = R.lvl[tid - 32];
        else if (tid >= 128 && tid < 133) R.dst[43 + tid - 128] = R.flag_tot[tid - 128];
        __threadfence_system();
    }
    __shared__ int wp[32], wt[32];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) {
        const int nb = *nboxes_dev;
        L.u_off[nb] = totals[0];
        L.v_off[nb] = totals[1];
        L.w_off[nb] = totals[2];
        L.x_off[nb] = totals[3];
    }
    const int per = (Pd.nkeys + 1023) / 1024;
    const int k0 = min(tid * per, Pd.nkeys), k1 = min(k0 + per, Pd.nkeys);
    int sp = 0, st = 0;
    for (int k = k0; k < k1; ++k) {
        const int c = Pd.cnt[k], t = (c + VPAIR_TILE - 1) / VPAIR_TILE;
        Pd.tile_cnt[k] = t;
        sp += c;
        st += t;
    }
    int ip = sp, it = st;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int a = __shfl_up_sync(0xffffffffu, ip, o), b = __shfl_up_sync(0xffffffffu, it, o);
        if (lane >= o) { ip += a; it += b; }
    }
    if (lane == 31) { wp[w] = ip; wt[w] = it; }
    __syncthreads();
    if (w == 0) {
        int a = wp[lane], b = wt[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int a2 = __shfl_up_sync(0xffffffffu, a, o), b2 = __shfl_up_sync(0xffffffffu, b, o);
            if (lane >= o) { a += a2; b += b2; }
        }
        wp[lane] = a;
        wt[lane] = b;
    }
    __syncthreads();
    int xp = (w ? wp[w - 1] : 0) + ip - sp, xt = (w ? wt[w - 1] : 0) + it - st;
    for (int k = k0; k < k1; ++k) {
        Pd.off[k] = xp;
        xp += Pd.cnt[k];
        Pd.tile_off[k] = xt;
        xt += Pd.tile_cnt[k];
    }
    if (tid == 1023) {
        Pd.off[Pd.nkeys] = wp[31];
        Pd.tile_off[Pd.nkeys] = wt[31];
        Pd.total_tiles[0] = wt[31];
        Pd.total_tiles[1] = wp[31];
    }
}

template <bool FILL>
__global__ void __launch_bounds__(256) k_lists_warp(TreeDev T, ListDev L, PairsDev Pd, int D) {
    pdl_enter();
    if (FILL) {
        // the key of every V-pair tile (k_lists_layout laid the tiles out)
        for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < Pd.nkeys; k += gridDim.x * blockDim.x) {
            const int x = Pd.tile_off[k], t1 = Pd.tile_cnt[k];
            for (int t = 0; t < t1; ++t) Pd.tile_key[x + t] = k;
        }
    }
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int wid = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)((gridDim.x * blockDim.x) >> 5);
    const int nh = *L.nheavy;
    for (int h = wid; h < nh; h += nw) {
        const int b = L.heavy[h];
        BoxGeom B = geom_of(T, b);
        const int l = B.level;
        int pU = 0, pV = 0, pW = 0, pX = 0;
        if (FILL) { pU = L.u_off[b]; pV = L.v_off[b]; pW = L.w_off[b]; pX = L.x_off[b]; }
        int nU = 0, nV = 0, nW = 0, nX = 0;
        // ---- U and W (B leaf): lane t < 27 takes slot t (z, then y, then x)
        if (T.b_leaf[b]) {
            const int n = 1 << l;
            const int qx = B.x + lane % 3 - 1, qy = B.y + (lane / 3) % 3 - 1, qz = B.z + lane / 9 - 1;
            const bool inr = lane < 27 && qx >= 0 && qy >= 0 && qz >= 0 && qx < n && qy < n && qz < n;
            int A = -1, mode = 0;          // 1 leaf colleague, 2 split colleague, 3 no box at this level
            if (inr) {
                const int64_t sl = dense_off(l) + morton3(qx, qy, qz);
                A = T.box_at[sl];
                if (A < 0) mode = 3;
                else if (T.vsrc[sl]) mode = T.b_leaf[A] ? 1 : 2;
            }
            int cu = mode == 1, cw = 0, coarse = -1;
            if (mode == 2) lists_descend<false>(T, L, B, D, A, 0, 0, cu, cw);
            if (mode == 3) coarse = coarse_leaf_src(T, l, qx, qy, qz);
            int eu = cu, ew = cw;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int a = __shfl_up_sync(0xffffffffu, eu, o), c = __shfl_up_sync(0xffffffffu, ew, o);
                if (lane >= o) { eu += a; ew += c; }
            }
            const int tu = __shfl_sync(0xffffffffu, eu, 31), tw = __shfl_sync(0xffffffffu, ew, 31);
            eu -= cu;
            ew -= cw;
            if (FILL) {
                if (mode == 1) L.u_src[pU + eu] = A;
                if (mode == 2) {
                    int du = 0, dw = 0;
                    lists_descend<true>(T, L, B, D, A, pU + eu, pW + ew, du, dw);
                }
            }
            // leaves covering missing slots: once each, in order of first appearance, after the rest
            const unsigned same = __match_any_sync(0xffffffffu, coarse);
            const bool rep = coarse >= 0 && (__ffs(same) - 1) == lane;
            const unsigned repm = __ballot_sync(0xffffffffu, rep);
            if (FILL && rep) L.u_src[pU + tu + __popc(repm & lt)] = coarse;
            nU = tu + __popc(repm);
            nW = tw;
        }
        // ---- X (leaves with sources adjacent to the parent, not to B), and whether any box
        // adjacent to the parent holds sources (else V is empty)
        bool parent_near_src = false;
        if (l >= 2) {
            const int n = 1 << (l - 1);
            const int qx = (B.x >> 1) + lane % 3 - 1, qy = (B.y >> 1) + (lane / 3) % 3 - 1, qz = (B.z >> 1) + lane / 9 - 1;
            const bool inr = lane < 27 && qx >= 0 && qy >= 0 && qz >= 0 && qx < n && qy < n && qz < n;
            int cand = -1;
            bool hs = false;
            if (inr) {
                const int64_t sl = dense_off(l - 1) + morton3(qx, qy, qz);
                const int Am = T.box_at[sl];
                if (Am >= 0) {
                    hs = T.vsrc[sl];
                    if (hs && T.b_leaf[Am]) cand = Am;
                } else {
                    cand = coarse_leaf_src(T, l - 1, qx, qy, qz);
                }
                if (cand >= 0 && adjacent(geom_of(T, cand), B, D)) cand = -1;
            }
            parent_near_src = __any_sync(0xffffffffu, hs);
            const unsigned same = __match_any_sync(0xffffffffu, cand);
            const bool rep = cand >= 0 && (__ffs(same) - 1) == lane;
            const unsigned repm = __ballot_sync(0xffffffffu, rep);
            if (FILL && rep) L.x_src[pX + __popc(repm & lt)] = cand;
            nX = __popc(repm);
        }
        // ---- V: the 6^3 candidates around the parent minus the 3^3 adjacent to B, 32 at a time
        if (l >= 2 && parent_near_src) {
            const int n = 1 << l;
            const int px = B.x & ~1, py = B.y & ~1, pz = B.z & ~1;
            const uint8_t *vs = T.vsrc + dense_off(l);
            const int *ba = T.box_at + dense_off(l);
#pragma unroll
            for (int k = 0; k < 7; ++k) {
                const int c = 32 * k + lane;
                const int qx = px - 2 + c % 6, qy = py - 2 + (c / 6) % 6, qz = pz - 2 + c / 36;
                const int ox = qx - B.x, oy = qy - B.y, oz = qz - B.z;
                uint32_t m = 0;
                bool hit = false;
                if (c < 216 && qx >= 0 && qy >= 0 && qz >= 0 && qx < n && qy < n && qz < n &&
                    !(abs(ox) <= 1 && abs(oy) <= 1 && abs(oz) <= 1)) {
                    m = morton3((uint32_t)qx, (uint32_t)qy, (uint32_t)qz);
                    hit = vs[m] != 0;
                }
                const unsigned hm = __ballot_sync(0xffffffffu, hit);
                if (hit) {
                    const int key = l * NSLOT + m2l_slot(ox, oy, oz);
                    if (FILL) {
                        const int pos = pV + nV + __popc(hm & lt);
                        const int A = ba[m];
                        L.v_src[pos] = A;
                        L.v_trg[pos] = b;
                        L.v_oc[pos] = (short)((ox + 3) + 7 * (oy + 3) + 49 * (oz + 3));
                        // the pair in its (level, offset) bucket, in any order within the bucket
                        const int q = Pd.off[key] + atomicAdd(Pd.cursor + key, 1);
                        Pd.trg[q] = b;
                        Pd.src[q] = A;
                    } else {
                        atomicAdd(Pd.cnt + key, 1);
                    }
                }
                nV += __popc(hm);
            }
        }
        if (!FILL && lane == 0) {
            L.u_cnt[b] = nU; L.v_cnt[b] = nV; L.w_cnt[b] = nW; L.x_cnt[b] = nX;
        }
    }
}

constexpr int LISTS_WARP_GRID = 152 * 8;

bool lists_count_launch(const TreeDev &T, const ListDev &L, const PairsDev &Pd, int cap, const int *nboxes_dev,
                        int D, int Lmax, int *scan_tmp, int *totals /* device [4] */, int *err, const ReadBack &R,
                        cudaStream_t st, bool zeroed) {
    const int nboxes = cap;   // counts and offsets span every slot; the ones past the last box stay 0
    if (nboxes <= 0) {
        cudaMemsetAsync(totals, 0, 4 * sizeof(int), st);
        return false;
    }
    if (!zeroed) cudaMemsetAsync(L.nheavy, 0, sizeof(int), st);
    launch_pdl(k_lists_classify, (nboxes + 255) / 256, 256, 0, st, T, L, cap, nboxes_dev);
    launch_pdl(k_lists_warp<false>, LISTS_WARP_GRID, 256, 0, st, T, L, Pd, D);
    ScanSet S{};
    S.in[0] = L.u_cnt; S.in[1] = L.v_cnt; S.in[2] = L.w_cnt; S.in[3] = L.x_cnt;
    S.out[0] = L.u_off; S.out[1] = L.v_off; S.out[2] = L.w_off; S.out[3] = L.x_off;
    for (int a = 0; a < 4; ++a) S.total[a] = totals + a;
    scan_exclusive_multi(S, 4, nboxes, scan_tmp, err, st, SCAN_WAIT_LIMIT, zeroed);
    launch_pdl(k_lists_layout, 1, 1024, 0, st, L, Pd, nboxes_dev, (const int *)totals, R);
    return R.dst != nullptr;
}

void lists_fill_launch(const TreeDev &T, const ListDev &L, const PairsDev &Pd, int nboxes, int D, int Lmax,
                       const int *totals, cudaStream_t st) {
    if (nboxes <= 0) return;
    (void)totals;
    launch_pdl(k_lists_warp<true>, LISTS_WARP_GRID, 256, 0, st, T, L, Pd, D);
}

}  // namespace sph
