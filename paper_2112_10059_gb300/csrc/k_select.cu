// Selection of sources and targets (paper Section 3: Eq. summationI, Eq. sourcepct,
// and the electric-field target rule of Section 5) as a GPU stream compaction
// that emits the selected cells directly in Morton order.
//
// Pass 1 (k_brick_stats, bricks of 16^3 cells): max q and max |E| over all cells (NaN
// ignored) and, per brick, the largest q, the smallest and largest |E| and whether an |E| is
// NaN.  A whole brick that those statistics decide (no source, and every cell or no cell a
// target) is emitted without reading it again.  Default: k_select_count (counts: decided
// bricks at once, the others read), k_scan2 (offsets), k_select_emit (points), no CTA waiting
// for another.  Alternatives: k_select_onepass does count, offsets and emit in one pass with a
// decoupled look-back across bricks (also the form without statistics); the two-pass form
// that follows (after k_grid_max, the maxima alone) is kept as a reference:
// Pass 2 (k_select_count): per 16^3 brick (a Morton-contiguous key range),
//         count selected sources / targets.
// Pass 3 (k_scan_bricks): exclusive scan of the brick counts.
// Pass 4 (k_select_emit): per brick, re-evaluate the rules, rank the cells in
//         Morton order inside the brick and write key, packed (i,j,k) and, for
//         sources, q (consumers scale it to I_h = source_scale * q * h^3).
// The rules compare in FP64: (double)q >= i_frac * (double)qmax.
#include <algorithm>

#include "sph_kernels.cuh"

namespace sph {

__device__ __forceinline__ unsigned f2ord(float f) {
    unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(unsigned u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__global__ void k_grid_max(const float *__restrict__ q, const float *__restrict__ e, int64_t n,
                           unsigned *__restrict__ out /* [2] ordered-uint maxima */) {
    pdl_enter();
    float mq = -INFINITY, me = -INFINITY;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // aligned float4 body (cudaMalloc'd inputs), four loads in flight per array and thread
    const int64_t n4 = ((reinterpret_cast<uintptr_t>(q ? q : e) & 15) == 0 &&
                        (!q || !e || (reinterpret_cast<uintptr_t>(e) & 15) == 0)) ? n / 4 : 0;
    const float4 *q4 = reinterpret_cast<const float4 *>(q), *e4 = reinterpret_cast<const float4 *>(e);
    auto fold = [](float m, float4 v) {
        if (v.x == v.x) m = fmaxf(m, v.x);
        if (v.y == v.y) m = fmaxf(m, v.y);
        if (v.z == v.z) m = fmaxf(m, v.z);
        if (v.w == v.w) m = fmaxf(m, v.w);
        return m;
    };
    int64_t i = tid;
    for (; i + 3 * stride < n4; i += 4 * stride) {
        float4 a[4], b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (q) a[u] = __ldg(q4 + i + u * stride);
            if (e) b[u] = __ldg(e4 + i + u * stride);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (q) mq = fold(mq, a[u]);
            if (e) me = fold(me, b[u]);
        }
    }
    for (; i < n4; i += stride) {
        if (q) mq = fold(mq, __ldg(q4 + i));
        if (e) me = fold(me, __ldg(e4 + i));
    }
    for (int64_t j = 4 * n4 + tid; j < n; j += stride) {
        if (q) { float v = __ldg(q + j); if (v == v) mq = fmaxf(mq, v); }
        if (e) { float v = __ldg(e + j); if (v == v) me = fmaxf(me, v); }
    }
    for (int o = 16; o > 0; o >>= 1) {
        mq = fmaxf(mq, __shfl_xor_sync(0xffffffffu, mq, o));
        me = fmaxf(me, __shfl_xor_sync(0xffffffffu, me, o));
    }
    __shared__ float sq[32], se[32];
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { sq[w] = mq; se[w] = me; }
    __syncthreads();
    if (w == 0) {
        int nw = blockDim.x >> 5;
        mq = l < nw ? sq[l] : -INFINITY;
        me = l < nw ? se[l] : -INFINITY;
        for (int o = 16; o > 0; o >>= 1) {
            mq = fmaxf(mq, __shfl_xor_sync(0xffffffffu, mq, o));
            me = fmaxf(me, __shfl_xor_sync(0xffffffffu, me, o));
        }
        if (l == 0) {
            if (q) atomicMax(out + 0, f2ord(mq));
            if (e) atomicMax(out + 1, f2ord(me));
        }
    }
}

struct SelRule {
    int nx, ny, nz;
    int brick_edge_log2;   // brick edge = 2^b (<= 16)
    int src_all;           // i_frac == 0
    double i_frac;
    int trg_mode;          // 0 all, 1 |E| rule, 2 mask
    double e_frac, e_app;
};

// Evaluate both rules for cell (x,y,z); returns bit0 = source, bit1 = target.
__device__ __forceinline__ int sel_bits(const SelRule &r, const float *q, const float *e,
                                        const uint8_t *mask, int x, int y, int z,
                                        double thr_q, double thr_e, bool qpos, float &qv) {
    if (x >= r.nx || y >= r.ny || z >= r.nz) return 0;
    int64_t lin = (int64_t)x + (int64_t)r.nx * ((int64_t)y + (int64_t)r.ny * z);
    qv = __ldg(q + lin);
    int b = 0;
    if (r.src_all) b |= 1;
    else if (qpos && (double)qv >= thr_q) b |= 1;
    if (r.trg_mode == 0) b |= 2;
    else if (r.trg_mode == 1) { float ev = __ldg(e + lin); if ((double)ev >= thr_e) b |= 2; }
    else { if (__ldg(mask + lin)) b |= 2; }
    return b;
}

__device__ __forceinline__ void thresholds(const SelRule &r, const unsigned *maxes, double &thr_q,
                                           double &thr_e, bool &qpos) {
    float qmax = ord2f(maxes[0]);
    float emax = ord2f(maxes[1]);
    qpos = qmax > 0.0f;
    thr_q = r.i_frac * (double)qmax;
    thr_e = r.e_app + r.e_frac * ((double)emax - r.e_app);
}

// One CTA per brick; blockDim.x = 512; brick of up to 16^3 cells.  The brick is read
// row by row (coalesced) into shared memory at local Morton positions; then thread t
// owns local keys 8t .. 8t+7, so a block scan in thread order is a scan in Morton order.
template <bool EMIT>
__global__ void __launch_bounds__(512) k_select_brick(
        SelRule r, const float *__restrict__ q, const float *__restrict__ e,
        const uint8_t *__restrict__ mask, const unsigned *__restrict__ maxes,
        int *__restrict__ cnt_s, int *__restrict__ cnt_t,            // [nbricks] (count pass)
        const int *__restrict__ off_s, const int *__restrict__ off_t,// [nbricks] (emit pass)
        uint32_t *__restrict__ src_key, uint32_t *__restrict__ src_pc, float *__restrict__ src_q,
        uint32_t *__restrict__ trg_key, uint32_t *__restrict__ trg_pc, uint8_t *__restrict__ tmask) {
    pdl_enter();
    const int b = r.brick_edge_log2;
    const int ncell = 1 << (3 * b);
    const uint32_t brick = blockIdx.x;
    uint32_t bx, by, bz;
    demorton3(brick, bx, by, bz);
    const int x0 = bx << b, y0 = by << b, z0 = bz << b;
    double thr_q, thr_e;
    bool qpos;
    thresholds(r, maxes, thr_q, thr_e, qpos);

    // stage the brick: coalesced loads in linear (x fastest) order, rule bits and q
    // stored at the cell's local Morton index
    __shared__ uint8_t s_bits[4096];
    __shared__ float s_q[4096];
    const int edge = 1 << b;
    for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
        int lx = c & (edge - 1), ly = (c >> b) & (edge - 1), lz = c >> (2 * b);
        uint32_t lk = morton3((uint32_t)lx, (uint32_t)ly, (uint32_t)lz);
        float qv = 0.0f;
        int bits = sel_bits(r, q, e, mask, x0 + lx, y0 + ly, z0 + lz, thr_q, thr_e, qpos, qv);
        s_bits[lk] = (uint8_t)bits;
        s_q[lk] = qv;
        if (EMIT && tmask && x0 + lx < r.nx && y0 + ly < r.ny && z0 + lz < r.nz)
            tmask[(int64_t)(x0 + lx) + (int64_t)r.nx * ((int64_t)(y0 + ly) + (int64_t)r.ny * (z0 + lz))] =
                (uint8_t)(bits >> 1);
    }
    __syncthreads();
    int my_bits[8];
    float my_q[8];
    int ns = 0, nt = 0;
    const int per = (ncell + blockDim.x - 1) / blockDim.x;   // 8 for a 16^3 brick, fewer for small grids
    for (int u = 0; u < per; ++u) {
        int lk = threadIdx.x * per + u;
        my_bits[u] = lk < ncell ? s_bits[lk] : 0;
        my_q[u] = lk < ncell ? s_q[lk] : 0.0f;
        ns += my_bits[u] & 1;
        nt += (my_bits[u] >> 1) & 1;
    }
    // block exclusive scan of (ns, nt) in thread order
    __shared__ int ws[16], wt[16];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int is = ns, it = nt;
    for (int o = 1; o < 32; o <<= 1) {
        int a = __shfl_up_sync(0xffffffffu, is, o);
        int c = __shfl_up_sync(0xffffffffu, it, o);
        if (lane >= o) { is += a; it += c; }
    }
    if (lane == 31) { ws[w] = is; wt[w] = it; }
    __syncthreads();
    if (w == 0) {
        int nw = blockDim.x >> 5;
        int a = lane < nw ? ws[lane] : 0;
        int c = lane < nw ? wt[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int a2 = __shfl_up_sync(0xffffffffu, a, o);
            int c2 = __shfl_up_sync(0xffffffffu, c, o);
            if (lane >= o) { a += a2; c += c2; }
        }
        if (lane < 16) { ws[lane] = a; wt[lane] = c; }
    }
    __syncthreads();
    int base_s = (w > 0 ? ws[w - 1] : 0) + is - ns;
    int base_t = (w > 0 ? wt[w - 1] : 0) + it - nt;
    if (!EMIT) {
        if (threadIdx.x == blockDim.x - 1) {
            cnt_s[brick] = base_s + ns;
            cnt_t[brick] = base_t + nt;
        }
        return;
    }
    int ps = off_s[brick] + base_s, pt = off_t[brick] + base_t;
    for (int u = 0; u < per; ++u) {
        int lk = threadIdx.x * per + u;
        if (!my_bits[u]) continue;
        uint32_t lx, ly, lz;
        demorton3((uint32_t)lk, lx, ly, lz);
        uint32_t key = (brick << (3 * b)) | (uint32_t)lk;
        uint32_t pc = pack_ijk(x0 + lx, y0 + ly, z0 + lz);
        if (my_bits[u] & 1) {
            src_key[ps] = key;
            src_pc[ps] = pc;
            src_q[ps] = my_q[u];
            ++ps;
        }
        if (my_bits[u] & 2) {
            trg_key[pt] = key;
            if (trg_pc) trg_pc[pt] = pc;
            ++pt;
        }
    }
}

// Exclusive scan of two int arrays of length n by one CTA of 1024 threads; totals
// written to tot[0], tot[1].
__global__ void __launch_bounds__(1024) k_scan2(const int *__restrict__ a, const int *__restrict__ b,
                                                int *__restrict__ oa, int *__restrict__ ob, int n,
                                                int *__restrict__ tot) {
    pdl_enter();
    __shared__ int sa[1024], sb[1024];
    int per = (n + 1023) / 1024;
    int beg = threadIdx.x * per, end = min(n, beg + per);
    int ra = 0, rb = 0;
    for (int i = beg; i < end; ++i) { ra += a[i]; rb += b[i]; }
    sa[threadIdx.x] = ra;
    sb[threadIdx.x] = rb;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        int va = threadIdx.x >= o ? sa[threadIdx.x - o] : 0;
        int vb = threadIdx.x >= o ? sb[threadIdx.x - o] : 0;
        __syncthreads();
        sa[threadIdx.x] += va;
        sb[threadIdx.x] += vb;
        __syncthreads();
    }
    int xa = sa[threadIdx.x] - ra, xb = sb[threadIdx.x] - rb;
    for (int i = beg; i < end; ++i) {
        oa[i] = xa; xa += a[i];
        ob[i] = xb; xb += b[i];
    }
    if (threadIdx.x == 1023) { tot[0] = sa[1023]; tot[1] = sb[1023]; }
}

// ---------------------------------------------------------------- one-pass selection
// Exact FP32 equivalent of the FP64 rule (double)v >= thr: the smallest float f with
// (double)f >= thr, so that v >= f decides every finite v exactly as the FP64 compare.
__device__ __forceinline__ float ge_threshold_f32(double thr) {
    float f = __double2float_rd(thr);          // (double)f <= thr
    if ((double)f < thr) f = nextafterf(f, INFINITY);
    return f;
}

// Look-back state of one brick: status in bits 62-63 (0 none, 1 own counts, 2 inclusive
// prefix), source count in bits 31-61, target count in bits 0-30.
__device__ __forceinline__ unsigned long long pack_state(unsigned st, unsigned ns, unsigned nt) {
    return ((unsigned long long)st << 62) | ((unsigned long long)ns << 31) | (unsigned long long)nt;
}

// Per brick of 16^3 cells (one CTA of 256 threads): bstat[brick] = (max q, min |E|, max |E|,
// 1 if an |E| is NaN else 0) over the brick's cells inside the grid, NaN values left out of the
// extremes (q or e nullptr: that part is not computed); the brick's maxima go into `out` (ordered
// uints, as k_grid_max).  Four threads per row of 16 cells, each one 16-byte load per array and
// row, four rows per thread: all eight loads in flight at once.
constexpr int STAT_T = 256;
__global__ void __launch_bounds__(STAT_T) k_brick_stats(SelRule r, const float *__restrict__ q,
                                                        const float *__restrict__ e, float4 *__restrict__ bstat,
                                                        unsigned *__restrict__ out) {
    pdl_enter();
    const uint32_t brick = blockIdx.x;
    uint32_t bx, by, bz;
    demorton3(brick, bx, by, bz);
    const int x0 = (int)bx << 4, y0 = (int)by << 4, z0 = (int)bz << 4;
    const int tid = threadIdx.x, seg = tid & 3;
    float mq = -INFINITY, lo = INFINITY, hi = -INFINITY;
    bool nan_e = false;
    auto take = [&](float vq, float ve, bool in) {
        if (!in) return;
        if (q && vq == vq) mq = fmaxf(mq, vq);
        if (e) {
            if (ve == ve) {
                lo = fminf(lo, ve);
                hi = fmaxf(hi, ve);
            } else {
                nan_e = true;
            }
        }
    };
    const bool vec = x0 + 16 <= r.nx && (r.nx & 3) == 0 && (reinterpret_cast<uintptr_t>(q) & 15) == 0 &&
                     (reinterpret_cast<uintptr_t>(e) & 15) == 0;
    if (vec) {
        float4 a[4], c[4];
        bool in[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int row = (tid >> 2) + 64 * k, y = y0 + (row & 15), z = z0 + (row >> 4);
            in[k] = y < r.ny && z < r.nz;
            const int64_t lin = (int64_t)x0 + 4 * seg + (int64_t)r.nx * ((int64_t)y + (int64_t)r.ny * z);
            a[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            c[k] = a[k];
            if (in[k] && q) a[k] = __ldg(reinterpret_cast<const float4 *>(q + lin));
            if (in[k] && e) c[k] = __ldg(reinterpret_cast<const float4 *>(e + lin));
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            take(a[k].x, c[k].x, in[k]);
            take(a[k].y, c[k].y, in[k]);
            take(a[k].z, c[k].z, in[k]);
            take(a[k].w, c[k].w, in[k]);
        }
    } else {
        for (int i = tid; i < 4096; i += STAT_T) {
            const int x = x0 + (i & 15), y = y0 + ((i >> 4) & 15), z = z0 + (i >> 8);
            const bool in = x < r.nx && y < r.ny && z < r.nz;
            const int64_t lin = in ? (int64_t)x + (int64_t)r.nx * ((int64_t)y + (int64_t)r.ny * z) : 0;
            take(in && q ? __ldg(q + lin) : 0.f, in && e ? __ldg(e + lin) : 0.f, in);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mq = fmaxf(mq, __shfl_xor_sync(0xffffffffu, mq, o));
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    nan_e = __any_sync(0xffffffffu, nan_e);
    __shared__ float s_mq[STAT_T / 32], s_lo[STAT_T / 32], s_hi[STAT_T / 32];
    __shared__ int s_nan[STAT_T / 32];
    const int w = tid >> 5, lane = tid & 31;
    if (lane == 0) {
        s_mq[w] = mq; s_lo[w] = lo; s_hi[w] = hi; s_nan[w] = nan_e;
    }
    __syncthreads();
    if (tid == 0) {
        for (int k = 1; k < STAT_T / 32; ++k) {
            mq = fmaxf(mq, s_mq[k]);
            lo = fminf(lo, s_lo[k]);
            hi = fmaxf(hi, s_hi[k]);
            nan_e = nan_e || s_nan[k];
        }
        bstat[brick] = make_float4(mq, lo, hi, nan_e ? 1.f : 0.f);
        if (q) atomicMax(out + 0, f2ord(mq));
        if (e) atomicMax(out + 1, f2ord(hi));
    }
}

// Status of brick `brick` from its statistics (st, as k_brick_stats): 1 if no cell is a source
// and every cell a target, 2 if no cell is selected at all, 0 if the cells must be read.  Only a
// brick of 16^3 cells wholly inside the grid is decided this way; the comparisons are those of
// the per-cell rules (v >= threshold in FP32, NaN never selected).
__device__ __forceinline__ int brick_mode(const SelRule &r, uint32_t brick, float4 st, float thr_q, float thr_e,
                                          bool qpos) {
    uint32_t bx, by, bz;
    demorton3(brick, bx, by, bz);
    if (((int)bx << 4) + 16 > r.nx || ((int)by << 4) + 16 > r.ny || ((int)bz << 4) + 16 > r.nz) return 0;
    if (r.src_all || (qpos && st.x >= thr_q)) return 0;       // a source in the brick
    if (r.trg_mode == 0) return 1;
    if (r.trg_mode != 1) return 0;
    if (st.w == 0.f && st.y >= thr_e) return 1;               // every |E| at or above the threshold
    if (!(st.z >= thr_e)) return 2;                           // none
    return 0;
}

// Decoupled look-back by the whole block: 512 predecessor states per round (every brick in
// flight is within a round or two); the nearest inclusive state ends the walk.  Adds the
// preceding bricks' counts into pre_s / pre_t; returns false (uniformly) if a round gave up
// after wait_limit polls.  rs, rt: [blockDim.x / 32] shared scratch; s_stop: shared int.
__device__ __forceinline__ bool look_back(const unsigned long long *state, int brick, unsigned wait_limit,
                                          unsigned &pre_s, unsigned &pre_t, unsigned *rs, unsigned *rt,
                                          int *s_stop) {
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int j = brick - 1; j >= 0; j -= (int)blockDim.x) {
        const int idx = j - tid;
        unsigned long long v = 0;
        unsigned stt = 2;                          // before brick 0: an inclusive zero
        bool ready = false;
        for (unsigned k = 0; k < wait_limit; ++k) {
            if (idx >= 0) {
                v = *((volatile const unsigned long long *)(state + idx));
                stt = (unsigned)(v >> 62);
            }
            if (__syncthreads_and(stt != 0)) {
                ready = true;
                break;
            }
            __nanosleep(64);
        }
        if (!ready) return false;                  // uniform: every thread saw the same vote
        if (tid == 0) *s_stop = (int)blockDim.x;
        __syncthreads();
        if (stt == 2u) atomicMin(s_stop, tid);
        __syncthreads();
        const int stop = *s_stop;
        unsigned cs = (tid <= stop && idx >= 0) ? (unsigned)((v >> 31) & 0x7FFFFFFFu) : 0u;
        unsigned ct = (tid <= stop && idx >= 0) ? (unsigned)(v & 0x7FFFFFFFu) : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            cs += __shfl_xor_sync(0xffffffffu, cs, o);
            ct += __shfl_xor_sync(0xffffffffu, ct, o);
        }
        if (lane == 0) {
            rs[w] = cs;
            rt[w] = ct;
        }
        __syncthreads();
        unsigned sum_s = 0, sum_t = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            sum_s += rs[k];
            sum_t += rt[k];
        }
        pre_s += sum_s;
        pre_t += sum_t;
        __syncthreads();                           // rs / rt / s_stop reused by the next round
        if (stop < (int)blockDim.x) break;
    }
    return true;
}

// After the look-back (thread 0): the brick's inclusive state (and the gave-up flag), and the
// totals from the last brick.
__device__ __forceinline__ void publish(unsigned long long *state, int brick, int nbr, bool failed, unsigned pre_s,
                                        unsigned pre_t, unsigned agg_s, unsigned agg_t, int *totals) {
    if (brick > 0) {
        if (failed) {
            atomicOr(totals + 2, 1);
            __threadfence();                       // the flag is visible before the state it taints
        }
        atomicExch(state + brick, pack_state(2u, pre_s + agg_s, pre_t + agg_t));
    }
    if (brick == nbr - 1) {
        __threadfence();
        bool bad = atomicOr(totals + 2, 0) != 0;
        totals[0] = bad ? -1 : (int)(pre_s + agg_s);
        totals[1] = bad ? -1 : (int)(pre_t + agg_t);
    }
}


// ---------------------------------------------------------------- parts shared by the brick kernels
// (blocks of SEL_T = 512 threads, bricks of up to 16^3 cells)
constexpr int SEL_T = 512;

// Thread `tid`'s 2x2x2 Morton micro-cube of the brick at (x0, y0, z0): the brick-local Morton
// keys 8 tid .. 8 tid + 7, so the 8 cells follow from one decode.  Both rules are evaluated for
// each cell (bit 0 source, bit 1 target; q kept for the sources); all loads are issued before
// any is used (a warp's cells form an 8x8x4 block, whose rows the L1 serves sector by sector).
// Cell u sits at (mx + (u & 1), my + ((u >> 1) & 1), mz + (u >> 2)): the pairs (u, u + 1), u
// even, are x-neighbours at an even x, read as one float2 when the row pitch and the arrays
// allow it.  The target mask is written if `tmask` (two cells per 2-byte store where aligned).
__device__ __forceinline__ void cube_rules(const SelRule &r, const float *__restrict__ q, const float *__restrict__ e,
                                           const uint8_t *__restrict__ mask, int tid, int x0, int y0, int z0,
                                           int ncell, float thr_q, float thr_e, bool qpos,
                                           uint8_t *__restrict__ tmask, int (&my_bits)[8], float (&my_q)[8],
                                           uint32_t &mx, uint32_t &my, uint32_t &mz) {
    demorton3((uint32_t)(8 * tid), mx, my, mz);
    const bool vec2 = (r.nx & 1) == 0 && (reinterpret_cast<uintptr_t>(q) & 7) == 0 &&
                      (r.trg_mode != 1 || (reinterpret_cast<uintptr_t>(e) & 7) == 0);
    float ev[8];
    uint32_t lin[8];
    bool in[8];
#pragma unroll
    for (int v2 = 0; v2 < 4; ++v2) {
        const int u0 = 2 * v2;
        const int x = x0 + (int)mx, y = y0 + (int)my + (v2 & 1), z = z0 + (int)mz + (v2 >> 1);
        const bool row = 8 * tid + u0 < ncell && y < r.ny && z < r.nz;
        in[u0] = row && x < r.nx;
        in[u0 + 1] = row && x + 1 < r.nx;
        const uint32_t l0 = row ? (uint32_t)x + (uint32_t)r.nx * ((uint32_t)y + (uint32_t)r.ny * (uint32_t)z) : 0u;
        lin[u0] = l0;
        lin[u0 + 1] = l0 + 1;
        if (vec2 && in[u0 + 1] && r.trg_mode != 2) {
            const float2 a = __ldg(reinterpret_cast<const float2 *>(q + l0));
            my_q[u0] = a.x;
            my_q[u0 + 1] = a.y;
            float2 c = make_float2(0.f, 0.f);
            if (r.trg_mode == 1) c = __ldg(reinterpret_cast<const float2 *>(e + l0));
            ev[u0] = c.x;
            ev[u0 + 1] = c.y;
        } else {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int u = u0 + h;
                my_q[u] = in[u] ? __ldg(q + lin[u]) : 0.f;
                ev[u] = (in[u] && r.trg_mode == 1) ? __ldg(e + lin[u]) : 0.f;
                if (in[u] && r.trg_mode == 2) ev[u] = __ldg(mask + lin[u]) ? 1.f : 0.f;
            }
        }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        int bits = 0;
        if (in[u]) {
            if (r.src_all || (qpos && my_q[u] >= thr_q)) bits |= 1;
            if (r.trg_mode == 0) bits |= 2;
            else if (r.trg_mode == 1) { if (ev[u] >= thr_e) bits |= 2; }
            else if (ev[u] != 0.f) bits |= 2;
        }
        my_bits[u] = bits;
    }
    if (tmask) {
#pragma unroll
        for (int v2 = 0; v2 < 4; ++v2) {
            const int u0 = 2 * v2;
            if (vec2 && in[u0 + 1]) {      // even index: one 2-byte store
                *reinterpret_cast<uint16_t *>(tmask + lin[u0]) =
                    (uint16_t)((my_bits[u0] >> 1) | ((my_bits[u0 + 1] >> 1) << 8));
            } else {
                if (in[u0]) tmask[lin[u0]] = (uint8_t)(my_bits[u0] >> 1);
                if (in[u0 + 1]) tmask[lin[u0 + 1]] = (uint8_t)(my_bits[u0 + 1] >> 1);
            }
        }
    }
}

// Block exclusive scan of (ns, nt) in thread order; ws, wt: [16] shared.  Gives this thread's
// exclusive offsets and the block's totals (ends with a barrier; ws / wt stay readable until
// the caller's next barrier).
__device__ __forceinline__ void block_scan2(int ns, int nt, int *ws, int *wt, int &base_s, int &base_t,
                                            unsigned &agg_s, unsigned &agg_t) {
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int is = ns, it = nt;
    for (int o = 1; o < 32; o <<= 1) {
        int a = __shfl_up_sync(0xffffffffu, is, o);
        int c = __shfl_up_sync(0xffffffffu, it, o);
        if (lane >= o) { is += a; it += c; }
    }
    if (lane == 31) { ws[w] = is; wt[w] = it; }
    __syncthreads();
    if (w == 0) {
        int nw = blockDim.x >> 5;
        int a = lane < nw ? ws[lane] : 0;
        int c = lane < nw ? wt[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int a2 = __shfl_up_sync(0xffffffffu, a, o);
            int c2 = __shfl_up_sync(0xffffffffu, c, o);
            if (lane >= o) { a += a2; c += c2; }
        }
        if (lane < 16) { ws[lane] = a; wt[lane] = c; }
    }
    __syncthreads();
    base_s = (w > 0 ? ws[w - 1] : 0) + is - ns;
    base_t = (w > 0 ? wt[w - 1] : 0) + it - nt;
    agg_s = (unsigned)ws[(blockDim.x >> 5) - 1];
    agg_t = (unsigned)wt[(blockDim.x >> 5) - 1];
}

// The micro-cube's selected cells written out: sources (few) straight to src_* from index ps;
// targets staged at their brick-local rank j (slot j + j / 32: a thread's consecutive ranks, 8
// apart from its neighbours', fall in distinct banks), then written by consecutive threads to
// trg_key[pt0 ..] (and trg_pc).  Ends after a barrier that follows the staging.
__device__ __forceinline__ void cube_emit(uint32_t brick, int b, int tid, int x0, int y0, int z0, uint32_t mx,
                                          uint32_t my, uint32_t mz, const int (&my_bits)[8], const float (&my_q)[8],
                                          int ps, int lt, unsigned pt0, unsigned agg_t, uint32_t *st_key,
                                          uint32_t *st_pc, uint32_t *__restrict__ src_key,
                                          uint32_t *__restrict__ src_pc, float *__restrict__ src_q,
                                          uint32_t *__restrict__ trg_key, uint32_t *__restrict__ trg_pc) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int lk = 8 * tid + u;
        if (!my_bits[u]) continue;
        const uint32_t key = (brick << (3 * b)) | (uint32_t)lk;
        const uint32_t pc = pack_ijk(x0 + mx + (u & 1), y0 + my + ((u >> 1) & 1), z0 + mz + (u >> 2));
        if (my_bits[u] & 1) {
            src_key[ps] = key;
            src_pc[ps] = pc;
            src_q[ps] = my_q[u];
            ++ps;
        }
        if (my_bits[u] & 2) {
            st_key[lt + (lt >> 5)] = key;
            if (trg_pc) st_pc[lt + (lt >> 5)] = pc;
            ++lt;
        }
    }
    __syncthreads();
    for (int i = tid; i < (int)agg_t; i += blockDim.x) {
        trg_key[pt0 + i] = st_key[i + (i >> 5)];
        if (trg_pc) trg_pc[pt0 + i] = st_pc[i + (i >> 5)];
    }
}

// A brick of 16^3 cells decided by its statistics (mode 1: every cell a target, mode 2: none;
// no source either way): its target mask, and for mode 1 its 4096 targets from trg_key[pt0]
// in Morton order (keys brick << 12 | i).
__device__ __forceinline__ void brick_emit_decided(const SelRule &r, uint32_t brick, int mode, int tid, int x0,
                                                   int y0, int z0, unsigned pt0, uint32_t *__restrict__ trg_key,
                                                   uint32_t *__restrict__ trg_pc, uint8_t *__restrict__ tmask) {
    if (tmask) {
        const uint8_t m = mode == 1 ? 1 : 0;
        if ((r.nx & 15) == 0 && (reinterpret_cast<uintptr_t>(tmask) & 15) == 0) {
            for (int row = tid; row < 256; row += blockDim.x) {   // one 16-byte store per row
                const int64_t o = (int64_t)x0 + (int64_t)r.nx * ((int64_t)(y0 + (row & 15)) +
                                                                 (int64_t)r.ny * (z0 + (row >> 4)));
                const uint32_t m4 = m * 0x01010101u;
                *reinterpret_cast<uint4 *>(tmask + o) = make_uint4(m4, m4, m4, m4);
            }
        } else {
            for (int i = tid; i < 4096; i += blockDim.x)
                tmask[(int64_t)(x0 + (i & 15)) +
                      (int64_t)r.nx * ((int64_t)(y0 + ((i >> 4) & 15)) + (int64_t)r.ny * (z0 + (i >> 8)))] = m;
        }
    }
    if (mode != 1) return;
    for (int i = tid; i < 4096; i += blockDim.x) {
        trg_key[pt0 + i] = (brick << 12) | (uint32_t)i;
        if (trg_pc) {
            uint32_t lx, ly, lz;
            demorton3((uint32_t)i, lx, ly, lz);
            trg_pc[pt0 + i] = pack_ijk(x0 + lx, y0 + ly, z0 + lz);
        }
    }
}

// Thresholds of both rules in FP32 (thread 0), for the whole block.
__device__ __forceinline__ void block_thresholds(const SelRule &r, const unsigned *maxes, float *s_thr_q,
                                                 float *s_thr_e, int *s_qpos) {
    double thr_q, thr_e;
    bool qpos;
    thresholds(r, maxes, thr_q, thr_e, qpos);
    *s_thr_q = ge_threshold_f32(thr_q);
    *s_thr_e = ge_threshold_f32(thr_e);
    *s_qpos = qpos;
}

// ---------------------------------------------------------------- one pass with look-back
// Each CTA takes the next brick in dispatch order (ticket), reads it, evaluates both rules,
// ranks its cells in Morton order, finds its output offset by decoupled look-back over the
// preceding bricks, and writes its points (a brick decided by its statistics: counts known,
// nothing read).
__global__ void __launch_bounds__(SEL_T) k_select_onepass(
        SelRule r, const float *__restrict__ q, const float *__restrict__ e, const uint8_t *__restrict__ mask,
        const unsigned *__restrict__ maxes, unsigned long long *__restrict__ state, unsigned *__restrict__ ticket,
        int nbr, int *__restrict__ totals, uint32_t *__restrict__ src_key, uint32_t *__restrict__ src_pc,
        float *__restrict__ src_q, uint32_t *__restrict__ trg_key, uint32_t *__restrict__ trg_pc,
        uint8_t *__restrict__ tmask, unsigned wait_limit, const float4 *__restrict__ bstat) {
    pdl_enter();
    __shared__ int s_brick, s_mode;
    __shared__ float s_thr_q, s_thr_e;
    __shared__ int s_qpos;
    __shared__ int ws[16], wt[16];
    __shared__ unsigned rs[16], rt[16];
    __shared__ int s_stop;
    __shared__ uint32_t st_key[4096 + 128], st_pc[4096 + 128];
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_brick = (int)atomicAdd(ticket, 1u);
        block_thresholds(r, maxes, &s_thr_q, &s_thr_e, &s_qpos);
        s_mode = bstat ? brick_mode(r, (uint32_t)s_brick, bstat[s_brick], s_thr_q, s_thr_e, s_qpos) : 0;
    }
    __syncthreads();
    const int brick = s_brick;
    const int b = r.brick_edge_log2;
    const int ncell = 1 << (3 * b);
    uint32_t bx, by, bz;
    demorton3((uint32_t)brick, bx, by, bz);
    const int x0 = bx << b, y0 = by << b, z0 = bz << b;
    if (s_mode != 0) {
        const unsigned agg_t = s_mode == 1 ? (unsigned)ncell : 0u;
        if (tid == 0) atomicExch(state + brick, pack_state(brick == 0 ? 2u : 1u, 0u, agg_t));
        unsigned pre_s = 0, pre_t = 0;
        const bool ok = look_back(state, brick, wait_limit, pre_s, pre_t, rs, rt, &s_stop);
        if (tid == 0) publish(state, brick, nbr, !ok, pre_s, pre_t, 0u, agg_t, totals);
        brick_emit_decided(r, (uint32_t)brick, s_mode, tid, x0, y0, z0, pre_t, trg_key, trg_pc, tmask);
        return;
    }
    int my_bits[8];
    float my_q[8];
    uint32_t mx, my, mz;
    cube_rules(r, q, e, mask, tid, x0, y0, z0, ncell, s_thr_q, s_thr_e, s_qpos, tmask, my_bits, my_q, mx, my, mz);
    int ns = 0, nt = 0;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        ns += my_bits[u] & 1;
        nt += (my_bits[u] >> 1) & 1;
    }
    int base_s, base_t;
    unsigned agg_s, agg_t;
    block_scan2(ns, nt, ws, wt, base_s, base_t, agg_s, agg_t);
    if (tid == 0) atomicExch(state + brick, pack_state(brick == 0 ? 2u : 1u, agg_s, agg_t));
    unsigned pre_s = 0, pre_t = 0;
    const bool ok = look_back(state, brick, wait_limit, pre_s, pre_t, rs, rt, &s_stop);
    if (tid == 0) publish(state, brick, nbr, !ok, pre_s, pre_t, agg_s, agg_t, totals);
    cube_emit((uint32_t)brick, b, tid, x0, y0, z0, mx, my, mz, my_bits, my_q, (int)pre_s + base_s, base_t, pre_t,
              agg_t, st_key, st_pc, src_key, src_pc, src_q, trg_key, trg_pc);
}

// ---------------------------------------------------------------- count, scan, emit (default)
// With per-brick statistics most bricks are decided without a read, and the selection runs as
// a count pass, the scan of the per-brick counts (k_scan2) and an emit pass, none of whose CTAs
// waits for another.  Both passes are persistent: CTA c takes the bricks c, c + gridDim.x, ...,
// SEL_T of them at a time (their modes found in parallel, one thread per brick); only the
// undecided ones are read (in both passes).

// counts of every brick: cnt_s / cnt_t [nbr]
__global__ void __launch_bounds__(SEL_T) k_select_count(SelRule r, const float *__restrict__ q,
                                                        const float *__restrict__ e, const uint8_t *__restrict__ mask,
                                                        const unsigned *__restrict__ maxes,
                                                        const float4 *__restrict__ bstat, int nbr,
                                                        int *__restrict__ cnt_s, int *__restrict__ cnt_t) {
    pdl_enter();
    __shared__ float s_thr_q, s_thr_e;
    __shared__ int s_qpos;
    __shared__ int s_und[SEL_T], s_nund;
    __shared__ int ws[16], wt[16];
    const int tid = threadIdx.x;
    if (tid == 0) {
        block_thresholds(r, maxes, &s_thr_q, &s_thr_e, &s_qpos);
        s_nund = 0;
    }
    __syncthreads();
    const int b = r.brick_edge_log2;
    const int ncell = 1 << (3 * b);
    for (int k0 = 0; blockIdx.x + (int64_t)k0 * gridDim.x < nbr; k0 += SEL_T) {
        const int64_t bk = blockIdx.x + (int64_t)(k0 + tid) * gridDim.x;
        if (bk < nbr) {
            const int m = brick_mode(r, (uint32_t)bk, bstat[bk], s_thr_q, s_thr_e, s_qpos);
            if (m != 0) {
                cnt_s[bk] = 0;
                cnt_t[bk] = m == 1 ? ncell : 0;
            } else {
                s_und[atomicAdd(&s_nund, 1)] = (int)bk;
            }
        }
        __syncthreads();
        const int nu = s_nund;
        for (int i = 0; i < nu; ++i) {
            const int brick = s_und[i];
            uint32_t bx, by, bz;
            demorton3((uint32_t)brick, bx, by, bz);
            int my_bits[8];
            float my_q[8];
            uint32_t mx, my, mz;
            cube_rules(r, q, e, mask, tid, bx << b, by << b, bz << b, ncell, s_thr_q, s_thr_e, s_qpos, nullptr,
                       my_bits, my_q, mx, my, mz);
            int ns = 0, nt = 0;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                ns += my_bits[u] & 1;
                nt += (my_bits[u] >> 1) & 1;
            }
            int base_s, base_t;
            unsigned agg_s, agg_t;
            block_scan2(ns, nt, ws, wt, base_s, base_t, agg_s, agg_t);
            if (tid == 0) {
                cnt_s[brick] = (int)agg_s;
                cnt_t[brick] = (int)agg_t;
            }
            __syncthreads();                       // ws / wt reused by the next brick
        }
        if (tid == 0) s_nund = 0;
        __syncthreads();
    }
}

// every brick's points from the scanned offsets off_s / off_t [nbr]
__global__ void __launch_bounds__(SEL_T) k_select_emit(
        SelRule r, const float *__restrict__ q, const float *__restrict__ e, const uint8_t *__restrict__ mask,
        const unsigned *__restrict__ maxes, const float4 *__restrict__ bstat, int nbr, const int *__restrict__ off_s,
        const int *__restrict__ off_t, uint32_t *__restrict__ src_key, uint32_t *__restrict__ src_pc,
        float *__restrict__ src_q, uint32_t *__restrict__ trg_key, uint32_t *__restrict__ trg_pc,
        uint8_t *__restrict__ tmask) {
    pdl_enter();
    __shared__ float s_thr_q, s_thr_e;
    __shared__ int s_qpos;
    __shared__ int s_mode[SEL_T], s_os[SEL_T], s_ot[SEL_T];
    __shared__ int ws[16], wt[16];
    __shared__ uint32_t st_key[4096 + 128], st_pc[4096 + 128];
    const int tid = threadIdx.x;
    if (tid == 0) block_thresholds(r, maxes, &s_thr_q, &s_thr_e, &s_qpos);
    __syncthreads();
    const int b = r.brick_edge_log2;
    const int ncell = 1 << (3 * b);
    for (int k0 = 0; blockIdx.x + (int64_t)k0 * gridDim.x < nbr; k0 += SEL_T) {
        const int64_t bk = blockIdx.x + (int64_t)(k0 + tid) * gridDim.x;
        if (bk < nbr) {
            s_mode[tid] = brick_mode(r, (uint32_t)bk, bstat[bk], s_thr_q, s_thr_e, s_qpos);
            s_os[tid] = off_s[bk];
            s_ot[tid] = off_t[bk];
        }
        __syncthreads();
        const int64_t left = (nbr - 1 - (blockIdx.x + (int64_t)k0 * gridDim.x)) / gridDim.x + 1;
        const int kn = (int)min((int64_t)SEL_T, left);
        for (int j = 0; j < kn; ++j) {
            const uint32_t brick = (uint32_t)(blockIdx.x + (int64_t)(k0 + j) * gridDim.x);
            uint32_t bx, by, bz;
            demorton3(brick, bx, by, bz);
            const int x0 = bx << b, y0 = by << b, z0 = bz << b;
            const int mode = s_mode[j];
            if (mode != 0) {
                brick_emit_decided(r, brick, mode, tid, x0, y0, z0, (unsigned)s_ot[j], trg_key, trg_pc, tmask);
                continue;
            }
            int my_bits[8];
            float my_q[8];
            uint32_t mx, my, mz;
            cube_rules(r, q, e, mask, tid, x0, y0, z0, ncell, s_thr_q, s_thr_e, s_qpos, tmask, my_bits, my_q, mx,
                       my, mz);
            int ns = 0, nt = 0;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                ns += my_bits[u] & 1;
                nt += (my_bits[u] >> 1) & 1;
            }
            int base_s, base_t;
            unsigned agg_s, agg_t;
            block_scan2(ns, nt, ws, wt, base_s, base_t, agg_s, agg_t);
            cube_emit(brick, b, tid, x0, y0, z0, mx, my, mz, my_bits, my_q, s_os[j] + base_s, base_t,
                      (unsigned)s_ot[j], agg_t, st_key, st_pc, src_key, src_pc, src_q, trg_key, trg_pc);
            __syncthreads();                       // staging and ws / wt reused by the next brick
        }
        __syncthreads();                           // s_mode / s_os / s_ot reused
    }
}

int select_launch(const SelectArgs &A, cudaStream_t st) {
    int b = A.brick_log2;
    int nbr = 1 << (3 * (A.D - b));
    SelRule r;
    r.nx = A.nx; r.ny = A.ny; r.nz = A.nz;
    r.brick_edge_log2 = b;
    r.src_all = A.i_frac == 0.0;
    r.i_frac = A.i_frac;
    r.trg_mode = A.mask ? 2 : (A.emag ? 1 : 0);
    r.e_frac = A.e_frac;
    r.e_app = A.e_app;
    int64_t n = (int64_t)A.nx * A.ny * A.nz;
    if (!A.zeroed) {
        cudaMemsetAsync(A.maxes, 0, 2 * sizeof(unsigned), st);
        cudaMemsetAsync(A.totals + 2, 0, sizeof(int), st);
    }
    int gm = (int)((n / 4 + 255) / 256);
    if (gm > 152 * 8) gm = 152 * 8;
    if (gm < 1) gm = 1;
    const float *gq = r.src_all ? nullptr : A.q, *ge = r.trg_mode == 1 ? A.emag : nullptr;
    // one pass over bricks of 16^3 cells: the maxima with the per-brick statistics
    const bool stats = !A.two_pass && A.bstat != nullptr && b == 4 && (gq || ge);
    const float4 *bstat = reinterpret_cast<const float4 *>(A.bstat);
    if (stats) launch_pdl(k_brick_stats, nbr, STAT_T, 0, st, r, gq, ge, reinterpret_cast<float4 *>(A.bstat), A.maxes);
    else if (gq || ge) launch_pdl(k_grid_max, gm, 256, 0, st, gq, ge, n, A.maxes);
    A.launched = (stats || gq || ge) ? 1 : 0;
    if (A.two_pass) {
        launch_pdl(k_select_brick<false>, nbr, 512, 0, st, r, A.q, A.emag, A.mask, A.maxes, A.cnt_s, A.cnt_t,
                                                   nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                                                   nullptr);
        launch_pdl(k_scan2, 1, 1024, 0, st, A.cnt_s, A.cnt_t, A.off_s, A.off_t, nbr, A.totals);
        launch_pdl(k_select_brick<true>, nbr, 512, 0, st, r, A.q, A.emag, A.mask, A.maxes, nullptr, nullptr,
                                                  A.off_s, A.off_t, A.src_key, A.src_pc, A.src_q,
                                                  A.trg_key, A.trg_pc, A.tmask);
        A.launched += 3;
        return cudaGetLastError() == cudaSuccess ? 0 : -1;
    }
    if (stats && !A.lookback) {
        const int grid = std::max(1, std::min(nbr, 2 * sm_count()));
        launch_pdl(k_select_count, grid, SEL_T, 0, st, r, A.q, A.emag, A.mask, (const unsigned *)A.maxes, bstat, nbr,
                   A.cnt_s, A.cnt_t);
        launch_pdl(k_scan2, 1, 1024, 0, st, A.cnt_s, A.cnt_t, A.off_s, A.off_t, nbr, A.totals);
        launch_pdl(k_select_emit, grid, SEL_T, 0, st, r, A.q, A.emag, A.mask, (const unsigned *)A.maxes, bstat, nbr,
                   (const int *)A.off_s, (const int *)A.off_t, A.src_key, A.src_pc, A.src_q, A.trg_key, A.trg_pc,
                   A.tmask);
        A.launched += 3;
        return cudaGetLastError() == cudaSuccess ? 1 : -1;
    }
    // one pass: the look-back states live in cnt_s .. cnt_t (2 ints per brick), the ticket in off_s[0]
    unsigned long long *state = reinterpret_cast<unsigned long long *>(A.cnt_s);
    unsigned *ticket = reinterpret_cast<unsigned *>(A.off_s);
    cudaMemsetAsync(state, 0, sizeof(unsigned long long) * nbr, st);
    cudaMemsetAsync(ticket, 0, sizeof(unsigned), st);
    launch_pdl(k_select_onepass, nbr, SEL_T, 0, st, r, A.q, A.emag, A.mask, A.maxes, state, ticket, nbr, A.totals,
                                          A.src_key, A.src_pc, A.src_q, A.trg_key, A.trg_pc, A.tmask, A.wait_limit,
                                          stats ? bstat : nullptr);
    A.launched += 1;
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace sph
