// Morton octree over the selected points and its interaction lists
// (paper Section 2.4: "each leaf cube contains no more than a prescribed number
// of points"; Eq. nearfar's near / far split; the recursive far-field hierarchy).
//
// Build: the grid is embedded in a 2^D cube of cells.  Level l has a dense
// array box_at[l][key] (8^l entries, -1 = no box) so every neighbour lookup is
// one load.  Level by level (top-down):
//   k_tree_flags  : for every child slot of a split parent, binary-search the
//                   Morton-sorted point keys for the child's [begin, end) ranges;
//   scan          : exclusive scan of the existence flags -> canonical index
//                   (boxes ordered by (level, key));
//   k_tree_emit   : write the compact box records and box_at[l].
// A box splits iff it holds more than S sources or more than S targets and its
// level is below D.  All of it is integer arithmetic, so the tree is
// bit-identical to the oracle's.
//
// Lists (per target-side box B, pairs (B, A)):
//   U: B leaf, A leaf with sources, adjacent (touching or overlapping closed cubes);
//   V: same level >= 2, parents adjacent, A not adjacent to B; offset code kept;
//   W: B leaf, A finer with sources, parent(A) adjacent to B, A not adjacent;
//   X: A leaf with sources, coarser than B, A adjacent to parent(B), not to B.
// k_lists<false> counts, a scan gives CSR offsets, k_lists<true> fills.
#include "sph_kernels.cuh"

namespace sph {

// ------------------------------------------------------------ device-wide scan
constexpr int SCAN_T = 1024, SCAN_PER = 4, SCAN_TILE = SCAN_T * SCAN_PER;

__global__ void __launch_bounds__(SCAN_T) k_scan_reduce(const int *__restrict__ in, int n, int *__restrict__ bsum) {
    int base = blockIdx.x * SCAN_TILE;
    int s = 0;
    for (int u = 0; u < SCAN_PER; ++u) {
        int i = base + u * SCAN_T + threadIdx.x;
        if (i < n) s += in[i];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ int ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = ws[threadIdx.x];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) bsum[blockIdx.x] = s;
    }
}

// exclusive scan of bsum[0..nb) in place by one CTA; total -> *total
__global__ void __launch_bounds__(SCAN_T) k_scan_top(int *__restrict__ bsum, int nb, int *__restrict__ total) {
    __shared__ int sh[SCAN_T];
    int per = (nb + SCAN_T - 1) / SCAN_T;
    int beg = threadIdx.x * per, end = min(nb, beg + per);
    int r = 0;
    for (int i = beg; i < end; ++i) r += bsum[i];
    sh[threadIdx.x] = r;
    __syncthreads();
    for (int o = 1; o < SCAN_T; o <<= 1) {
        int v = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
        __syncthreads();
        sh[threadIdx.x] += v;
        __syncthreads();
    }
    int x = sh[threadIdx.x] - r;
    for (int i = beg; i < end; ++i) { int v = bsum[i]; bsum[i] = x; x += v; }
    if (threadIdx.x == SCAN_T - 1 && total) *total = sh[SCAN_T - 1];
}

__global__ void __launch_bounds__(SCAN_T) k_scan_final(const int *__restrict__ in, int *__restrict__ out, int n,
                                                       const int *__restrict__ bsum) {
    __shared__ int ws[32];
    int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_PER;
    int v[SCAN_PER];
    int s = 0;
    for (int u = 0; u < SCAN_PER; ++u) {
        int i = base + u;
        v[u] = i < n ? in[i] : 0;
        s += v[u];
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int inc = s;
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) ws[w] = inc;
    __syncthreads();
    if (w == 0) {
        int t = ws[lane];
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        ws[lane] = t;
    }
    __syncthreads();
    int x = bsum[blockIdx.x] + (w ? ws[w - 1] : 0) + inc - s;
    for (int u = 0; u < SCAN_PER; ++u) {
        int i = base + u;
        if (i < n) out[i] = x;
        x += v[u];
    }
}

size_t scan_tmp_ints(int n) { return (size_t)(n + SCAN_TILE - 1) / SCAN_TILE + 1; }

// out[i] = sum_{j<i} in[j]; *total = sum (device).  tmp: scan_tmp_ints(n) ints.
void scan_exclusive(const int *in, int *out, int n, int *total, int *tmp, cudaStream_t st) {
    if (n <= 0) {
        cudaMemsetAsync(total, 0, sizeof(int), st);
        return;
    }
    int nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    k_scan_reduce<<<nb, SCAN_T, 0, st>>>(in, n, tmp);
    k_scan_top<<<1, SCAN_T, 0, st>>>(tmp, nb, total);
    k_scan_final<<<nb, SCAN_T, 0, st>>>(in, out, n, tmp);
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
__global__ void k_tree_ranges(int n, const uint32_t *__restrict__ key, int D, int Lmax, int *__restrict__ beg,
                              int *__restrict__ end) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t k = key[i];
    // two keys fall in different slots of level l iff their highest differing bit b (0-based)
    // satisfies b >= 3 (D - l), i.e. for every l >= D - b / 3; only those levels are written
    auto first_level = [&](uint32_t other) {
        const int b = 31 - __clz(k ^ other);
        const int l0 = D - b / 3;
        return l0 < 0 ? 0 : l0;
    };
    const int lb = i == 0 ? 0 : first_level(key[i - 1]);
    const int le = i + 1 == n ? 0 : first_level(key[i + 1]);
    for (int l = lb; l <= Lmax; ++l) beg[dense_off(l) + (k >> (3 * (D - l)))] = i;
    for (int l = le; l <= Lmax; ++l) end[dense_off(l) + (k >> (3 * (D - l)))] = i + 1;
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
__global__ void k_tree_emit_all(TreeDev T, int64_t nslot, int Lmax, int D, int S, const int *__restrict__ flag,
                                const int *__restrict__ pos, const int *__restrict__ rsb,
                                const int *__restrict__ rse, const int *__restrict__ rtb,
                                const int *__restrict__ rte, const int *__restrict__ total,
                                const uint32_t *__restrict__ skey, int ns, const uint32_t *__restrict__ tkey, int nt) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s <= Lmax) {       // level table (threads 0..Lmax)
        const int l = (int)s;
        const int b0 = pos[dense_off(l)];
        const int b1 = l < Lmax ? pos[dense_off(l + 1)] : *total;
        T.lvl_base[l] = b0;
        T.lvl_count[l] = b1 - b0;
    }
    if (s >= nslot) return;
    if (!flag[s]) {
        T.box_at[s] = -1;
        return;
    }
    const int l = level_of_slot(s, Lmax);
    const int64_t m = s - dense_off(l);
    const int idx = pos[s];
    T.box_at[s] = idx;
    int sb = rsb[s], se = rse[s], tb = rtb[s], te = rte[s];
    // an empty range starts where the slot's first key would be inserted
    const uint32_t lo = (uint32_t)m << (3 * (D - l));
    if (se == sb) sb = se = lower_bound_u32(skey, 0, ns, lo);
    if (te == tb) tb = te = lower_bound_u32(tkey, 0, nt, lo);
    T.b_level[idx] = l;
    T.b_key[idx] = (uint32_t)m;
    T.b_sb[idx] = sb; T.b_se[idx] = se;
    T.b_tb[idx] = tb; T.b_te[idx] = te;
    T.b_parent[idx] = l > 0 ? pos[dense_off(l - 1) + (m >> 3)] : -1;
    T.b_leaf[idx] = !(l < D && (se - sb > S || te - tb > S));
}

// occ[s] = 1 if the slot's region holds a source point, or lies inside a leaf that holds
// sources (the deepest existing box over the slot); levels 0..Lmax-1.
__global__ void k_src_occ(TreeDev T, int64_t nslot, int Lmax, const int *__restrict__ rsb,
                          const int *__restrict__ rse, uint8_t *__restrict__ occ) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nslot) return;
    uint8_t o = rse[s] > rsb[s];
    if (!o) {
        int l = level_of_slot(s, Lmax);
        int64_t m = s - dense_off(l);
        for (; l >= 0; --l, m >>= 3) {
            const int B = T.box_at[dense_off(l) + m];
            if (B >= 0) {
                o = T.b_leaf[B] && T.b_se[B] > T.b_sb[B];
                break;
            }
        }
    }
    occ[s] = o;
}

__global__ void k_src_near(int64_t nslot, int Lmax, const uint8_t *__restrict__ occ, uint8_t *__restrict__ near) {
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
    cudaMemsetAsync(A.rsb, 0, nslot * sizeof(int), st);
    cudaMemsetAsync(A.rse, 0, nslot * sizeof(int), st);
    cudaMemsetAsync(A.rtb, 0, nslot * sizeof(int), st);
    cudaMemsetAsync(A.rte, 0, nslot * sizeof(int), st);
    if (A.ns > 0) k_tree_ranges<<<(A.ns + 255) / 256, 256, 0, st>>>(A.ns, A.skey, A.D, A.Lmax, A.rsb, A.rse);
    if (A.nt > 0) k_tree_ranges<<<(A.nt + 255) / 256, 256, 0, st>>>(A.nt, A.tkey, A.D, A.Lmax, A.rtb, A.rte);
    const int grid = (int)((nslot + 255) / 256);
    k_tree_exists<<<grid, 256, 0, st>>>(nslot, A.Lmax, A.D, A.S, A.rsb, A.rse, A.rtb, A.rte, A.flag);
    int *total = A.pos + nslot;
    scan_exclusive(A.flag, A.pos, (int)nslot, total, A.scan_tmp, st);
    k_tree_emit_all<<<grid, 256, 0, st>>>(A.T, nslot, A.Lmax, A.D, A.S, A.flag, A.pos, A.rsb, A.rse, A.rtb,
                                          A.rte, total, A.skey, A.ns, A.tkey, A.nt);
    const int64_t npar = dense_off(A.Lmax);        // slots of levels 0..Lmax-1
    if (npar > 0 && A.occ && A.near) {
        const int g2 = (int)((npar + 255) / 256);
        k_src_occ<<<g2, 256, 0, st>>>(A.T, npar, A.Lmax - 1, A.rsb, A.rse, A.occ);
        k_src_near<<<g2, 256, 0, st>>>(npar, A.Lmax - 1, A.occ, A.near);
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

__device__ __forceinline__ int lookup(const TreeDev &T, int level, int x, int y, int z) {
    int n = 1 << level;
    if (x < 0 || y < 0 || z < 0 || x >= n || y >= n || z >= n) return -1;
    return T.box_at[dense_off(level) + morton3(x, y, z)];
}

template <bool FILL>
__global__ void k_lists(TreeDev T, ListDev L, int nboxes, int D, int Lmax) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nboxes) return;
    int nU = 0, nV = 0, nW = 0, nX = 0;
    int pU = 0, pV = 0, pW = 0, pX = 0;
    if (FILL) { pU = L.u_off[b]; pV = L.v_off[b]; pW = L.w_off[b]; pX = L.x_off[b]; }
    int nt = T.b_te[b] - T.b_tb[b];
    if (nt > 0) {
        BoxGeom B = geom_of(T, b);
        const int l = B.level;
        // nothing with sources anywhere around the parent: every list is empty
        if (l >= 1 && T.near && !T.near[dense_off(l - 1) + morton3(B.x >> 1, B.y >> 1, B.z >> 1)]) nt = 0;
    }
    if (nt > 0) {
        BoxGeom B = geom_of(T, b);
        const int l = B.level;
        // ---- U and W (B leaf)
        if (T.b_leaf[b]) {
            int coarse[27];
            int ncoarse = 0;
            int stk[128];
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        int qx = B.x + dx, qy = B.y + dy, qz = B.z + dz;
                        int n = 1 << l;
                        if (qx < 0 || qy < 0 || qz < 0 || qx >= n || qy >= n || qz >= n) continue;
                        int A = lookup(T, l, qx, qy, qz);
                        if (A >= 0) {
                            if (T.b_se[A] <= T.b_sb[A]) continue;   // no sources anywhere below A
                            if (T.b_leaf[A]) {
                                if (T.b_se[A] > T.b_sb[A]) {
                                    if (FILL) L.u_src[pU] = A;
                                    ++pU; ++nU;
                                }
                            } else {
                                int sp = 0;
                                // push children of the colleague
                                uint32_t ck = T.b_key[A] << 3;
                                for (int c = 0; c < 8; ++c) {
                                    int C = T.box_at[dense_off(l + 1) + ck + c];
                                    if (C >= 0) stk[sp++] = C;
                                }
                                while (sp > 0) {
                                    int Dn = stk[--sp];
                                    BoxGeom G = geom_of(T, Dn);
                                    bool hs = T.b_se[Dn] > T.b_sb[Dn];
                                    if (adjacent(G, B, D)) {
                                        if (T.b_leaf[Dn]) {
                                            if (hs) {
                                                if (FILL) L.u_src[pU] = Dn;
                                                ++pU; ++nU;
                                            }
                                        } else if (sp + 8 <= 128) {
                                            uint32_t k2 = T.b_key[Dn] << 3;
                                            for (int c = 0; c < 8; ++c) {
                                                int C = T.box_at[dense_off(G.level + 1) + k2 + c];
                                                if (C >= 0) stk[sp++] = C;
                                            }
                                        }
                                    } else if (hs) {
                                        if (FILL) L.w_src[pW] = Dn;
                                        ++pW; ++nW;
                                    }
                                }
                            }
                        } else {
                            for (int m = l - 1; m >= 0; --m) {
                                int sh = l - m;
                                int Am = lookup(T, m, qx >> sh, qy >> sh, qz >> sh);
                                if (Am >= 0) {
                                    if (T.b_leaf[Am] && T.b_se[Am] > T.b_sb[Am]) {
                                        bool dup = false;
                                        for (int u = 0; u < ncoarse; ++u) dup |= coarse[u] == Am;
                                        if (!dup) coarse[ncoarse++] = Am;
                                    }
                                    break;
                                }
                            }
                        }
                    }
            for (int u = 0; u < ncoarse; ++u) {
                if (FILL) L.u_src[pU] = coarse[u];
                ++pU; ++nU;
            }
        }
        // ---- X, and whether any box adjacent to the parent holds sources (else V is empty)
        bool parent_near_src = false;
        if (l >= 2) {
            int cx = B.x >> 1, cy = B.y >> 1, cz = B.z >> 1;
            int found[27];
            int nf = 0;
            int n = 1 << (l - 1);
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        int qx = cx + dx, qy = cy + dy, qz = cz + dz;
                        if (qx < 0 || qy < 0 || qz < 0 || qx >= n || qy >= n || qz >= n) continue;
                        for (int m = l - 1; m >= 0; --m) {
                            int sh = l - 1 - m;
                            int Am = lookup(T, m, qx >> sh, qy >> sh, qz >> sh);
                            if (Am >= 0) {
                                bool hs = T.b_se[Am] > T.b_sb[Am];
                                if (m == l - 1) parent_near_src |= hs;
                                if (T.b_leaf[Am] && hs) {
                                    BoxGeom G = geom_of(T, Am);
                                    if (!adjacent(G, B, D)) {
                                        bool dup = false;
                                        for (int u = 0; u < nf; ++u) dup |= found[u] == Am;
                                        if (!dup) found[nf++] = Am;
                                    }
                                }
                                break;
                            }
                        }
                    }
            for (int u = 0; u < nf; ++u) {
                if (FILL) L.x_src[pX] = found[u];
                ++pX; ++nX;
            }
        }
        // ---- V (children of the parent's neighbours that hold sources)
        if (l >= 2 && parent_near_src) {
            int px = (B.x >> 1) << 1, py = (B.y >> 1) << 1, pz = (B.z >> 1) << 1;
            for (int dz = -2; dz <= 3; ++dz)
                for (int dy = -2; dy <= 3; ++dy)
                    for (int dx = -2; dx <= 3; ++dx) {
                        int qx = px + dx, qy = py + dy, qz = pz + dz;
                        int ox = qx - B.x, oy = qy - B.y, oz = qz - B.z;
                        if (abs(ox) <= 1 && abs(oy) <= 1 && abs(oz) <= 1) continue;
                        int A = lookup(T, l, qx, qy, qz);
                        if (A >= 0 && T.b_se[A] > T.b_sb[A]) {
                            if (FILL) {
                                L.v_src[pV] = A;
                                L.v_trg[pV] = b;
                                L.v_oc[pV] = (short)((ox + 3) + 7 * (oy + 3) + 49 * (oz + 3));
                            }
                            ++pV; ++nV;
                        }
                    }
        }
    }
    if (!FILL) {
        L.u_cnt[b] = nU; L.v_cnt[b] = nV; L.w_cnt[b] = nW; L.x_cnt[b] = nX;
    }
}

void lists_count_launch(const TreeDev &T, const ListDev &L, int nboxes, int D, int Lmax, int *scan_tmp,
                        int *totals /* device [4] */, cudaStream_t st) {
    if (nboxes <= 0) {
        cudaMemsetAsync(totals, 0, 4 * sizeof(int), st);
        return;
    }
    k_lists<false><<<(nboxes + 127) / 128, 128, 0, st>>>(T, L, nboxes, D, Lmax);
    scan_exclusive(L.u_cnt, L.u_off, nboxes, totals + 0, scan_tmp, st);
    scan_exclusive(L.v_cnt, L.v_off, nboxes, totals + 1, scan_tmp, st);
    scan_exclusive(L.w_cnt, L.w_off, nboxes, totals + 2, scan_tmp, st);
    scan_exclusive(L.x_cnt, L.x_off, nboxes, totals + 3, scan_tmp, st);
}

__global__ void k_close_offsets(ListDev L, int nboxes, const int *__restrict__ totals) {
    if (threadIdx.x == 0) {
        L.u_off[nboxes] = totals[0];
        L.v_off[nboxes] = totals[1];
        L.w_off[nboxes] = totals[2];
        L.x_off[nboxes] = totals[3];
    }
}

void lists_fill_launch(const TreeDev &T, const ListDev &L, int nboxes, int D, int Lmax,
                       const int *totals, cudaStream_t st) {
    if (nboxes <= 0) return;
    k_close_offsets<<<1, 32, 0, st>>>(L, nboxes, totals);
    k_lists<true><<<(nboxes + 127) / 128, 128, 0, st>>>(T, L, nboxes, D, Lmax);
}

}  // namespace sph
