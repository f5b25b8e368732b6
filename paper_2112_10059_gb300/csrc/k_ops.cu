// Precomputed translation operators of the kernel-independent FMM (paper
// Section 2.4, Eq. s2l and Figure fmulloc).  Box at level l has half-width
// w_l = h 2^(D-l) / 2.  G is the kernel of Eq. gfun; it has two length scales,
// so every level needs its own M2L matrices.
//
// FAR_CHEB (default): artificial source points = tensor Chebyshev nodes
// x_m = c + w (t_a, t_b, t_c), t_k = cos((2k+1) pi / (2p)); S_m(y) is the tensor
// Lagrange polynomial of node m.
//   M2M_c[i][j] = S_i(child c node j, in parent coordinates)          (all levels)
//   L2L_c[i][j] = S_j(child c node i, in parent coordinates)          (all levels)
//   M2L_{l,o}[i][j] = G(|x_i - (2 w_l o + y_j)|)                       (per level)
//
// FAR_SURFACE (the equivalent / check surfaces of Figure fmulloc):
//   UC2E_l = pinv(K(upward check, upward equivalent))        radii 2.95 w / 1.05 w
//   DC2E_l = pinv(K(downward check, downward equivalent))    radii 1.05 w / 2.95 w
// with every pseudo-inverse folded in (the passes carry check potentials):
//   M2M_{l,c} = K(parent upward check, child c upward equivalent) UC2E_{l+1}
//   L2L_{l,c} = K(child c downward check, parent downward equivalent) DC2E_{l-1}
//   M2L_{l,o} = K(target downward check, source upward equivalent at 2 w o) UC2E_l
//   E_l       = K(cell centres of a box, downward equivalent) DC2E_l  (L2P table)
// The pseudo-inverses solve Eq. s2l in the least-squares sense by a truncated
// SVD from one-sided (Hestenes) Jacobi rotations in FP64 on the GPU, one CTA per
// matrix; singular values below eps * sigma_max are dropped.
//
// FP64 is used only here; every stored operator is FP32 (plus BF16 hi / lo of M2L).
#include <cuda_bf16.h>
#include <vector>
#include "sph_kernels.cuh"

namespace sph {

// ---------------------------------------------------------------- node tables
__global__ void k_nodes_init(int method, int order, int n, int npad, float *nodes, float *cheb_t) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (method == FAR_CHEB && m < order)
        cheb_t[m] = (float)cos((2.0 * m + 1.0) * 3.14159265358979323846 / (2.0 * order));
    if (m >= npad) return;
    float x = 0.f, y = 0.f, z = 0.f;
    if (m < n) {
        if (method == FAR_CHEB) {
            int a = m % order, b = (m / order) % order, c = m / (order * order);
            x = (float)cos((2.0 * a + 1.0) * 3.14159265358979323846 / (2.0 * order));
            y = (float)cos((2.0 * b + 1.0) * 3.14159265358979323846 / (2.0 * order));
            z = (float)cos((2.0 * c + 1.0) * 3.14159265358979323846 / (2.0 * order));
        } else {
            int cnt = 0;
            for (int a = 0; a < order; ++a)
                for (int b = 0; b < order; ++b)
                    for (int c = 0; c < order; ++c) {
                        bool surf = (a == 0 || a == order - 1 || b == 0 || b == order - 1 || c == 0 ||
                                     c == order - 1);
                        if (!surf) continue;
                        if (cnt == m) {
                            x = -1.0f + 2.0f * a / (order - 1);
                            y = -1.0f + 2.0f * b / (order - 1);
                            z = -1.0f + 2.0f * c / (order - 1);
                        }
                        ++cnt;
                    }
        }
    }
    nodes[4 * m + 0] = x;
    nodes[4 * m + 1] = y;
    nodes[4 * m + 2] = z;
    nodes[4 * m + 3] = 0.f;
}

__global__ void k_slot_init(short *slot_of_code) {
    if (threadIdx.x == 0) {
        int s = 0;
        for (int c = 0; c < SPH_NOFF; ++c) {
            int ox = c % 7 - 3, oy = (c / 7) % 7 - 3, oz = c / 49 - 3;
            bool near = abs(ox) <= 1 && abs(oy) <= 1 && abs(oz) <= 1;
            slot_of_code[c] = near ? (short)-1 : (short)(s++);
        }
    }
}

// 1D Lagrange basis polynomial k of the Chebyshev nodes, in FP64.
__device__ double lagrange64(int order, int k, double x) {
    double tk = cos((2.0 * k + 1.0) * 3.14159265358979323846 / (2.0 * order));
    double v = 1.0;
    for (int j = 0; j < order; ++j) {
        if (j == k) continue;
        double tj = cos((2.0 * j + 1.0) * 3.14159265358979323846 / (2.0 * order));
        v *= (x - tj) / (tk - tj);
    }
    return v;
}

// Chebyshev M2M / L2L for child c, transposed storage [col][row]:
//   m2m: row = parent node, col = child node: S_row(child node col in parent coordinates)
//   l2l: row = child node,  col = parent node: S_col(child node row in parent coordinates)
__global__ void k_cheb_m2m_l2l(int order, int n, int npad, float *__restrict__ m2m_t, float *__restrict__ l2l_t) {
    int c = blockIdx.y;
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * n) return;
    int pn = e / n, ch = e % n;     // parent node, child node
    int ia = pn % order, ib = (pn / order) % order, ic = pn / (order * order);
    int ja = ch % order, jb = (ch / order) % order, jc = ch / (order * order);
    double sx = (c & 1) ? 0.5 : -0.5, sy = (c & 2) ? 0.5 : -0.5, sz = (c & 4) ? 0.5 : -0.5;
    double tja = cos((2.0 * ja + 1.0) * 3.14159265358979323846 / (2.0 * order));
    double tjb = cos((2.0 * jb + 1.0) * 3.14159265358979323846 / (2.0 * order));
    double tjc = cos((2.0 * jc + 1.0) * 3.14159265358979323846 / (2.0 * order));
    double v = lagrange64(order, ia, sx + 0.5 * tja) * lagrange64(order, ib, sy + 0.5 * tjb) *
               lagrange64(order, ic, sz + 0.5 * tjc);
    size_t base = (size_t)c * npad * npad;
    m2m_t[base + (size_t)ch * npad + pn] = (float)v;
    l2l_t[base + (size_t)pn * npad + ch] = (float)v;
}

// Chebyshev L2P table of a box of edge e cells: out[k * rows + m] = S_k(cell m), m the
// local Morton index of the cell, unit coordinate (2 l + 1 - e) / e per axis.
__global__ void k_cheb_etab(int order, int e, int n, float *__restrict__ out) {
    int rows = e * e * e;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * n) return;
    int m = idx / n, k = idx % n;
    uint32_t lx, ly, lz;
    demorton3((uint32_t)m, lx, ly, lz);
    int a = k % order, b = (k / order) % order, c = k / (order * order);
    double v = lagrange64(order, a, (2.0 * lx + 1 - e) / e) * lagrange64(order, b, (2.0 * ly + 1 - e) / e) *
               lagrange64(order, c, (2.0 * lz + 1 - e) / e);
    out[(size_t)k * rows + m] = (float)v;
}

// Kernel matrix K[i][j] = G(|t_i - s_j|), t_i = ct + rt * u_i, s_j = cs + rs * u_j (cm).
struct MatSpec {
    double ct[3], rt, cs[3], rs;
    double *out;       // row-major n x n (FP64), or nullptr
    float *out_t;      // FP32 transposed [j][i] (npad stride), or nullptr
};

__global__ void k_kmat(const MatSpec *__restrict__ specs, const float *__restrict__ nodes, int n, int npad,
                       double alpha, double beta, double C) {
    const MatSpec S = specs[blockIdx.y];
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * n) return;
    int i = e / n, j = e % n;
    double dx = (S.ct[0] + S.rt * nodes[4 * i + 0]) - (S.cs[0] + S.rs * nodes[4 * j + 0]);
    double dy = (S.ct[1] + S.rt * nodes[4 * i + 1]) - (S.cs[1] + S.rs * nodes[4 * j + 1]);
    double dz = (S.ct[2] + S.rt * nodes[4 * i + 2]) - (S.cs[2] + S.rs * nodes[4 * j + 2]);
    double g = g64(sqrt(dx * dx + dy * dy + dz * dz), alpha, beta, C);
    if (S.out) S.out[e] = g;
    if (S.out_t) S.out_t[(size_t)j * npad + i] = (float)g;
}

// Round-robin pairing: round r (0..n-2), pair k (0..n/2-1); every unordered pair once per sweep.
__device__ __forceinline__ void rr_pair(int n, int r, int k, int &p, int &q) {
    const int n1 = n - 1;
    if (k == 0) { p = r; q = n1; }
    else { p = (r + k) % n1; q = (r - k + n1) % n1; }
}

// One CTA per matrix (n even).  K: row-major n x n.  Out: pinv row-major n x n.
// scratch: 2 n*n doubles per matrix (V, and W when it does not fit in shared memory).
__global__ void __launch_bounds__(1024) k_jacobi_pinv(double *const *__restrict__ Ks, double *const *__restrict__ Ps,
                                                     double *__restrict__ scratch, int n, int w_in_smem,
                                                     double eps, int max_sweeps) {
    extern __shared__ double smem_d[];
    double *V = scratch + (size_t)blockIdx.x * 2 * n * n;                   // column-major
    double *Wsh = w_in_smem ? smem_d : V + (size_t)n * n;                   // column-major W[j*n + i]
    double *inv2 = w_in_smem ? smem_d + (size_t)n * n : smem_d;
    __shared__ int changed;
    __shared__ double smax2;
    const double *K = Ks[blockIdx.x];
    double *Pout = Ps[blockIdx.x];
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        int i = e / n, j = e % n;
        Wsh[(size_t)j * n + i] = K[e];
        V[(size_t)j * n + i] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) changed = 0;
        __syncthreads();
        for (int r = 0; r < n - 1; ++r) {
            for (int k = warp; k < n / 2; k += nw) {
                int p, q;
                rr_pair(n, r, k, p, q);
                double *wp = Wsh + (size_t)p * n, *wq = Wsh + (size_t)q * n;
                double a = 0, b = 0, g = 0;
                for (int i = lane; i < n; i += 32) {
                    double x = wp[i], y = wq[i];
                    a = fma(x, x, a);
                    b = fma(y, y, b);
                    g = fma(x, y, g);
                }
                for (int o = 16; o > 0; o >>= 1) {
                    a += __shfl_xor_sync(0xffffffffu, a, o);
                    b += __shfl_xor_sync(0xffffffffu, b, o);
                    g += __shfl_xor_sync(0xffffffffu, g, o);
                }
                if (g != 0.0 && fabs(g) > 1e-15 * sqrt(a * b)) {
                    double zeta = (b - a) / (2.0 * g);
                    double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                    double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
                    for (int i = lane; i < n; i += 32) {
                        double x = wp[i], y = wq[i];
                        wp[i] = c * x - s * y;
                        wq[i] = s * x + c * y;
                    }
                    double *vp = V + (size_t)p * n, *vq = V + (size_t)q * n;
                    for (int i = lane; i < n; i += 32) {
                        double x = vp[i], y = vq[i];
                        vp[i] = c * x - s * y;
                        vq[i] = s * x + c * y;
                    }
                    if (lane == 0) changed = 1;
                }
            }
            __syncthreads();
        }
        if (!changed) break;
        __syncthreads();
    }
    for (int j = warp; j < n; j += nw) {
        double s = 0;
        for (int i = lane; i < n; i += 32) s = fma(Wsh[(size_t)j * n + i], Wsh[(size_t)j * n + i], s);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) inv2[j] = s;   // sigma^2
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0;
        for (int j = 0; j < n; ++j) m = fmax(m, inv2[j]);
        smax2 = m;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double s2 = inv2[j];
        inv2[j] = (s2 > eps * eps * smax2 && s2 > 0) ? 1.0 / s2 : 0.0;
    }
    __syncthreads();
    // pinv[i][k] = sum_j V[i][j] W[k][j] / sigma_j^2   (A V = W, A = W V^T)
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        int i = e / n, kk = e % n;
        double acc = 0;
        for (int j = 0; j < n; ++j) acc = fma(V[(size_t)j * n + i] * inv2[j], Wsh[(size_t)j * n + kk], acc);
        Pout[e] = acc;
    }
}

// C = A * B with A: M x n, B: n x n (FP64, row-major), written to FP32:
//   transposed != 0: out[j*npad + i];  transposed == 0: out[i*npad + j]
struct GemmSpec {
    const double *A, *B;
    float *out;
    int M, transposed;
};
__global__ void __launch_bounds__(256) k_gemm64(const GemmSpec *__restrict__ specs, int n, int npad) {
    const GemmSpec S = specs[blockIdx.z];
    if ((int)blockIdx.y * 16 >= S.M) return;
    __shared__ double As[16][17], Bs[16][17];
    int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
    int i = blockIdx.y * 16 + ty, j = blockIdx.x * 16 + tx;
    double acc = 0;
    for (int k0 = 0; k0 < n; k0 += 16) {
        As[ty][tx] = (i < S.M && k0 + tx < n) ? S.A[(size_t)i * n + k0 + tx] : 0.0;
        Bs[ty][tx] = (k0 + ty < n && j < n) ? S.B[(size_t)(k0 + ty) * n + j] : 0.0;
        __syncthreads();
        for (int k = 0; k < 16; ++k) acc = fma(As[ty][k], Bs[k][tx], acc);
        __syncthreads();
    }
    if (i < S.M && j < n) {
        if (S.transposed) S.out[(size_t)j * npad + i] = (float)acc;
        else S.out[(size_t)i * npad + j] = (float)acc;
    }
}

// K[m][j] = G(|c_m - rs u_j|) for the cell centres c_m of a box of edge e cells,
// m = lx + e (ly + e lz), c = ((2 l + 1 - e) h/2) per axis.
__global__ void k_kmat_cells64(int e, int n, double hh, double rs, const float *__restrict__ nodes, double alpha,
                               double beta, double C, double *__restrict__ out) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    int rows = e * e * e;
    if (idx >= rows * n) return;
    int m = idx / n, j = idx % n;
    int lx = m % e, ly = (m / e) % e, lz = m / (e * e);
    double dx = (2 * lx + 1 - e) * hh - rs * nodes[4 * j + 0];
    double dy = (2 * ly + 1 - e) * hh - rs * nodes[4 * j + 1];
    double dz = (2 * lz + 1 - e) * hh - rs * nodes[4 * j + 2];
    out[idx] = g64(sqrt(dx * dx + dy * dy + dz * dz), alpha, beta, C);
}

// Ball integral of G (self term): int_0^a (e^{-alpha r} - e^{-beta r}) / (L r) dr by composite
// Simpson on the smooth integrand (its value at r = 0 is (beta - alpha)/L), 2^14 panels.
__global__ void k_self_int(double a, double alpha, double beta, double *out) {
    const int N = 1 << 14;
    double L = log(beta / alpha);
    double hh = a / N;
    double s = 0;
    for (int m = threadIdx.x; m <= N; m += blockDim.x) {
        double r = m * hh;
        double f = (m == 0) ? (beta - alpha) / L : exp(-alpha * r) * (-expm1(-(beta - alpha) * r)) / (L * r);
        double wgt = (m == 0 || m == N) ? 1.0 : ((m & 1) ? 4.0 : 2.0);
        s += wgt * f;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int u = 0; u < (int)(blockDim.x >> 5); ++u) t += ws[u];
        *out = t * hh / 3.0;
    }
}

// ---------------------------------------------------------------- FP64 work buffer
// FAR_SURFACE: per level l (0..Lmax) 20 n*n blocks (Kuc, Kdc, UC2E, DC2E, Km2m[8], Kl2l[8]);
// then 2 n*n of Jacobi scratch per pseudo-inverse (2 per level), NSLOT n*n for one
// level's M2L kernel matrices and 4096 n for one L2P cell matrix.  Both methods end
// with 64 Ki doubles of launch tables.
constexpr size_t BLK = 20;

size_t ops_work_doubles(int method, int n, int Lmax) {
    const size_t nn = (size_t)n * n;
    if (method == FAR_CHEB) return 64 * 1024;
    return (size_t)(Lmax + 1) * BLK * nn + 4 * (size_t)(Lmax + 1) * nn + NSLOT * nn + 4096 * (size_t)n + 64 * 1024;
}

static int edge_of(int D, int l) { return 1 << (D - l); }

size_t ops_etab_floats(int method, int npad, int D, int Lmax) {
    size_t s = npad;
    for (int l = 2; l <= Lmax; ++l) {
        int e = edge_of(D, l);
        if (e <= ETAB_MAX_EDGE) s += (size_t)e * e * e * npad;
    }
    return s;
}

// level whose boxes have edge 4 and get the composed L2L + L2P images, or -1
static int l2pc_level(int D, int Lmax) {
    const int l = D - 2;
    return (l >= 3 && l <= Lmax && l < 16 && 4 <= ETAB_MAX_EDGE) ? l : -1;
}

size_t ops_l2p_img_elems(int D, int Lmax) {
    size_t s = 0;
    for (int l = 2; l <= Lmax && l < 16; ++l) {
        int e = edge_of(D, l);
        if (e <= ETAB_MAX_EDGE) s += l2p_image_elems(e);
    }
    if (l2pc_level(D, Lmax) >= 0) s += 8 * l2p_image_elems(4);
    return s;
}

void ops_layout(int D, int Lmax, double *work, OpsDev &O) {
    for (int l = 0; l < 16; ++l) O.e_off[l] = -1;
    for (int l = 0; l < 16; ++l) O.l2p_off[l] = -1;
    O.l2pc_off = -1;
    if (O.method == FAR_CHEB && O.l2p_img) {
        long long off = 0;
        for (int l = 2; l <= Lmax && l < 16; ++l) {
            int e = edge_of(D, l);
            if (e <= ETAB_MAX_EDGE) {
                O.l2p_off[l] = off;
                off += (long long)l2p_image_elems(e);
            }
        }
        if (l2pc_level(D, Lmax) >= 0) O.l2pc_off = off;
    }
    O.uc64 = O.dc64 = nullptr;
    O.pinv_stride = 0;
    long long off = 0;
    for (int l = 2; l <= Lmax && l < 16; ++l) {
        int e = edge_of(D, l);
        if (e <= ETAB_MAX_EDGE) {
            O.e_off[l] = off;
            off += (long long)e * e * e * O.npad;
        }
    }
    if (O.method != FAR_SURFACE) return;
    const size_t nn = (size_t)O.n * O.n;
    O.pinv_stride = (long long)(BLK * nn);
    O.uc64 = work + 2 * nn;
    O.dc64 = work + 3 * nn;
}

static void offsets_of(int slot, int &ox, int &oy, int &oz) {
    ox = oy = oz = 0;
    int s = 0;
    for (int code = 0; code < SPH_NOFF; ++code) {
        int x = code % 7 - 3, y = (code / 7) % 7 - 3, z = code / 49 - 3;
        if (abs(x) <= 1 && abs(y) <= 1 && abs(z) <= 1) continue;
        if (s == slot) { ox = x; oy = y; oz = z; return; }
        ++s;
    }
}

static int build_cheb(const OpsBuildArgs &A, cudaStream_t st, double C) {
    const OpsDev &O = A.ops;
    const int n = O.n, np = O.npad;
    const size_t pp = (size_t)np * np;
    cudaMemsetAsync(O.m2m_t, 0, sizeof(float) * (A.Lmax + 1) * 8 * pp, st);
    cudaMemsetAsync(O.l2l_t, 0, sizeof(float) * (A.Lmax + 1) * 8 * pp, st);
    cudaMemsetAsync(O.m2l_t, 0, sizeof(float) * (A.Lmax + 1) * NSLOT * pp, st);
    // interpolation operators are the same on every level: build level 0, copy
    k_cheb_m2m_l2l<<<dim3((n * n + 255) / 256, 8), 256, 0, st>>>(O.order, n, np, O.m2m_t, O.l2l_t);
    for (int l = 1; l <= A.Lmax; ++l) {
        cudaMemcpyAsync(O.m2m_t + (size_t)l * 8 * pp, O.m2m_t, sizeof(float) * 8 * pp, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(O.l2l_t + (size_t)l * 8 * pp, O.l2l_t, sizeof(float) * 8 * pp, cudaMemcpyDeviceToDevice, st);
    }
    // M2L kernel matrices between node sets, per level
    std::vector<MatSpec> ms;
    for (int l = 2; l <= A.Lmax; ++l) {
        double w = A.h * (double)(1 << (A.D - l)) * 0.5;
        for (int slot = 0; slot < NSLOT; ++slot) {
            int ox, oy, oz;
            offsets_of(slot, ox, oy, oz);
            MatSpec m{};
            m.rt = w;
            m.cs[0] = 2.0 * w * ox; m.cs[1] = 2.0 * w * oy; m.cs[2] = 2.0 * w * oz;
            m.rs = w;
            m.out = nullptr;
            m.out_t = O.m2l_t + ((size_t)l * NSLOT + slot) * pp;
            ms.push_back(m);
        }
    }
    // L2P interpolation tables (rows beyond n of the padded K dimension stay zero)
    cudaMemsetAsync(O.e_tab, 0, sizeof(float) * ops_etab_floats(O.method, np, A.D, A.Lmax), st);
    for (int l = 2; l <= A.Lmax; ++l) {
        if (O.e_off[l] < 0) continue;
        int e = 1 << (A.D - l);
        k_cheb_etab<<<(e * e * e * n + 255) / 256, 256, 0, st>>>(O.order, e, n, O.e_tab + O.e_off[l]);
    }
    if (!ms.empty()) {
        MatSpec *dms = (MatSpec *)A.work;
        cudaMemcpyAsync(dms, ms.data(), sizeof(MatSpec) * ms.size(), cudaMemcpyHostToDevice, st);
        for (size_t k0 = 0; k0 < ms.size(); k0 += NSLOT)
            k_kmat<<<dim3((n * n + 255) / 256, NSLOT), 256, 0, st>>>(dms + k0, O.nodes, n, np, A.alpha, A.beta, C);
    }
    return 0;
}

static int build_surface(const OpsBuildArgs &A, cudaStream_t st, double C) {
    const OpsDev &O = A.ops;
    const Radii R = O.r;
    const int n = O.n, np = O.npad;
    const int L0 = 2, L1 = A.Lmax;
    const size_t nn = (size_t)n * n, pp = (size_t)np * np;
    double *work = A.work;
    auto Kuc = [&](int l) { return work + ((size_t)l * BLK + 0) * nn; };
    auto Kdc = [&](int l) { return work + ((size_t)l * BLK + 1) * nn; };
    auto UC = [&](int l) { return work + ((size_t)l * BLK + 2) * nn; };
    auto DC = [&](int l) { return work + ((size_t)l * BLK + 3) * nn; };
    auto Km2m = [&](int l, int c) { return work + ((size_t)l * BLK + 4 + c) * nn; };
    auto Kl2l = [&](int l, int c) { return work + ((size_t)l * BLK + 12 + c) * nn; };
    double *jac = work + (size_t)(A.Lmax + 1) * BLK * nn;
    double *km2l = jac + 4 * (size_t)(A.Lmax + 1) * nn;
    double *kcell = km2l + (size_t)NSLOT * nn;
    char *tables = (char *)(kcell + 4096 * (size_t)n);
    auto half = [&](int l) { return A.h * (double)(1 << (A.D - l)) * 0.5; };

    std::vector<MatSpec> specs;
    for (int l = L0; l <= L1; ++l) {
        double w = half(l);
        MatSpec s{};
        s.rt = R.uc * w; s.rs = R.ue * w; s.out = Kuc(l);
        specs.push_back(s);
        s = MatSpec{};
        s.rt = R.dc * w; s.rs = R.de * w; s.out = Kdc(l);
        specs.push_back(s);
        for (int c = 0; c < 8; ++c) {
            if (l < L1) {   // parent (l) upward check <- child (l+1) upward equivalent
                double cw = w * 0.5;
                MatSpec m{};
                m.rt = R.uc * w;
                m.cs[0] = ((c & 1) ? 1 : -1) * cw;
                m.cs[1] = ((c & 2) ? 1 : -1) * cw;
                m.cs[2] = ((c & 4) ? 1 : -1) * cw;
                m.rs = R.ue * cw;
                m.out = Km2m(l, c);
                specs.push_back(m);
            }
            if (l > L0) {   // child (l) downward check <- parent (l-1) downward equivalent
                MatSpec m{};
                m.ct[0] = ((c & 1) ? 1 : -1) * w;
                m.ct[1] = ((c & 2) ? 1 : -1) * w;
                m.ct[2] = ((c & 4) ? 1 : -1) * w;
                m.rt = R.dc * w;
                m.rs = R.de * 2.0 * w;
                m.out = Kl2l(l, c);
                specs.push_back(m);
            }
        }
    }
    MatSpec *dspecs = (MatSpec *)tables;
    cudaMemcpyAsync(dspecs, specs.data(), sizeof(MatSpec) * specs.size(), cudaMemcpyHostToDevice, st);
    k_kmat<<<dim3((n * n + 255) / 256, (unsigned)specs.size()), 256, 0, st>>>(dspecs, O.nodes, n, np, A.alpha,
                                                                              A.beta, C);
    // pseudo-inverses: 2 per level
    std::vector<double *> kin, pout;
    for (int l = L0; l <= L1; ++l) {
        kin.push_back(Kuc(l)); pout.push_back(UC(l));
        kin.push_back(Kdc(l)); pout.push_back(DC(l));
    }
    const int npi = (int)kin.size();
    double **dptr = (double **)(tables + sizeof(MatSpec) * (specs.size() + 1));
    cudaMemcpyAsync(dptr, kin.data(), sizeof(double *) * npi, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(dptr + npi, pout.data(), sizeof(double *) * npi, cudaMemcpyHostToDevice, st);
    const int w_in_smem = (nn + n) * sizeof(double) <= 200 * 1024;
    size_t smem = (w_in_smem ? nn * sizeof(double) : 0) + n * sizeof(double);
    cudaFuncSetAttribute(k_jacobi_pinv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_jacobi_pinv<<<npi, 1024, smem, st>>>(dptr, dptr + npi, jac, n, w_in_smem, A.eps, 40);

    cudaMemsetAsync(O.m2m_t, 0, sizeof(float) * (A.Lmax + 1) * 8 * pp, st);
    cudaMemsetAsync(O.l2l_t, 0, sizeof(float) * (A.Lmax + 1) * 8 * pp, st);
    cudaMemsetAsync(O.m2l_t, 0, sizeof(float) * (A.Lmax + 1) * NSLOT * pp, st);
    std::vector<GemmSpec> gs;
    for (int l = L0; l <= L1; ++l)
        for (int c = 0; c < 8; ++c) {
            if (l < L1) gs.push_back(GemmSpec{Km2m(l, c), UC(l + 1), O.m2m_t + ((size_t)l * 8 + c) * pp, n, 1});
            if (l > L0) gs.push_back(GemmSpec{Kl2l(l, c), DC(l - 1), O.l2l_t + ((size_t)l * 8 + c) * pp, n, 1});
        }
    GemmSpec *dgs = (GemmSpec *)(dptr + 2 * npi + 2);
    if (!gs.empty()) {
        cudaMemcpyAsync(dgs, gs.data(), sizeof(GemmSpec) * gs.size(), cudaMemcpyHostToDevice, st);
        k_gemm64<<<dim3((n + 15) / 16, (n + 15) / 16, (unsigned)gs.size()), 256, 0, st>>>(dgs, n, np);
    }
    // M2L per level
    std::vector<MatSpec> ms;
    std::vector<GemmSpec> gm;
    for (int l = L0; l <= L1; ++l) {
        double w = half(l);
        for (int slot = 0; slot < NSLOT; ++slot) {
            int ox, oy, oz;
            offsets_of(slot, ox, oy, oz);
            MatSpec m{};
            m.rt = R.dc * w;
            m.cs[0] = 2.0 * w * ox; m.cs[1] = 2.0 * w * oy; m.cs[2] = 2.0 * w * oz;
            m.rs = R.ue * w;
            m.out = km2l + (size_t)slot * nn;
            ms.push_back(m);
            gm.push_back(GemmSpec{km2l + (size_t)slot * nn, UC(l), O.m2l_t + ((size_t)l * NSLOT + slot) * pp, n, 1});
        }
    }
    MatSpec *dm2l = (MatSpec *)(dgs + gs.size() + 2);
    GemmSpec *dgm = (GemmSpec *)(dm2l + ms.size() + 2);
    cudaMemcpyAsync(dm2l, ms.data(), sizeof(MatSpec) * ms.size(), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(dgm, gm.data(), sizeof(GemmSpec) * gm.size(), cudaMemcpyHostToDevice, st);
    for (int l = L0; l <= L1; ++l) {
        size_t k = (size_t)(l - L0) * NSLOT;
        k_kmat<<<dim3((n * n + 255) / 256, NSLOT), 256, 0, st>>>(dm2l + k, O.nodes, n, np, A.alpha, A.beta, C);
        k_gemm64<<<dim3((n + 15) / 16, (n + 15) / 16, NSLOT), 256, 0, st>>>(dgm + k, n, np);
    }
    // L2P tables (padding columns must read as zero)
    cudaMemsetAsync(O.e_tab, 0, sizeof(float) * ops_etab_floats(O.method, np, A.D, A.Lmax), st);
    GemmSpec *dge = dgm + gm.size() + 2;
    int ne = 0;
    for (int l = L0; l <= L1; ++l) {
        if (O.e_off[l] < 0) continue;
        int e = edge_of(A.D, l);
        int rows = e * e * e;
        k_kmat_cells64<<<(rows * n + 255) / 256, 256, 0, st>>>(e, n, 0.5 * A.h, R.de * half(l), O.nodes, A.alpha,
                                                               A.beta, C, kcell);
        GemmSpec g{kcell, DC(l), O.e_tab + O.e_off[l], rows, 0};
        cudaMemcpyAsync(dge + ne, &g, sizeof g, cudaMemcpyHostToDevice, st);
        k_gemm64<<<dim3((n + 15) / 16, (rows + 15) / 16, 1), 256, 0, st>>>(dge + ne, n, np);
        ++ne;
    }
    return 0;
}

// Composed L2L + L2P tables of a child box of edge 4 (FP64 sums of the FP32 operators):
//   C_c[k][cell] = sum_i E[i][cell] L2L_c[i][k]
// E in the L2P table layout [i][cell] (cells of the 4^3 box in local Morton order), L2L_c as
// stored ([k][i], stride npad), output in the L2P table layout, one [npad][64] block per child.
__global__ void k_l2p_compose(const float *__restrict__ etab, const float *__restrict__ l2l, int n, int npad,
                              float *__restrict__ out) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 8 * n * 64) return;
    const int cell = idx % 64, k = (idx / 64) % n, c = idx / (64 * n);
    const float *L = l2l + (size_t)c * npad * npad + (size_t)k * npad;
    double v = 0.0;
    for (int i = 0; i < n; ++i) v += (double)etab[(size_t)i * 64 + cell] * (double)L[i];
    out[(size_t)c * npad * 64 + (size_t)k * 64 + cell] = (float)v;
}

int ops_build(const OpsBuildArgs &A, cudaStream_t st) {
    const OpsDev &O = A.ops;
    const double C = 1.0 / (4.0 * 3.14159265358979323846 * log(A.beta / A.alpha));
    k_nodes_init<<<(O.npad + 127) / 128, 128, 0, st>>>(O.method, O.order, O.n, O.npad, O.nodes, O.cheb_t);
    k_slot_init<<<1, 32, 0, st>>>(O.slot_of_code);
    k_self_int<<<1, 256, 0, st>>>(A.h * cbrt(3.0 / (4.0 * 3.14159265358979323846)), A.alpha, A.beta, O.self_int);
    if (A.Lmax >= 2) {
        if (O.method == FAR_CHEB) build_cheb(A, st, C);
        else build_surface(A, st, C);
        if (O.m2l_img && tc_supported(O)) {
            make_images(O.m2l_t, O.npad, (A.Lmax + 1) * NSLOT, O.m2l_img, st);
            make_images(O.l2l_t, O.npad, (A.Lmax + 1) * 8, O.l2l_img, st);
            if (O.m2m_img) make_images(O.m2m_t, O.npad, (A.Lmax + 1) * 8, O.m2m_img, st);
        }
        if (O.l2p_img && O.method == FAR_CHEB && tc_supported(O)) {
            for (int l = 2; l <= A.Lmax && l < 16; ++l)
                if (O.e_off[l] >= 0 && O.l2p_off[l] >= 0)
                    make_l2p_images(O.e_tab + O.e_off[l], edge_of(A.D, l), O.n, O.l2p_img + O.l2p_off[l], st);
            const int lc = l2pc_level(A.D, A.Lmax);
            if (lc >= 0 && O.l2pc_off >= 0 && O.e_off[lc] >= 0) {
                // composed tables [8][npad][64] in the FP64 work array (used as FP32 scratch: the
                // Chebyshev build keeps nothing there), then their images
                float *comp = reinterpret_cast<float *>(A.work);
                const int total = 8 * O.n * 64;
                k_l2p_compose<<<(total + 255) / 256, 256, 0, st>>>(O.e_tab + O.e_off[lc],
                                                                    O.l2l_t + (size_t)lc * 8 * O.npad * O.npad,
                                                                    O.n, O.npad, comp);
                for (int c = 0; c < 8; ++c)
                    make_l2p_images(comp + (size_t)c * O.npad * 64, 4, O.n,
                                    O.l2p_img + O.l2pc_off + (size_t)c * l2p_image_elems(4), st);
            }
        }
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace sph
