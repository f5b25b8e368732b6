// Precomputed translation operators of the kernel-independent FMM (paper
// Section 2.4, Eq. s2l and Figure fmulloc): for each tree level l (box
// half-width w_l = h 2^(D-l) / 2) and the current gas (alpha, beta):
//   UC2E_l = pinv(K(upward check, upward equivalent))        radii 2.95 w / 1.05 w
//   DC2E_l = pinv(K(downward check, downward equivalent))    radii 1.05 w / 2.95 w
//   M2M_{l,c} = UC2E_l  * K(parent upward check, child c upward equivalent)
//   L2L_{l,c} = DC2E_l  * K(child c downward check, parent downward equivalent)
//   M2L_{l,o} = K(target downward check, source upward equivalent at offset 2 w o),
//               o in [-3,3]^3 \ [-1,1]^3 (316 offsets)
// G is the photoionization kernel of Eq. gfun; it has two length scales, so
// unlike the Laplace kernel every level needs its own operators.
//
// FP64 is used only here.  The pseudo-inverses solve Eq. s2l in the least-squares
// sense by a truncated SVD computed with one-sided (Hestenes) Jacobi rotations in
// FP64 on the GPU, one CTA per matrix, columns held in shared memory; singular
// values below eps * sigma_max are dropped.
#include <cuda_bf16.h>
#include "sph_kernels.cuh"

namespace sph {

constexpr int P = SPH_P;
constexpr int PPAD = SPH_PP;
constexpr int NSLOT = 316;

__device__ __forceinline__ double g64(double R, double alpha, double beta, double C) {
    return C * exp(-alpha * R) * (-expm1(-(beta - alpha) * R)) / (R * R * R);
}

__global__ void k_surf_init(float *surf) {
    int m = threadIdx.x;
    if (m < P) {
        float x, y, z;
        surf_unit(m, x, y, z);
        surf[4 * m + 0] = x;
        surf[4 * m + 1] = y;
        surf[4 * m + 2] = z;
        surf[4 * m + 3] = 0.f;
    }
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

// Kernel matrix K[i][j] = G(|t_i - s_j|), t_i = ct + rt * u_i, s_j = cs + rs * u_j (cm).
struct MatSpec {
    double ct[3], rt, cs[3], rs;
    double *out;   // row-major P x P
};

__global__ void k_kmat64(const MatSpec *__restrict__ specs, const float *__restrict__ surf, double alpha,
                         double beta, double C) {
    const MatSpec S = specs[blockIdx.y];
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= P * P) return;
    int i = e / P, j = e % P;
    double dx = (S.ct[0] + S.rt * surf[4 * i + 0]) - (S.cs[0] + S.rs * surf[4 * j + 0]);
    double dy = (S.ct[1] + S.rt * surf[4 * i + 1]) - (S.cs[1] + S.rs * surf[4 * j + 1]);
    double dz = (S.ct[2] + S.rt * surf[4 * i + 2]) - (S.cs[2] + S.rs * surf[4 * j + 2]);
    double R = sqrt(dx * dx + dy * dy + dz * dz);
    S.out[e] = g64(R, alpha, beta, C);
}

// Round-robin pairing: round r (0..P-2), pair k (0..P/2-1); every unordered pair once per sweep.
__device__ __forceinline__ void rr_pair(int r, int k, int &p, int &q) {
    const int n1 = P - 1;
    if (k == 0) { p = r; q = n1; }
    else { p = (r + k) % n1; q = (r - k + n1) % n1; }
}

// One CTA per matrix.  K: row-major P x P.  Out: pinv row-major P x P.  Vg: P*P scratch.
__global__ void __launch_bounds__(1024) k_jacobi_pinv(double *const *__restrict__ Ks, double *const *__restrict__ Ps,
                                                     double *__restrict__ Vscratch, double eps, int max_sweeps,
                                                     int *__restrict__ sweeps_used) {
    extern __shared__ double Wsh[];           // column-major W[j*P + i], then inv2[P]
    double *inv2 = Wsh + P * P;
    __shared__ int changed;
    const double *K = Ks[blockIdx.x];
    double *Pout = Ps[blockIdx.x];
    double *V = Vscratch + (size_t)blockIdx.x * P * P;   // column-major
    for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
        int i = e / P, j = e % P;
        Wsh[j * P + i] = K[e];
        V[j * P + i] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) changed = 0;
        __syncthreads();
        for (int r = 0; r < P - 1; ++r) {
            for (int k = warp; k < P / 2; k += nw) {
                int p, q;
                rr_pair(r, k, p, q);
                double *wp = Wsh + p * P, *wq = Wsh + q * P;
                double a = 0, b = 0, g = 0;
                for (int i = lane; i < P; i += 32) {
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
                    for (int i = lane; i < P; i += 32) {
                        double x = wp[i], y = wq[i];
                        wp[i] = c * x - s * y;
                        wq[i] = s * x + c * y;
                    }
                    double *vp = V + p * P, *vq = V + q * P;
                    for (int i = lane; i < P; i += 32) {
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
    // singular values sigma_j = |w_j|; inv2_j = 1/sigma_j^2 above the cutoff
    for (int j = warp; j < P; j += nw) {
        double s = 0;
        for (int i = lane; i < P; i += 32) s = fma(Wsh[j * P + i], Wsh[j * P + i], s);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) inv2[j] = s;   // sigma^2 for now
    }
    __syncthreads();
    __shared__ double smax2;
    if (threadIdx.x == 0) {
        double m = 0;
        for (int j = 0; j < P; ++j) m = fmax(m, inv2[j]);
        smax2 = m;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < P; j += blockDim.x) {
        double s2 = inv2[j];
        inv2[j] = (s2 > eps * eps * smax2 && s2 > 0) ? 1.0 / s2 : 0.0;
    }
    __syncthreads();
    // pinv[i][k] = sum_j V[i][j] W[k][j] / sigma_j^2   (A V = W, A = W V^T)
    for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
        int i = e / P, kk = e % P;
        double acc = 0;
        for (int j = 0; j < P; ++j) acc = fma(V[j * P + i] * inv2[j], Wsh[j * P + kk], acc);
        Pout[e] = acc;
    }
    if (threadIdx.x == 0 && sweeps_used) sweeps_used[blockIdx.x] = sweep;
}

// C = A * B (P x P, FP64, row-major), written as FP32 transposed into out_t[j*PPAD + i].
struct GemmSpec {
    const double *A, *B;
    float *out_t;
};
__global__ void __launch_bounds__(256) k_gemm64_t32(const GemmSpec *__restrict__ specs) {
    const GemmSpec S = specs[blockIdx.z];
    __shared__ double As[16][17], Bs[16][17];
    int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
    int i = blockIdx.y * 16 + ty, j = blockIdx.x * 16 + tx;
    double acc = 0;
    for (int k0 = 0; k0 < P; k0 += 16) {
        As[ty][tx] = (i < P && k0 + tx < P) ? S.A[i * P + k0 + tx] : 0.0;
        Bs[ty][tx] = (k0 + ty < P && j < P) ? S.B[(k0 + ty) * P + j] : 0.0;
        __syncthreads();
        for (int k = 0; k < 16; ++k) acc = fma(As[ty][k], Bs[k][tx], acc);
        __syncthreads();
    }
    if (i < P && j < P) S.out_t[j * PPAD + i] = (float)acc;
}

// FP64 row-major P x P -> FP32 transposed padded
__global__ void k_to_f32t(const double *__restrict__ A, float *__restrict__ out_t) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= P * P) return;
    int i = e / P, j = e % P;
    out_t[j * PPAD + i] = (float)A[e];
}

// M2L operators of one level: [slot][j][i] FP32 and, if bf != nullptr, BF16 hi/lo [slot][part][i][k].
__global__ void k_m2l_build(const float *__restrict__ surf, double w, double alpha, double beta, double C,
                            float *__restrict__ m2l_t, uint16_t *__restrict__ bf) {
    int slot = blockIdx.y;
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= P * P) return;
    // decode slot -> offset
    int s = 0, code = 0;
    for (int c = 0; c < SPH_NOFF; ++c) {
        int ox = c % 7 - 3, oy = (c / 7) % 7 - 3, oz = c / 49 - 3;
        if (abs(ox) <= 1 && abs(oy) <= 1 && abs(oz) <= 1) continue;
        if (s == slot) { code = c; break; }
        ++s;
    }
    int ox = code % 7 - 3, oy = (code / 7) % 7 - 3, oz = code / 49 - 3;
    int i = e / P, j = e % P;   // i: target check point, j: source equivalent point
    double rt = R_DC * w, rs = R_UE * w;
    double dx = rt * surf[4 * i + 0] - (2.0 * w * ox + rs * surf[4 * j + 0]);
    double dy = rt * surf[4 * i + 1] - (2.0 * w * oy + rs * surf[4 * j + 1]);
    double dz = rt * surf[4 * i + 2] - (2.0 * w * oz + rs * surf[4 * j + 2]);
    double R = sqrt(dx * dx + dy * dy + dz * dz);
    double g = g64(R, alpha, beta, C);
    m2l_t[(size_t)slot * PPAD * PPAD + j * PPAD + i] = (float)g;
    if (bf) {
        float gf = (float)g;
        __nv_bfloat16 hi = __float2bfloat16_rn(gf);
        __nv_bfloat16 lo = __float2bfloat16_rn(gf - __bfloat162float(hi));
        size_t base = (size_t)slot * 2 * PPAD * PPAD;
        bf[base + i * PPAD + j] = __bfloat16_as_ushort(hi);
        bf[base + PPAD * PPAD + i * PPAD + j] = __bfloat16_as_ushort(lo);
    }
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

size_t ops_work_doubles(int Lmax) {
    // per level: Kuc, Kdc, UC2E, DC2E, 8 Km2m, 8 Kl2l (20 P*P, 2 spare); then 22 P*P of
    // Jacobi scratch (one P*P per pseudo-inverse) and 64 Ki doubles for launch tables
    return (size_t)(Lmax + 2) * 22 * P * P + 64 * 1024;
}

int ops_build(const OpsBuildArgs &A, cudaStream_t st) {
    const OpsDev &O = A.ops;
    const double C = 1.0 / (4.0 * 3.14159265358979323846 * log(A.beta / A.alpha));
    k_surf_init<<<1, 160, 0, st>>>(O.surf);
    k_slot_init<<<1, 32, 0, st>>>(O.slot_of_code);
    k_self_int<<<1, 256, 0, st>>>(A.h * cbrt(3.0 / (4.0 * 3.14159265358979323846)), A.alpha, A.beta, O.self_int);
    const int L0 = 2, L1 = A.Lmax;   // operators are used on levels >= 2
    if (L1 < L0) return cudaGetLastError() == cudaSuccess ? 0 : -1;
    const size_t PP2 = (size_t)P * P;
    double *work = A.work;
    auto Kuc = [&](int l) { return work + ((size_t)l * 22 + 0) * PP2; };
    auto Kdc = [&](int l) { return work + ((size_t)l * 22 + 1) * PP2; };
    auto UC = [&](int l) { return work + ((size_t)l * 22 + 2) * PP2; };
    auto DC = [&](int l) { return work + ((size_t)l * 22 + 3) * PP2; };
    auto Km2m = [&](int l, int c) { return work + ((size_t)l * 22 + 4 + c) * PP2; };
    auto Kl2l = [&](int l, int c) { return work + ((size_t)l * 22 + 12 + c) * PP2; };
    double *jacobi_scratch = work + (size_t)(A.Lmax + 1) * 22 * PP2;
    auto half = [&](int l) { return A.h * (double)(1 << (A.D - l)) * 0.5; };

    // host-side spec tables (small), copied with the stream
    const int nl = L1 - L0 + 1;
    int nspec = 0;
    MatSpec specs[11 * 18];
    for (int l = L0; l <= L1; ++l) {
        double w = half(l);
        MatSpec s{};
        s.rt = R_UC * w; s.rs = R_UE * w; s.out = Kuc(l);
        specs[nspec++] = s;
        s = MatSpec{};
        s.rt = R_DC * w; s.rs = R_DE * w; s.out = Kdc(l);
        specs[nspec++] = s;
        for (int c = 0; c < 8; ++c) {
            double cw = w * 0.5;   // child half-width
            double off[3] = {((c & 1) ? 1 : -1) * cw, ((c & 2) ? 1 : -1) * cw, ((c & 4) ? 1 : -1) * cw};
            if (l < L1) {   // M2M: child (l+1) upward equivalent -> parent (l) upward check
                MatSpec m{};
                m.rt = R_UC * w;
                for (int d = 0; d < 3; ++d) m.cs[d] = off[d];
                m.rs = R_UE * cw;
                m.out = Km2m(l, c);
                specs[nspec++] = m;
            }
            if (l > L0) {   // L2L: parent (l-1) downward equivalent -> child (l) downward check
                double pw = 2.0 * w;
                double coff[3] = {((c & 1) ? 1 : -1) * w, ((c & 2) ? 1 : -1) * w, ((c & 4) ? 1 : -1) * w};
                MatSpec m{};
                for (int d = 0; d < 3; ++d) m.ct[d] = coff[d];
                m.rt = R_DC * w;
                m.rs = R_DE * pw;
                m.out = Kl2l(l, c);
                specs[nspec++] = m;
            }
        }
    }
    MatSpec *dspecs = (MatSpec *)(jacobi_scratch + 22 * PP2);   // launch tables
    cudaMemcpyAsync(dspecs, specs, sizeof(MatSpec) * nspec, cudaMemcpyHostToDevice, st);
    k_kmat64<<<dim3((P * P + 255) / 256, nspec), 256, 0, st>>>(dspecs, O.surf, A.alpha, A.beta, C);

    // pseudo-inverses: 2 per level
    double *kin[22], *pout[22];
    int np = 0;
    for (int l = L0; l <= L1; ++l) {
        kin[np] = Kuc(l); pout[np] = UC(l); ++np;
        kin[np] = Kdc(l); pout[np] = DC(l); ++np;
    }
    double **dptr = (double **)(dspecs + nspec + 1);
    cudaMemcpyAsync(dptr, kin, sizeof(double *) * np, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(dptr + np, pout, sizeof(double *) * np, cudaMemcpyHostToDevice, st);
    size_t smem = (size_t)P * P * sizeof(double) + P * sizeof(double);
    cudaFuncSetAttribute(k_jacobi_pinv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_jacobi_pinv<<<np, 1024, smem, st>>>(dptr, dptr + np, jacobi_scratch, A.eps, 40,
                                          nullptr);

    // FP32 transposed copies and composed M2M / L2L
    cudaMemsetAsync(O.uc2e_t, 0, sizeof(float) * (A.Lmax + 1) * PPAD * PPAD, st);
    cudaMemsetAsync(O.dc2e_t, 0, sizeof(float) * (A.Lmax + 1) * PPAD * PPAD, st);
    cudaMemsetAsync(O.m2m_t, 0, sizeof(float) * (A.Lmax + 1) * 8 * PPAD * PPAD, st);
    cudaMemsetAsync(O.l2l_t, 0, sizeof(float) * (A.Lmax + 1) * 8 * PPAD * PPAD, st);
    GemmSpec gs[11 * 16];
    int ng = 0;
    for (int l = L0; l <= L1; ++l) {
        k_to_f32t<<<(P * P + 255) / 256, 256, 0, st>>>(UC(l), O.uc2e_t + (size_t)l * PPAD * PPAD);
        k_to_f32t<<<(P * P + 255) / 256, 256, 0, st>>>(DC(l), O.dc2e_t + (size_t)l * PPAD * PPAD);
        for (int c = 0; c < 8; ++c) {
            if (l < L1) gs[ng++] = GemmSpec{UC(l), Km2m(l, c), O.m2m_t + ((size_t)l * 8 + c) * PPAD * PPAD};
            if (l > L0) gs[ng++] = GemmSpec{DC(l), Kl2l(l, c), O.l2l_t + ((size_t)l * 8 + c) * PPAD * PPAD};
        }
    }
    if (ng > 0) {
        GemmSpec *dgs = (GemmSpec *)(dptr + 2 * np);
        cudaMemcpyAsync(dgs, gs, sizeof(GemmSpec) * ng, cudaMemcpyHostToDevice, st);
        k_gemm64_t32<<<dim3((P + 15) / 16, (P + 15) / 16, ng), 256, 0, st>>>(dgs);
    }
    // M2L per level
    cudaMemsetAsync(O.m2l_t, 0, sizeof(float) * (A.Lmax + 1) * NSLOT * PPAD * PPAD, st);
    if (O.m2l_bf) cudaMemsetAsync(O.m2l_bf, 0, sizeof(uint16_t) * (A.Lmax + 1) * NSLOT * 2 * PPAD * PPAD, st);
    for (int l = L0; l <= L1; ++l) {
        k_m2l_build<<<dim3((P * P + 255) / 256, NSLOT), 256, 0, st>>>(
            O.surf, half(l), A.alpha, A.beta, C, O.m2l_t + (size_t)l * NSLOT * PPAD * PPAD,
            O.m2l_bf ? O.m2l_bf + (size_t)l * NSLOT * 2 * PPAD * PPAD : nullptr);
    }
    (void)nl;
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace sph
