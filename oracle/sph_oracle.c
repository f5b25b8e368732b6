/*
 * FP64 CPU oracle for the photoionization source S_ph.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU path computes.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark may build, load or call it;
 * the product library never links it and shares no code with it.
 *
 * What it computes (paper Section 2.1 and Section 2.4):
 *   Eq. integral: S_ph(x) = \iiint I(y) g(|x-y|) / (4 pi |x-y|^2) dy
 *   Eq. gfun:     g(r) = p_O2 (e^{-chi_min p_O2 r} - e^{-chi_max p_O2 r}) / (p_O2 r ln(chi_max/chi_min))
 *   Eq. summation: S_ph(x_i) = sum_j G(x_i, y_j) I_h(y_j), I_h = I * (cell volume)
 * With alpha = chi_min p_O2, beta = chi_max p_O2, L = ln(beta/alpha) the
 * discrete kernel between distinct cell centres is
 *   G(R) = (e^{-alpha R} - e^{-beta R}) / (4 pi L R^3),
 * evaluated in the cancellation-free form e^{-alpha R} * (-expm1(-(beta-alpha) R)).
 * The cell's own contribution (R = 0) is the integral of G over a ball with
 * the cell's volume, radius a = h (3/(4 pi))^{1/3}:
 *   int_ball G dV = int_0^a (e^{-alpha r} - e^{-beta r}) / (L r) dr
 *                 = 1 - (E1(alpha a) - E1(beta a)) / L,
 * so the self term is I(x) times that number.
 *
 * Selection (Section 3, Eq. summationI and Eq. sourcepct; Section 5 target rule):
 *   sources  J = { n : q[n] >= i_frac * max q }     (i_frac == 0: every cell)
 *   targets  T = { n : |E|[n] >= e_app + e_frac (max|E| - e_app) }, or an explicit mask,
 * every comparison in FP64 on FP32 inputs promoted to double.
 *
 * Parity pins (tests/test_oracle_pins.py): high-precision evaluation of Eq. gfun,
 * quadrature of the self integral, photon conservation (int G dV = 1), the
 * spherical-source radial integral, reciprocity, translation, linearity,
 * brute force in extended precision, and an FFT convolution of the same sum.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define O_PI 3.14159265358979323846
#define O_EULER 0.57721566490153286061

/* Eq. gfun divided by 4 pi R^2 (the discrete kernel between distinct cells). */
double oracle_G(double R, double alpha, double beta)
{
    double L = log(beta / alpha);
    return exp(-alpha * R) * (-expm1(-(beta - alpha) * R)) / (4.0 * O_PI * L * R * R * R);
}

/* Exponential integral E1(x), x > 0.
 * x <= 1: power series E1(x) = -gamma - ln x - sum_{k>=1} (-x)^k / (k k!)  (A&S 5.1.11).
 * x > 1 : continued fraction E1(x) = e^{-x} / (x+1 - 1/(x+3 - 4/(x+5 - 9/(x+7 - ...))))
 *         (even form of A&S 5.1.22), evaluated from the tail backwards. */
double oracle_E1(double x)
{
    if (x <= 0.0) return INFINITY;
    if (x <= 1.0) {
        double term = 1.0, sum = 0.0;
        for (int k = 1; k < 200; ++k) {
            term *= -x / (double)k;
            double add = term / (double)k;
            sum += add;
            if (fabs(add) < 1e-18 * fabs(sum)) break;
        }
        return -O_EULER - log(x) - sum;
    }
    double t = 0.0;
    for (int k = 400; k >= 1; --k) {
        double kk = (double)k;
        t = kk * kk / (x + 2.0 * kk + 1.0 - t);
    }
    return exp(-x) / (x + 1.0 - t);
}

/* int over a ball of radius a of G dV = 1 - (E1(alpha a) - E1(beta a))/L (dimensionless). */
double oracle_self_integral(double a, double alpha, double beta)
{
    double L = log(beta / alpha);
    return 1.0 - (oracle_E1(alpha * a) - oracle_E1(beta * a)) / L;
}

/* Radius of the ball whose volume is one cell, h^3. */
double oracle_self_radius(double h)
{
    return h * cbrt(3.0 / (4.0 * O_PI));
}

/* Selection (Section 3).  Outputs ascending linear indices.  Returns 0. */
int oracle_select(int64_t ncell, const float *q, const float *emag, const uint8_t *mask,
                  double i_frac, double e_frac, double e_app,
                  int32_t *J, int64_t *nJ, int32_t *T, int64_t *nT)
{
    int64_t cj = 0, ct = 0;
    if (i_frac == 0.0) {
        for (int64_t n = 0; n < ncell; ++n) J[cj++] = (int32_t)n;
    } else {
        double qmax = -INFINITY;
        for (int64_t n = 0; n < ncell; ++n)
            if ((double)q[n] > qmax) qmax = (double)q[n];
        if (qmax > 0.0) {
            double thr = i_frac * qmax;
            for (int64_t n = 0; n < ncell; ++n)
                if ((double)q[n] >= thr) J[cj++] = (int32_t)n;
        }
    }
    if (mask) {
        for (int64_t n = 0; n < ncell; ++n)
            if (mask[n]) T[ct++] = (int32_t)n;
    } else if (emag) {
        double emax = -INFINITY;
        for (int64_t n = 0; n < ncell; ++n)
            if ((double)emag[n] > emax) emax = (double)emag[n];
        double thr = e_app + e_frac * (emax - e_app);
        for (int64_t n = 0; n < ncell; ++n)
            if ((double)emag[n] >= thr) T[ct++] = (int32_t)n;
    } else {
        for (int64_t n = 0; n < ncell; ++n) T[ct++] = (int32_t)n;
    }
    *nJ = cj;
    *nT = ct;
    return 0;
}

/* Neumaier-compensated accumulation. */
static inline void neumaier_add(double *sum, double *comp, double v)
{
    double t = *sum + v;
    if (fabs(*sum) >= fabs(v)) *comp += (*sum - t) + v;
    else *comp += (v - t) + *sum;
    *sum = t;
}

/* Eq. summation restricted to the selected sets (Eq. summationI):
 *   S[t] = sum_{s in J, s != t} G(R_ts) I_h[s] + [t in J] I[t] * self_integral
 * for every t in T (in the order given), I_h = source_scale * q * h^3,
 * R_ts = h * |integer cell offset|.  J must be ascending.  S has nT entries.
 * self_mode 0 drops the self term. */
int oracle_sph(int nx, int ny, int nz, double h, double alpha, double beta,
               const float *q, double source_scale,
               const int32_t *J, int64_t nJ, const int32_t *T, int64_t nT,
               int self_mode, double *S)
{
    const double vol = h * h * h;
    const double self_int = oracle_self_integral(oracle_self_radius(h), alpha, beta);
    int64_t t;
#pragma omp parallel for schedule(dynamic, 16)
    for (t = 0; t < nT; ++t) {
        int32_t nt = T[t];
        int it = nt % nx, jt = (nt / nx) % ny, kt = nt / (nx * ny);
        double sum = 0.0, comp = 0.0;
        int self_in_J = 0;
        for (int64_t s = 0; s < nJ; ++s) {
            int32_t ns = J[s];
            if (ns == nt) { self_in_J = 1; continue; }
            int is = ns % nx, js = (ns / nx) % ny, ks = ns / (nx * ny);
            double di = (double)(it - is), dj = (double)(jt - js), dk = (double)(kt - ks);
            double R = h * sqrt(di * di + dj * dj + dk * dk);
            double Ih = source_scale * (double)q[ns] * vol;
            neumaier_add(&sum, &comp, oracle_G(R, alpha, beta) * Ih);
        }
        if (self_in_J && self_mode == 1)
            neumaier_add(&sum, &comp, source_scale * (double)q[nt] * self_int);
        S[t] = sum + comp;
    }
    (void)nz;
    return 0;
}

/* Same sum with the pair kernel evaluated in long double (extended precision on
 * x86 and __float128-class quad on aarch64), plain summation in long double.
 * Used only on tiny grids as a brute-force check of oracle_sph. */
int oracle_sph_longdouble(int nx, int ny, int nz, double h, double alpha, double beta,
                          const float *q, double source_scale,
                          const int32_t *J, int64_t nJ, const int32_t *T, int64_t nT,
                          int self_mode, double self_int, double *S)
{
    long double hl = h, al = alpha, bl = beta;
    long double L = logl(bl / al);
    long double vol = hl * hl * hl;
    for (int64_t t = 0; t < nT; ++t) {
        int32_t nt = T[t];
        int it = nt % nx, jt = (nt / nx) % ny, kt = nt / (nx * ny);
        long double sum = 0.0L;
        for (int64_t s = 0; s < nJ; ++s) {
            int32_t ns = J[s];
            if (ns == nt) {
                if (self_mode == 1) sum += (long double)source_scale * (long double)q[nt] * (long double)self_int;
                continue;
            }
            int is = ns % nx, js = (ns / nx) % ny, ks = ns / (nx * ny);
            long double d2 = (long double)((it - is) * (it - is) + (jt - js) * (jt - js) + (kt - ks) * (kt - ks));
            long double R = hl * sqrtl(d2);
            long double G = (expl(-al * R) - expl(-bl * R)) / (4.0L * (long double)O_PI * L * R * R * R);
            sum += G * (long double)source_scale * (long double)q[ns] * vol;
        }
        S[t] = (double)sum;
    }
    (void)nz;
    return 0;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the OpenMP loops from now on (timing of the single-thread rate). */
void oracle_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
