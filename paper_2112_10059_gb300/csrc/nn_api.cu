// C ABI of the learned surrogate (include/sph_nn.h): network object, forward and backward
// passes over the kernels of k_nn.cu, Adam, input preparation.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/sph_nn.h"
#include "nn_internal.h"
#include "nn_kernels.cuh"

using namespace sph::nn;

namespace {

struct LayerSpec {
    const char *name;
    int ci, co, lvl;
};
const LayerSpec LAYERS[12] = {{"c00", 16, 16, 0}, {"c01", 16, 16, 0}, {"c10", 16, 32, 1}, {"c11", 32, 32, 1},
                              {"c20", 32, 32, 2}, {"c21", 32, 32, 2}, {"c30", 32, 32, 3}, {"c31", 32, 32, 3},
                              {"c22", 32, 32, 2}, {"c12", 32, 32, 1}, {"c02", 32, 16, 0}, {"c03", 16, 16, 0}};
enum { C00, C01, C10, C11, C20, C21, C30, C31, C22, C12, C02, C03, NLAYER };
constexpr int HEAD_W = 32, HEAD_N = 34;
constexpr float LOSS_LAMBDA = 0.01f, LOSS_EPS = 1e-4f;

int64_t count_params() {
    int64_t n = 0;
    for (const auto &L : LAYERS) n += (int64_t)L.co * NTAPS * L.ci + L.co;
    return n + HEAD_N;
}

}  // namespace

struct sph_nn {
    int device = 0;
    cudaStream_t stream = nullptr;
    int edge = 0, lg0 = 0, cap = 0;
    std::string err;
    bool poisoned = false;
    int64_t P = 0;
    size_t p_off[NLAYER] = {}, head_off = 0;
    size_t img_f_off[NLAYER] = {}, img_d_off[NLAYER] = {}, dw_off[NLAYER] = {};
    float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr, *dw = nullptr;
    size_t dw_total = 0;
    float *wpart = nullptr;      // [WGRAD_MAX_SPLIT][rows][N] partial weight gradients (fixed-order sums)
    float *hpart = nullptr;      // [HEAD_MAX_BLOCKS][34] partial head gradients
    uint16_t *img = nullptr;
    double *loss = nullptr;
    int *errflag = nullptr;
    unsigned *maxbits = nullptr;
    float *scratch = nullptr;       // pooled fields for input preparation
    size_t scratch_n = 0;
    int step = 0;
    // activations and gradients (BF16), capacity cap samples
    std::vector<void *> allocs;
    uint16_t *a00, *s0, *p0, *a10, *s1, *p1, *a20, *s2, *p2, *a30, *b3, *u2, *d2, *u1, *d1, *u0, *d0, *v0, *f;
    uint16_t *g_f, *g_v0, *g_d0, *g_u0, *g_d1, *g_u1, *g_d2, *g_u2, *g_b3, *g_a30, *g_p2, *g_s2, *g_a20, *g_p1,
        *g_s1, *g_a10, *g_p0, *g_s0, *g_a00;
    float *y = nullptr;
};

namespace {

int fail(sph_nn *n, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (n) n->err = buf;
    return code;
}

int cuda_fail(sph_nn *n, cudaError_t e, const char *where) {
    if (n) n->poisoned = true;
    return fail(n, SPH_ECUDA, "CUDA error in %s: %s", where, cudaGetErrorString(e));
}

#define NCK(call)                                                \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail(n, e_, #call);   \
    } while (0)

template <class T>
int alloc(sph_nn *n, T *&p, size_t count) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T) + 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(n, SPH_ENOMEM, "cudaMalloc of %zu bytes failed", count * sizeof(T));
    }
    n->allocs.push_back(q);
    p = static_cast<T *>(q);
    return SPH_OK;
}

int lg_of(int edge) {
    int lg = 0;
    while ((1 << lg) < edge) ++lg;
    return (1 << lg) == edge ? lg : -1;
}

size_t vox(const sph_nn *n, int batch, int lvl) { return (size_t)batch << (3 * (n->lg0 - lvl)); }

int conv_layer(sph_nn *n, int L, int batch, const uint16_t *in, uint16_t *out, const uint16_t *add, bool dgrad,
               const uint16_t *mask) {
    const LayerSpec &S = LAYERS[L];
    ConvArgs a;
    a.x = in;
    a.w = n->img + (dgrad ? n->img_d_off[L] : n->img_f_off[L]);
    a.bias = dgrad ? nullptr : n->params + n->p_off[L] + (size_t)S.co * NTAPS * S.ci;
    a.add = add;
    a.mask = mask;
    a.out = out;
    a.relu = dgrad ? 0 : 1;
    a.nvox = (int)vox(n, batch, S.lvl);
    a.lg = n->lg0 - S.lvl;
    a.err = n->errflag;
    int r = dgrad ? conv(a, S.co, S.ci, n->stream) : conv(a, S.ci, S.co, n->stream);
    return r ? fail(n, SPH_EINTERNAL, "unsupported layer shape") : SPH_OK;
}

int wgrad_layer(sph_nn *n, int L, int batch, const uint16_t *x, const uint16_t *dz) {
    const LayerSpec &S = LAYERS[L];
    WgradArgs a;
    a.x = x;
    a.dz = dz;
    a.dw = n->dw + n->dw_off[L];
    a.nvox = (int)vox(n, batch, S.lvl);
    a.lg = n->lg0 - S.lvl;
    a.chunks_per_cta = 0;
    a.err = n->errflag;
    a.part = n->wpart;
    return wgrad(a, S.ci, S.co, n->stream) ? fail(n, SPH_EINTERNAL, "unsupported layer shape") : SPH_OK;
}

int refresh_images(sph_nn *n) {
    for (int L = 0; L < NLAYER; ++L)
        make_images(n->params + n->p_off[L], LAYERS[L].ci, LAYERS[L].co, n->img + n->img_f_off[L],
                    n->img + n->img_d_off[L], n->stream);
    NCK(cudaGetLastError());
    return SPH_OK;
}

int forward_pass(sph_nn *n, int B, const uint16_t *x) {
    const int lg0 = n->lg0;
    int r = SPH_OK;
#define RUN(expr)            \
    do {                     \
        r = (expr);          \
        if (r) return r;     \
    } while (0)
    RUN(conv_layer(n, C00, B, x, n->a00, nullptr, false, nullptr));
    RUN(conv_layer(n, C01, B, n->a00, n->s0, nullptr, false, nullptr));
    pool2(n->s0, n->p0, B, lg0 - 1, 16, n->stream);
    RUN(conv_layer(n, C10, B, n->p0, n->a10, nullptr, false, nullptr));
    RUN(conv_layer(n, C11, B, n->a10, n->s1, nullptr, false, nullptr));
    pool2(n->s1, n->p1, B, lg0 - 2, 32, n->stream);
    RUN(conv_layer(n, C20, B, n->p1, n->a20, nullptr, false, nullptr));
    RUN(conv_layer(n, C21, B, n->a20, n->s2, nullptr, false, nullptr));
    pool2(n->s2, n->p2, B, lg0 - 3, 32, n->stream);
    RUN(conv_layer(n, C30, B, n->p2, n->a30, nullptr, false, nullptr));
    RUN(conv_layer(n, C31, B, n->a30, n->b3, nullptr, false, nullptr));
    up_add(n->b3, n->s2, n->u2, B, lg0 - 2, 32, n->stream);
    RUN(conv_layer(n, C22, B, n->u2, n->d2, nullptr, false, nullptr));
    up_add(n->d2, n->s1, n->u1, B, lg0 - 1, 32, n->stream);
    RUN(conv_layer(n, C12, B, n->u1, n->d1, nullptr, false, nullptr));
    up_add(n->d1, nullptr, n->u0, B, lg0, 32, n->stream);
    RUN(conv_layer(n, C02, B, n->u0, n->d0, nullptr, false, nullptr));
    add(n->d0, n->s0, n->v0, vox(n, B, 0) * 16, n->stream);
    RUN(conv_layer(n, C03, B, n->v0, n->f, nullptr, false, nullptr));
    return SPH_OK;
}

int backward_pass(sph_nn *n, int B, const uint16_t *x, const float *t) {
    const int lg0 = n->lg0;
    cudaStream_t st = n->stream;
    int r = SPH_OK;
    NCK(cudaMemsetAsync(n->dw, 0, n->dw_total * sizeof(float), st));
    NCK(cudaMemsetAsync(n->grads + n->head_off, 0, HEAD_N * sizeof(float), st));
    NCK(cudaMemsetAsync(n->loss, 0, sizeof(double), st));
    const float *hw = n->params + n->head_off;
    head_loss_backward(n->f, hw, hw + HEAD_W, t, n->g_f, n->grads + n->head_off, n->loss, (int)vox(n, B, 0),
                       LOSS_LAMBDA, LOSS_EPS, st, n->hpart);
    RUN(wgrad_layer(n, C03, B, n->v0, n->g_f));
    RUN(conv_layer(n, C03, B, n->g_f, n->g_v0, nullptr, true, nullptr));
    mask_mul(n->g_v0, n->d0, n->g_d0, vox(n, B, 0) * 16, st);
    RUN(wgrad_layer(n, C02, B, n->u0, n->g_d0));
    RUN(conv_layer(n, C02, B, n->g_d0, n->g_u0, nullptr, true, nullptr));
    up_back_mask(n->g_u0, n->d1, n->g_d1, B, lg0 - 1, 32, st);
    RUN(wgrad_layer(n, C12, B, n->u1, n->g_d1));
    RUN(conv_layer(n, C12, B, n->g_d1, n->g_u1, nullptr, true, nullptr));
    up_back_mask(n->g_u1, n->d2, n->g_d2, B, lg0 - 2, 32, st);
    RUN(wgrad_layer(n, C22, B, n->u2, n->g_d2));
    RUN(conv_layer(n, C22, B, n->g_d2, n->g_u2, nullptr, true, nullptr));
    up_back_mask(n->g_u2, n->b3, n->g_b3, B, lg0 - 3, 32, st);
    RUN(wgrad_layer(n, C31, B, n->a30, n->g_b3));
    RUN(conv_layer(n, C31, B, n->g_b3, n->g_a30, nullptr, true, n->a30));
    RUN(wgrad_layer(n, C30, B, n->p2, n->g_a30));
    RUN(conv_layer(n, C30, B, n->g_a30, n->g_p2, nullptr, true, nullptr));
    pool_back_add_mask(n->g_p2, n->g_u2, n->s2, n->g_s2, B, lg0 - 2, 32, st);
    RUN(wgrad_layer(n, C21, B, n->a20, n->g_s2));
    RUN(conv_layer(n, C21, B, n->g_s2, n->g_a20, nullptr, true, n->a20));
    RUN(wgrad_layer(n, C20, B, n->p1, n->g_a20));
    RUN(conv_layer(n, C20, B, n->g_a20, n->g_p1, nullptr, true, nullptr));
    pool_back_add_mask(n->g_p1, n->g_u1, n->s1, n->g_s1, B, lg0 - 1, 32, st);
    RUN(wgrad_layer(n, C11, B, n->a10, n->g_s1));
    RUN(conv_layer(n, C11, B, n->g_s1, n->g_a10, nullptr, true, n->a10));
    RUN(wgrad_layer(n, C10, B, n->p0, n->g_a10));
    RUN(conv_layer(n, C10, B, n->g_a10, n->g_p0, nullptr, true, nullptr));
    pool_back_add_mask(n->g_p0, n->g_v0, n->s0, n->g_s0, B, lg0, 16, st);
    RUN(wgrad_layer(n, C01, B, n->a00, n->g_s0));
    RUN(conv_layer(n, C01, B, n->g_s0, n->g_a00, nullptr, true, n->a00));
    RUN(wgrad_layer(n, C00, B, x, n->g_a00));
    for (int L = 0; L < NLAYER; ++L)
        collect_grads(n->dw + n->dw_off[L], LAYERS[L].ci, LAYERS[L].co, n->grads + n->p_off[L], st);
    NCK(cudaGetLastError());
    return SPH_OK;
#undef RUN
}

int check_err(sph_nn *n) {
    int e = 0;
    NCK(cudaMemcpyAsync(&e, n->errflag, sizeof(int), cudaMemcpyDeviceToHost, n->stream));
    NCK(cudaStreamSynchronize(n->stream));
    if (e) return fail(n, SPH_ETIMEOUT, "a tensor-core tile of the network gave up waiting");
    return SPH_OK;
}

uint64_t splitmix(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double normal(uint64_t &s) {
    double u1 = ((splitmix(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    double u2 = (splitmix(s) >> 11) * (1.0 / 9007199254740992.0);
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2);
}

}  // namespace

int sph::nn::net_edge(const sph_nn *n) { return n ? n->edge : 0; }
cudaStream_t sph::nn::net_stream(const sph_nn *n) { return n ? n->stream : nullptr; }
const char *sph::nn::net_error(const sph_nn *n) { return n ? n->err.c_str() : ""; }

extern "C" {

int64_t sph_nn_num_params(void) { return count_params(); }

const char *sph_nn_last_error(const sph_nn *n) { return n ? n->err.c_str() : "null network"; }

void sph_nn_destroy(sph_nn *n) {
    if (!n) return;
    cudaSetDevice(n->device);
    if (n->stream) cudaStreamSynchronize(n->stream);
    for (void *p : n->allocs) cudaFree(p);
    delete n;
}

int sph_nn_create(sph_nn **out, int device, void *stream, int edge, int max_batch) {
    if (!out) return SPH_EINVAL;
    *out = nullptr;
    const int lg = lg_of(edge);
    if (lg < 3 || lg > 8 || max_batch < 1 || max_batch > 64) return SPH_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return SPH_ECUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return SPH_ECUDA;
    sph_nn *n = new (std::nothrow) sph_nn();
    if (!n) return SPH_ENOMEM;
    n->device = device;
    n->stream = static_cast<cudaStream_t>(stream);
    n->edge = edge;
    n->lg0 = lg;
    n->cap = max_batch;
    init_attributes();
    size_t po = 0, io = 0, dwo = 0;
    for (int L = 0; L < NLAYER; ++L) {
        const LayerSpec &S = LAYERS[L];
        n->p_off[L] = po;
        po += (size_t)S.co * NTAPS * S.ci + S.co;
        n->img_f_off[L] = io;
        io += (size_t)conv_chunks(S.ci) * S.co * 64;
        n->img_d_off[L] = io;
        io += (size_t)conv_chunks(S.co) * S.ci * 64;
        n->dw_off[L] = dwo;
        dwo += (size_t)wgrad_rows(S.ci) * S.co;
    }
    n->head_off = po;
    n->P = (int64_t)po + HEAD_N;
    n->dw_total = dwo;
    int r = SPH_OK;
    auto A = [&](auto *&p, size_t cnt) {
        if (!r) r = alloc(n, p, cnt);
    };
    A(n->params, n->P);
    A(n->grads, n->P);
    A(n->m, n->P);
    A(n->v, n->P);
    A(n->dw, dwo);
    A(n->wpart, (size_t)WGRAD_MAX_SPLIT * wgrad_rows(32) * 32);
    A(n->hpart, (size_t)HEAD_MAX_BLOCKS * 34);
    A(n->img, io);
    A(n->loss, 1);
    A(n->errflag, 1);
    A(n->maxbits, 4);
    const int B = max_batch;
    const size_t V0 = vox(n, B, 0), V1 = vox(n, B, 1), V2 = vox(n, B, 2), V3 = vox(n, B, 3);
    A(n->a00, V0 * 16); A(n->s0, V0 * 16); A(n->p0, V1 * 16); A(n->a10, V1 * 32); A(n->s1, V1 * 32);
    A(n->p1, V2 * 32); A(n->a20, V2 * 32); A(n->s2, V2 * 32); A(n->p2, V3 * 32); A(n->a30, V3 * 32);
    A(n->b3, V3 * 32); A(n->u2, V2 * 32); A(n->d2, V2 * 32); A(n->u1, V1 * 32); A(n->d1, V1 * 32);
    A(n->u0, V0 * 32); A(n->d0, V0 * 16); A(n->v0, V0 * 16); A(n->f, V0 * 16);
    A(n->g_f, V0 * 16); A(n->g_v0, V0 * 16); A(n->g_d0, V0 * 16); A(n->g_u0, V0 * 32); A(n->g_d1, V1 * 32);
    A(n->g_u1, V1 * 32); A(n->g_d2, V2 * 32); A(n->g_u2, V2 * 32); A(n->g_b3, V3 * 32); A(n->g_a30, V3 * 32);
    A(n->g_p2, V3 * 32); A(n->g_s2, V2 * 32); A(n->g_a20, V2 * 32); A(n->g_p1, V2 * 32); A(n->g_s1, V1 * 32);
    A(n->g_a10, V1 * 32); A(n->g_p0, V1 * 16); A(n->g_s0, V0 * 16); A(n->g_a00, V0 * 16);
    if (!r) {
        n->scratch_n = 3 * (size_t)edge * edge * edge;
        A(n->scratch, n->scratch_n);
    }
    if (r) {
        sph_nn_destroy(n);
        return r;
    }
    if (cudaMemsetAsync(n->errflag, 0, sizeof(int), n->stream) != cudaSuccess ||
        cudaMemsetAsync(n->params, 0, n->P * sizeof(float), n->stream) != cudaSuccess ||
        cudaMemsetAsync(n->img, 0, io * sizeof(uint16_t), n->stream) != cudaSuccess) {
        sph_nn_destroy(n);
        return SPH_ECUDA;
    }
    *out = n;
    return SPH_OK;
}

int sph_nn_set_params(sph_nn *n, const float *host, int64_t cnt) {
    if (!n || !host || cnt != n->P) return fail(n, SPH_EINVAL, "parameter count must be %lld", (long long)(n ? n->P : 0));
    if (n->poisoned) return SPH_ECUDA;
    NCK(cudaSetDevice(n->device));
    NCK(cudaMemcpyAsync(n->params, host, cnt * sizeof(float), cudaMemcpyHostToDevice, n->stream));
    NCK(cudaMemsetAsync(n->m, 0, cnt * sizeof(float), n->stream));
    NCK(cudaMemsetAsync(n->v, 0, cnt * sizeof(float), n->stream));
    n->step = 0;
    int r = refresh_images(n);
    if (r) return r;
    NCK(cudaStreamSynchronize(n->stream));
    return SPH_OK;
}

int sph_nn_get_params(sph_nn *n, float *host, int64_t cnt) {
    if (!n || !host || cnt != n->P) return fail(n, SPH_EINVAL, "bad parameter buffer");
    if (n->poisoned) return SPH_ECUDA;
    NCK(cudaSetDevice(n->device));
    NCK(cudaMemcpyAsync(host, n->params, cnt * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
    NCK(cudaStreamSynchronize(n->stream));
    return SPH_OK;
}

int sph_nn_get_grads(sph_nn *n, float *host, int64_t cnt) {
    if (!n || !host || cnt != n->P) return fail(n, SPH_EINVAL, "bad gradient buffer");
    if (n->poisoned) return SPH_ECUDA;
    NCK(cudaSetDevice(n->device));
    NCK(cudaMemcpyAsync(host, n->grads, cnt * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
    NCK(cudaStreamSynchronize(n->stream));
    return SPH_OK;
}

int sph_nn_init(sph_nn *n, uint64_t seed) {
    if (!n) return SPH_EINVAL;
    std::vector<float> h(n->P, 0.f);
    uint64_t s = seed;
    for (int L = 0; L < NLAYER; ++L) {
        const LayerSpec &S = LAYERS[L];
        const double sd = std::sqrt(2.0 / (NTAPS * S.ci));
        const size_t nw = (size_t)S.co * NTAPS * S.ci;
        for (size_t i = 0; i < nw; ++i) {
            // first layer: channels >= 4 carry no input; keep their weights zero
            const int c = (int)(i % S.ci);
            const double w = normal(s) * sd;
            h[n->p_off[L] + i] = (L == C00 && c >= 4) ? 0.f : (float)w;
        }
    }
    for (int i = 0; i < HEAD_W; ++i) h[n->head_off + i] = (float)(normal(s) * 0.25 * 0.1);
    h[n->head_off + HEAD_W + 1] = -4.6f;     // error head starts near ln(1e-2)
    return sph_nn_set_params(n, h.data(), n->P);
}

int sph_nn_forward(sph_nn *n, int B, const uint16_t *x, float *y) {
    if (!n || !x || !y || B < 1 || B > n->cap) return fail(n, SPH_EINVAL, "bad forward arguments");
    if (n->poisoned) return SPH_ECUDA;
    NCK(cudaSetDevice(n->device));
    int r = forward_pass(n, B, x);
    if (r) return r;
    const float *hw = n->params + n->head_off;
    head_forward(n->f, hw, hw + HEAD_W, y, (int)vox(n, B, 0), n->stream);
    NCK(cudaGetLastError());
    return SPH_OK;
}

int sph_nn_backward(sph_nn *n, int B, const uint16_t *x, const float *t, double *loss_host) {
    if (!n || !x || !t || B < 1 || B > n->cap) return fail(n, SPH_EINVAL, "bad backward arguments");
    if (n->poisoned) return SPH_ECUDA;
    NCK(cudaSetDevice(n->device));
    int r = forward_pass(n, B, x);
    if (!r) r = backward_pass(n, B, x, t);
    if (r) return r;
    if (loss_host) {
        double l = 0;
        NCK(cudaMemcpyAsync(&l, n->loss, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
        r = check_err(n);
        if (r) return r;
        *loss_host = l / (double)vox(n, B, 0);
    }
    return SPH_OK;
}

int sph_nn_adam(sph_nn *n, float lr, float b1, float b2, float eps) {
    if (!n || !(lr >= 0) || !(b1 >= 0 && b1 < 1) || !(b2 >= 0 && b2 < 1) || !(eps > 0))
        return fail(n, SPH_EINVAL, "bad Adam arguments");
    if (n->poisoned) return SPH_ECUDA;
    NCK(cudaSetDevice(n->device));
    ++n->step;
    const float bc1 = (float)(1.0 - std::pow((double)b1, n->step));
    const float bc2 = (float)(1.0 - std::pow((double)b2, n->step));
    adam(n->params, n->grads, n->m, n->v, (size_t)n->P, lr, b1, b2, eps, bc1, bc2, n->stream);
    return refresh_images(n);
}

int sph_nn_train_step(sph_nn *n, int B, const uint16_t *x, const float *t, float lr, double *loss_host) {
    int r = sph_nn_backward(n, B, x, t, loss_host);
    if (r) return r;
    return sph_nn_adam(n, lr, 0.9f, 0.999f, 1e-8f);
}

int sph_nn_make_inputs(sph_nn *n, int nf, int factor, const float *I, const float *E, const float *S, uint16_t *x) {
    if (!n || !I || !S || !x || factor < 1 || nf != factor * n->edge)
        return fail(n, SPH_EINVAL, "fine grid must be factor * edge");
    if (n->poisoned) return SPH_ECUDA;
    NCK(cudaSetDevice(n->device));
    const size_t nc = (size_t)n->edge * n->edge * n->edge;
    float *Ic = n->scratch, *Im = n->scratch + nc, *Ec = E ? n->scratch + 2 * nc : nullptr;
    pool_avg_f32(I, nf, factor, Ic, n->stream);
    pool_max_f32(I, nf, factor, Im, n->stream);
    if (E) pool_avg_f32(E, nf, factor, Ec, n->stream);
    max4(Ic, Ec, S, Im, nc, n->maxbits, n->stream);
    make_inputs(Ic, Ec, S, Im, n->maxbits, x, nc, n->stream);
    NCK(cudaGetLastError());
    return SPH_OK;
}

int sph_nn_make_target(sph_nn *n, int nf, int factor, const float *Sf, const float *Sc, float *t) {
    if (!n || !Sf || !Sc || !t || factor < 1 || nf != factor * n->edge)
        return fail(n, SPH_EINVAL, "fine grid must be factor * edge");
    if (n->poisoned) return SPH_ECUDA;
    NCK(cudaSetDevice(n->device));
    const size_t nc = (size_t)n->edge * n->edge * n->edge;
    pool_avg_f32(Sf, nf, factor, n->scratch, n->stream);
    make_target(n->scratch, Sc, t, nc, n->stream);
    NCK(cudaGetLastError());
    return SPH_OK;
}

int sph_pool_avg(int device, void *stream, int nf, int factor, const float *fine, float *coarse) {
    if (!fine || !coarse || factor < 1 || nf < factor || nf % factor) return SPH_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return SPH_ECUDA;
    pool_avg_f32(fine, nf, factor, coarse, static_cast<cudaStream_t>(stream));
    return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_ECUDA;
}

int sph_nn_conv3d(int device, void *stream, int mode, int C, int N, int edge, int batch, const uint16_t *x,
                  const float *w, const float *bias, const uint16_t *addp, const uint16_t *mask, int relu,
                  uint16_t *out) {
    const int lg = lg_of(edge);
    if (lg < 0 || lg > 8 || batch < 1 || !x || !w || !out || (mode != 0 && mode != 1)) return SPH_EINVAL;
    if ((C != 16 && C != 32) || (N != 16 && N != 32)) return SPH_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return SPH_ECUDA;
    init_attributes();
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint16_t *img_f = nullptr, *img_d = nullptr;
    int *err = nullptr;
    const size_t nf = (size_t)conv_chunks(C) * N * 64, nd = (size_t)conv_chunks(N) * C * 64;
    if (cudaMalloc(&img_f, (nf + nd) * sizeof(uint16_t)) != cudaSuccess || cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(img_f);
        return SPH_ENOMEM;
    }
    img_d = img_f + nf;
    cudaMemsetAsync(err, 0, sizeof(int), st);
    make_images(w, C, N, img_f, img_d, st);
    ConvArgs a;
    a.x = x;
    a.w = mode == 0 ? img_f : img_d;
    a.bias = mode == 0 ? bias : nullptr;
    a.add = addp;
    a.mask = mask;
    a.out = out;
    a.relu = mode == 0 ? relu : 0;
    a.nvox = batch << (3 * lg);
    a.lg = lg;
    a.err = err;
    int r = mode == 0 ? conv(a, C, N, st) : conv(a, N, C, st);
    int e = 0;
    cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaError_t ce = cudaStreamSynchronize(st);
    cudaFree(img_f);
    cudaFree(err);
    if (ce != cudaSuccess || cudaGetLastError() != cudaSuccess) return SPH_ECUDA;
    if (r) return SPH_EINTERNAL;
    return e ? SPH_ETIMEOUT : SPH_OK;
}

int sph_nn_conv3d_wgrad(int device, void *stream, int C, int N, int edge, int batch, const uint16_t *x,
                        const uint16_t *dz, float *dwout) {
    const int lg = lg_of(edge);
    if (lg < 0 || lg > 8 || batch < 1 || !x || !dz || !dwout) return SPH_EINVAL;
    if ((C != 16 && C != 32) || (N != 16 && N != 32)) return SPH_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return SPH_ECUDA;
    init_attributes();
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float *dw = nullptr;
    int *err = nullptr;
    const size_t rows = wgrad_rows(C);
    if (cudaMalloc(&dw, rows * N * sizeof(float)) != cudaSuccess || cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(dw);
        return SPH_ENOMEM;
    }
    cudaMemsetAsync(dw, 0, rows * N * sizeof(float), st);
    cudaMemsetAsync(err, 0, sizeof(int), st);
    WgradArgs a;
    a.x = x;
    a.dz = dz;
    a.dw = dw;
    a.nvox = batch << (3 * lg);
    a.lg = lg;
    a.chunks_per_cta = 0;
    a.err = err;
    int r = wgrad(a, C, N, st);
    collect_grads(dw, C, N, dwout, st);
    int e = 0;
    cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaError_t ce = cudaStreamSynchronize(st);
    cudaFree(dw);
    cudaFree(err);
    if (ce != cudaSuccess || cudaGetLastError() != cudaSuccess) return SPH_ECUDA;
    if (r) return SPH_EINTERNAL;
    return e ? SPH_ETIMEOUT : SPH_OK;
}

}  // extern "C"
