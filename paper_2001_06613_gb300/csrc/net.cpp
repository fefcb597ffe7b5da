// Learned temporal predictor: host runtime of the network (buffers, the
// forward and backward launch sequences, Adam) and its C interface.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/stml_net.h"
#include "kernels.h"
#include "net.h"

using namespace stml;
using namespace stml::net;

namespace {

struct LayerDef {
    int cin_real, cin, cout, level;
};
// e0a e0b e1a e1b e2a e2b ba bb d2a d2b d1a d1b d0a d0b (the order of the parameter vector)
constexpr LayerDef kDefs[kLayers] = {
    {7, 32, 32, 0},     {32, 32, 32, 0},   {32, 32, 64, 1},   {64, 64, 64, 1},   {64, 64, 96, 2},
    {96, 96, 96, 2},    {96, 96, 128, 3},  {128, 128, 128, 3}, {224, 224, 96, 2}, {96, 96, 96, 2},
    {160, 160, 64, 1},  {64, 64, 64, 1},   {96, 96, 32, 0},   {32, 32, 32, 0}};
enum { E0A, E0B, E1A, E1B, E2A, E2B, BA, BB, D2A, D2B, D1A, D1B, D0A, D0B };

constexpr long long layer_w(int l) { return 9LL * kDefs[l].cin_real * kDefs[l].cout; }
constexpr long long param_total() {
    long long n = 0;
    for (int l = 0; l < kLayers; ++l) n += layer_w(l) + kDefs[l].cout;
    return n + kHeadIn * kOutCh + kOutCh;
}
constexpr long long kParams = param_total();
static_assert(kParams == 906274, "parameter count");

inline int pad8(int n) { return (n + 7) / 8 * 8; }

}  // namespace

struct stml_net {
    cudaStream_t stream = nullptr;
    int device = 0;
    int maxB = 0, maxH8 = 0, maxW8 = 0;
    long long P0 = 0;                    // maxB * maxH8 * maxW8
    long long w_off[kLayers] = {}, b_off[kLayers] = {}, head_off = 0;
    float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    bf16* wbuf = nullptr;
    PackTable pt{};
    // activations, channels-last BF16 (level l has P0 / 4^l pixels)
    bf16* act[kLayers] = {};
    bf16 *x0 = nullptr, *pool[3] = {};
    float *base = nullptr, *tgt = nullptr;
    // backward buffers
    bf16 *gz1 = nullptr, *gz2 = nullptr;
    float *fup = nullptr, *skip[3] = {}, *dp = nullptr;
    float *wpart = nullptr, *bpart = nullptr, *hpart = nullptr;
    size_t wpart_cap = 0, bpart_cap = 0;
    double *loss_d = nullptr, *loss_h = nullptr;
    int *err_d = nullptr, *err_h = nullptr;      // set by a convolution whose bounded wait expired
    Sample *smp_d = nullptr, *smp_h = nullptr;
    cudaEvent_t smp_ev = nullptr;
    bool smp_pending = false;
    long long step = 0;
    std::string err;
};

namespace {

stml_status net_fail(stml_net* n, stml_status s, const std::string& msg) {
    if (n) n->err = msg;
    else set_context_free_error(msg);
    return s;
}

#define NCK(net, call)                                                     \
    do {                                                                   \
        cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess)                                             \
            return net_fail(net, STML_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// the same, inside functions that return cudaError_t
#define ECK(call)                            \
    do {                                     \
        cudaError_t e_ = (call);             \
        if (e_ != cudaSuccess) return e_;    \
    } while (0)

template <typename T>
cudaError_t nalloc(T** p, size_t count) {
    return cudaMalloc(reinterpret_cast<void**>(p), (count ? count : 1) * sizeof(T));
}

void free_all(stml_net* n) {
    auto f = [](auto*& p) {
        if (p) cudaFree(p);
        p = nullptr;
    };
    f(n->theta); f(n->m); f(n->v); f(n->grad); f(n->wbuf);
    for (auto& a : n->act) f(a);
    f(n->x0);
    for (auto& a : n->pool) f(a);
    f(n->base); f(n->tgt); f(n->gz1); f(n->gz2); f(n->fup);
    for (auto& a : n->skip) f(a);
    f(n->dp); f(n->wpart); f(n->bpart); f(n->hpart); f(n->loss_d); f(n->smp_d); f(n->err_d);
    if (n->loss_h) cudaFreeHost(n->loss_h);
    if (n->err_h) cudaFreeHost(n->err_h);
    n->err_h = nullptr;
    if (n->smp_h) cudaFreeHost(n->smp_h);
    n->loss_h = nullptr;
    n->smp_h = nullptr;
    if (n->smp_ev) cudaEventDestroy(n->smp_ev);
    n->smp_ev = nullptr;
}

cudaError_t alloc_all(stml_net* n) {
    const long long P0 = n->P0;
    long long o = 0;
    for (int l = 0; l < kLayers; ++l) {
        n->w_off[l] = o;
        o += layer_w(l);
        n->b_off[l] = o;
        o += kDefs[l].cout;
    }
    n->head_off = o;
    ECK(nalloc(&n->theta, kParams));
    ECK(nalloc(&n->m, kParams));
    ECK(nalloc(&n->v, kParams));
    ECK(nalloc(&n->grad, kParams));
    long long wtot = 0;
    for (int l = 0; l < kLayers; ++l) wtot += 9LL * kDefs[l].cin * kDefs[l].cout * (l == E0A ? 1 : 2);
    ECK(nalloc(&n->wbuf, wtot));
    bf16* w = n->wbuf;
    n->pt.n = kLayers;
    for (int l = 0; l < kLayers; ++l) {
        n->pt.cin_real[l] = kDefs[l].cin_real;
        n->pt.cin[l] = kDefs[l].cin;
        n->pt.cout[l] = kDefs[l].cout;
        n->pt.w_off[l] = n->w_off[l];
        n->pt.wf[l] = w;
        w += 9LL * kDefs[l].cin * kDefs[l].cout;
        n->pt.wd[l] = l == E0A ? nullptr : w;
        if (l != E0A) w += 9LL * kDefs[l].cin * kDefs[l].cout;
    }
    ECK(nalloc(&n->err_d, 1));
    ECK(cudaMemset(n->err_d, 0, sizeof(int)));
    ECK(cudaMallocHost(reinterpret_cast<void**>(&n->err_h), sizeof(int)));
    for (int l = 0; l < kLayers; ++l)
        ECK(nalloc(&n->act[l], (size_t)((P0 >> (2 * kDefs[l].level)) * kDefs[l].cout)));
    ECK(nalloc(&n->x0, (size_t)(P0 * kInPad)));
    ECK(nalloc(&n->pool[0], (size_t)((P0 >> 2) * 32)));
    ECK(nalloc(&n->pool[1], (size_t)((P0 >> 4) * 64)));
    ECK(nalloc(&n->pool[2], (size_t)((P0 >> 6) * 96)));
    ECK(nalloc(&n->base, (size_t)(P0 * 2)));
    ECK(nalloc(&n->tgt, (size_t)(P0 * 2)));
    ECK(nalloc(&n->gz1, (size_t)(P0 * 32)));
    ECK(nalloc(&n->gz2, (size_t)(P0 * 32)));
    ECK(nalloc(&n->fup, (size_t)(P0 * 64)));
    ECK(nalloc(&n->skip[0], (size_t)(P0 * 32)));
    ECK(nalloc(&n->skip[1], (size_t)((P0 >> 2) * 64)));
    ECK(nalloc(&n->skip[2], (size_t)((P0 >> 4) * 96)));
    ECK(nalloc(&n->dp, (size_t)((P0 >> 2) * 32)));
    n->wpart_cap = 4u << 20;
    n->bpart_cap = 256 * 128;
    ECK(nalloc(&n->wpart, n->wpart_cap));
    ECK(nalloc(&n->bpart, n->bpart_cap));
    ECK(nalloc(&n->hpart, 1024 * 67));
    ECK(nalloc(&n->loss_d, 1));
    ECK(nalloc(&n->smp_d, (size_t)n->maxB));
    ECK(cudaMallocHost(reinterpret_cast<void**>(&n->loss_h), sizeof(double)));
    ECK(cudaMallocHost(reinterpret_cast<void**>(&n->smp_h), sizeof(Sample) * n->maxB));
    ECK(cudaEventCreateWithFlags(&n->smp_ev, cudaEventDisableTiming));
    return cudaSuccess;
}

cudaError_t upload_params(stml_net* n, const float* host) {
    ECK(cudaMemcpyAsync(n->theta, host, kParams * sizeof(float), cudaMemcpyHostToDevice, n->stream));
    ECK(cudaMemsetAsync(n->m, 0, kParams * sizeof(float), n->stream));
    ECK(cudaMemsetAsync(n->v, 0, kParams * sizeof(float), n->stream));
    n->step = 0;
    ECK(launch_pack(n->theta, n->pt, n->stream));
    count_launches(1);
    return cudaStreamSynchronize(n->stream);
}

// Copies B descriptors to the device (waiting until the previous copy of the
// pinned staging array has been consumed).
cudaError_t upload_samples(stml_net* n, const Sample* smp, int B, cudaStream_t s) {
    if (n->smp_pending) ECK(cudaEventSynchronize(n->smp_ev));
    std::memcpy(n->smp_h, smp, sizeof(Sample) * B);
    ECK(cudaMemcpyAsync(n->smp_d, n->smp_h, sizeof(Sample) * B, cudaMemcpyHostToDevice, s));
    ECK(cudaEventRecord(n->smp_ev, s));
    n->smp_pending = true;
    return cudaSuccess;
}

ConvIn cin1(const bf16* a, int ca) { return ConvIn{a, ca, 0, nullptr, 0}; }
ConvIn cin2(const bf16* a, int ca, const bf16* b, int cb) { return ConvIn{a, ca, 1, b, cb}; }

// Input of every layer in the forward pass.
ConvIn layer_input(const stml_net* n, int l) {
    switch (l) {
        case E0A: return cin1(n->x0, kInPad);
        case E1A: return cin1(n->pool[0], 32);
        case E2A: return cin1(n->pool[1], 64);
        case BA: return cin1(n->pool[2], 96);
        case D2A: return cin2(n->act[BB], 128, n->act[E2B], 96);
        case D1A: return cin2(n->act[D2B], 96, n->act[E1B], 64);
        case D0A: return cin2(n->act[D1B], 64, n->act[E0B], 32);
        default: return cin1(n->act[l - 1], kDefs[l].cin);
    }
}

cudaError_t forward_pass(stml_net* n, int B, int H, int W, bool train, cudaStream_t s) {
    const int H8 = pad8(H), W8 = pad8(W);
    ECK(launch_assemble(n->smp_d, B, H, W, H8, W8, n->x0, n->base, train ? n->tgt : nullptr, s));
    int launches = 1;
    for (int l = 0; l < kLayers; ++l) {
        const int lv = kDefs[l].level;
        if (l == E1A || l == E2A || l == BA) {
            const int pl = lv - 1;
            ECK(launch_pool2(n->act[l - 1], n->pool[pl], B, H8 >> pl, W8 >> pl, kDefs[l].cin, s));
            ++launches;
        }
        ConvOut o{CONV_FWD, n->theta + n->b_off[l], n->act[l], nullptr, nullptr, nullptr, 0};
        ECK(launch_conv3(layer_input(n, l), n->pt.wf[l], kDefs[l].cin, kDefs[l].cout, B, H8 >> lv, W8 >> lv, o,
                         n->err_d, s));
        ++launches;
    }
    count_launches(launches);
    return cudaSuccess;
}

// Weight and bias gradients of layer l from its dY' (G) into n->grad.
cudaError_t layer_wgrad(stml_net* n, int l, const bf16* G, int B, int H8, int W8, cudaStream_t s) {
    const int lv = kDefs[l].level;
    const int H = H8 >> lv, W = W8 >> lv;
    int ws = 0, bs = 0;
    ECK(launch_wgrad3(layer_input(n, l), G, kDefs[l].cin, kDefs[l].cout, B, H, W, n->wpart, n->wpart_cap, &ws,
                      n->err_d, s));
    ECK(launch_colsum(G, (long long)B * H * W, kDefs[l].cout, n->bpart, n->bpart_cap, &bs, s));
    ECK(launch_reduce_grad(n->wpart, ws, kDefs[l].cin, kDefs[l].cin_real, kDefs[l].cout, n->bpart, bs, n->grad,
                           n->w_off[l], n->b_off[l], s));
    count_launches(3);
    return cudaSuccess;
}

// Input gradient of layer l from its dY' (G): flipped weights, epilogue `o`.
cudaError_t layer_dgrad(stml_net* n, int l, const bf16* G, int B, int H8, int W8, const ConvOut& o,
                        cudaStream_t s) {
    const int lv = kDefs[l].level;
    count_launches(1);
    return launch_conv3(cin1(G, kDefs[l].cout), n->pt.wd[l], kDefs[l].cout, kDefs[l].cin, B, H8 >> lv, W8 >> lv,
                        o, n->err_d, s);
}

ConvOut mask_out(bf16* y, const bf16* mask) { return ConvOut{CONV_MASK, nullptr, y, mask, nullptr, nullptr, 0}; }
ConvOut split_out(float* f1, int n1, float* f2) { return ConvOut{CONV_SPLIT, nullptr, nullptr, nullptr, f1, f2, n1}; }

// Loss and the full gradient (n->grad); the loss lands in n->loss_d.
cudaError_t backward_pass(stml_net* n, int B, int H, int W, cudaStream_t s) {
    const int H8 = pad8(H), W8 = pad8(W);
    const float inv_count = 1.f / (float)(2.0 * B * H * W);
    int hb = 0;
    ECK(launch_head(n->act[D0B], n->theta + n->head_off, n->base, n->tgt, n->smp_d, B, H, W, H8, W8, 1, inv_count,
                    n->hpart, &hb, n->gz1, s));
    ECK(launch_reduce_head(n->hpart, hb, n->grad, n->head_off, inv_count, n->loss_d, s));
    count_launches(2);
    bf16 *g = n->gz1, *g2 = n->gz2;
    auto swap = [&]() { std::swap(g, g2); };
    // decoder level 0
    ECK(layer_wgrad(n, D0B, g, B, H8, W8, s));
    ECK(layer_dgrad(n, D0B, g, B, H8, W8, mask_out(g2, n->act[D0A]), s));
    swap();
    ECK(layer_wgrad(n, D0A, g, B, H8, W8, s));
    ECK(layer_dgrad(n, D0A, g, B, H8, W8, split_out(n->fup, 64, n->skip[0]), s));
    ECK(launch_upback(n->fup, n->act[D1B], g2, B, H8, W8, 64, s));
    swap();
    // decoder level 1
    ECK(layer_wgrad(n, D1B, g, B, H8, W8, s));
    ECK(layer_dgrad(n, D1B, g, B, H8, W8, mask_out(g2, n->act[D1A]), s));
    swap();
    ECK(layer_wgrad(n, D1A, g, B, H8, W8, s));
    ECK(layer_dgrad(n, D1A, g, B, H8, W8, split_out(n->fup, 96, n->skip[1]), s));
    ECK(launch_upback(n->fup, n->act[D2B], g2, B, H8 >> 1, W8 >> 1, 96, s));
    swap();
    // decoder level 2
    ECK(layer_wgrad(n, D2B, g, B, H8, W8, s));
    ECK(layer_dgrad(n, D2B, g, B, H8, W8, mask_out(g2, n->act[D2A]), s));
    swap();
    ECK(layer_wgrad(n, D2A, g, B, H8, W8, s));
    ECK(layer_dgrad(n, D2A, g, B, H8, W8, split_out(n->fup, 128, n->skip[2]), s));
    ECK(launch_upback(n->fup, n->act[BB], g2, B, H8 >> 2, W8 >> 2, 128, s));
    swap();
    // bottleneck
    ECK(layer_wgrad(n, BB, g, B, H8, W8, s));
    ECK(layer_dgrad(n, BB, g, B, H8, W8, mask_out(g2, n->act[BA]), s));
    swap();
    ECK(layer_wgrad(n, BA, g, B, H8, W8, s));
    ECK(layer_dgrad(n, BA, g, B, H8, W8, split_out(n->dp, 96, nullptr), s));
    ECK(launch_combine(n->dp, n->skip[2], n->act[E2B], g2, B, H8 >> 2, W8 >> 2, 96, s));
    swap();
    // encoder level 2
    ECK(layer_wgrad(n, E2B, g, B, H8, W8, s));
    ECK(layer_dgrad(n, E2B, g, B, H8, W8, mask_out(g2, n->act[E2A]), s));
    swap();
    ECK(layer_wgrad(n, E2A, g, B, H8, W8, s));
    ECK(layer_dgrad(n, E2A, g, B, H8, W8, split_out(n->dp, 64, nullptr), s));
    ECK(launch_combine(n->dp, n->skip[1], n->act[E1B], g2, B, H8 >> 1, W8 >> 1, 64, s));
    swap();
    // encoder level 1
    ECK(layer_wgrad(n, E1B, g, B, H8, W8, s));
    ECK(layer_dgrad(n, E1B, g, B, H8, W8, mask_out(g2, n->act[E1A]), s));
    swap();
    ECK(layer_wgrad(n, E1A, g, B, H8, W8, s));
    ECK(layer_dgrad(n, E1A, g, B, H8, W8, split_out(n->dp, 32, nullptr), s));
    ECK(launch_combine(n->dp, n->skip[0], n->act[E0B], g2, B, H8, W8, 32, s));
    swap();
    // encoder level 0
    ECK(layer_wgrad(n, E0B, g, B, H8, W8, s));
    ECK(layer_dgrad(n, E0B, g, B, H8, W8, mask_out(g2, n->act[E0A]), s));
    swap();
    ECK(layer_wgrad(n, E0A, g, B, H8, W8, s));
    count_launches(6);
    return cudaSuccess;
}

// STML_ETIMEOUT (and the flag cleared) if a convolution's bounded wait
// expired since the last check; the stream must be synchronised.
stml_status check_err(stml_net* n) {
    NCK(n, cudaMemcpy(n->err_h, n->err_d, sizeof(int), cudaMemcpyDeviceToHost));
    if (*n->err_h) {
        const bool drained = *n->err_h == 1;
        NCK(n, cudaMemset(n->err_d, 0, sizeof(int)));
        return net_fail(n, STML_ETIMEOUT, drained ? "a convolution's bounded wait expired"
                                                  : "a convolution's bounded wait expired with tensor-core work "
                                                    "still in flight: results undefined, discard the context");
    }
    return STML_OK;
}

stml_status check_batch(stml_net* n, const stml_net_sample* smp, int B, int H, int W, bool need_target,
                        bool need_out) {
    if (!n) return net_fail(nullptr, STML_EINVAL, "net is NULL");
    if (!smp || B < 1 || B > n->maxB || H < 1 || W < 1 || pad8(H) > n->maxH8 || pad8(W) > n->maxW8)
        return net_fail(n, STML_EINVAL, "batch larger than the network's buffers or empty");
    for (int b = 0; b < B; ++b) {
        const stml_net_sample& s = smp[b];
        if (!s.y_l || !s.y_r || !s.T_l || !s.T_k || !s.T_r || (need_target && !s.target) || (need_out && !s.out))
            return net_fail(n, STML_EINVAL, "a sample lacks a pointer");
        if (s.ld < W || s.ld_img < W || s.plane < (long long)s.ld * (H - 1) + W)
            return net_fail(n, STML_EINVAL, "sample strides smaller than the crop");
        if (!(s.h > 0.f) || !(s.w_l >= 0.f && s.w_l <= 1.f))
            return net_fail(n, STML_EINVAL, "sample h must be > 0 and w_l in [0, 1]");
    }
    return STML_OK;
}

void to_internal(const stml_net_sample* smp, int B, std::vector<Sample>& out) {
    out.resize(B);
    for (int b = 0; b < B; ++b) {
        const stml_net_sample& s = smp[b];
        out[b] = Sample{s.y_l, s.y_r, s.T_l, s.T_k, s.T_r, s.target, s.out, s.plane, s.ld, s.ld_img, 0, s.w_l, s.h};
    }
}

}  // namespace

// ---------------------------------------------------- used by the registration
bool stml::net::fits(const ::stml_net* n, int H, int W) { return n && pad8(H) <= n->maxH8 && pad8(W) <= n->maxW8; }
int stml::net::max_batch(const ::stml_net* n) { return n ? n->maxB : 0; }
bool stml::net::timed_out(::stml_net* n) {
    if (cudaMemcpy(n->err_h, n->err_d, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return true;
    if (!*n->err_h) return false;
    cudaMemset(n->err_d, 0, sizeof(int));
    return true;
}

cudaError_t stml::net::forward_on(::stml_net* n, const Sample* smp, int B, int H, int W, cudaStream_t s) {
    if (B < 1 || B > n->maxB || !fits(n, H, W)) return cudaErrorInvalidValue;
    ECK(upload_samples(n, smp, B, s));
    ECK(forward_pass(n, B, H, W, false, s));
    int hb = 0;
    ECK(launch_head(n->act[D0B], n->theta + n->head_off, n->base, nullptr, n->smp_d, B, H, W, pad8(H), pad8(W), 0,
                    0.f, nullptr, &hb, nullptr, s));
    count_launches(1);
    return cudaSuccess;
}

// ============================================================== C interface
extern "C" {

size_t stml_net_param_count(void) { return (size_t)kParams; }

stml_status stml_net_create(const float* params, size_t n_params, int max_batch, int max_h, int max_w,
                            void* cuda_stream, stml_net** out) {
    if (!out) return net_fail(nullptr, STML_EINVAL, "out is NULL");
    *out = nullptr;
    if (!params || n_params != (size_t)kParams)
        return net_fail(nullptr, STML_EINVAL, "params must hold stml_net_param_count() floats");
    if (max_batch < 1 || max_h < 1 || max_w < 1 || (long long)max_batch * pad8(max_h) * pad8(max_w) > (1LL << 30))
        return net_fail(nullptr, STML_EINVAL, "bad network capacity");
    stml_net* n = new stml_net();
    n->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaGetDevice(&n->device);
    n->maxB = max_batch;
    n->maxH8 = pad8(max_h);
    n->maxW8 = pad8(max_w);
    n->P0 = (long long)max_batch * n->maxH8 * n->maxW8;
    cudaError_t e = alloc_all(n);
    if (e == cudaSuccess) e = upload_params(n, params);
    if (e != cudaSuccess) {
        const std::string msg = std::string("stml_net_create: ") + cudaGetErrorString(e);
        free_all(n);
        delete n;
        return net_fail(nullptr, e == cudaErrorMemoryAllocation ? STML_ENOMEM : STML_ECUDA, msg);
    }
    *out = n;
    return STML_OK;
}

void stml_net_destroy(stml_net* n) {
    if (!n) return;
    cudaSetDevice(n->device);
    cudaStreamSynchronize(n->stream);
    free_all(n);
    delete n;
}

const char* stml_net_last_error(const stml_net* n) { return n ? n->err.c_str() : ""; }

stml_status stml_net_set_params(stml_net* n, const float* params, size_t n_params) {
    if (!n) return net_fail(nullptr, STML_EINVAL, "net is NULL");
    if (!params || n_params != (size_t)kParams) return net_fail(n, STML_EINVAL, "wrong parameter count");
    cudaSetDevice(n->device);
    NCK(n, upload_params(n, params));
    return STML_OK;
}

stml_status stml_net_get_params(stml_net* n, float* params, size_t n_params) {
    if (!n) return net_fail(nullptr, STML_EINVAL, "net is NULL");
    if (!params || n_params != (size_t)kParams) return net_fail(n, STML_EINVAL, "wrong parameter count");
    cudaSetDevice(n->device);
    NCK(n, cudaMemcpyAsync(params, n->theta, kParams * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
    NCK(n, cudaStreamSynchronize(n->stream));
    return check_err(n);
}

stml_status stml_net_forward(stml_net* n, const stml_net_sample* smp, int B, int H, int W) {
    stml_status st = check_batch(n, smp, B, H, W, false, true);
    if (st != STML_OK) return st;
    cudaSetDevice(n->device);
    std::vector<Sample> s;
    to_internal(smp, B, s);
    NCK(n, forward_on(n, s.data(), B, H, W, n->stream));
    return STML_OK;
}

stml_status stml_net_loss_grad(stml_net* n, const stml_net_sample* smp, int B, int H, int W, double* loss,
                               float* grad) {
    stml_status st = check_batch(n, smp, B, H, W, true, false);
    if (st != STML_OK) return st;
    cudaSetDevice(n->device);
    std::vector<Sample> s;
    to_internal(smp, B, s);
    NCK(n, upload_samples(n, s.data(), B, n->stream));
    NCK(n, forward_pass(n, B, H, W, true, n->stream));
    NCK(n, backward_pass(n, B, H, W, n->stream));
    NCK(n, cudaMemcpyAsync(n->loss_h, n->loss_d, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
    if (grad) NCK(n, cudaMemcpyAsync(grad, n->grad, kParams * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
    NCK(n, cudaStreamSynchronize(n->stream));
    if (loss) *loss = *n->loss_h;
    return check_err(n);
}

stml_status stml_net_train_step(stml_net* n, const stml_net_sample* smp, int B, int H, int W, const stml_adam* opt,
                                double* loss) {
    stml_status st = check_batch(n, smp, B, H, W, true, false);
    if (st != STML_OK) return st;
    const stml_adam def{1e-3, 0.9, 0.999, 1e-8};
    const stml_adam& a = opt ? *opt : def;
    if (!(a.lr > 0) || !(a.beta1 >= 0 && a.beta1 < 1) || !(a.beta2 >= 0 && a.beta2 < 1) || !(a.eps > 0))
        return net_fail(n, STML_EINVAL, "bad Adam parameters");
    cudaSetDevice(n->device);
    std::vector<Sample> s;
    to_internal(smp, B, s);
    NCK(n, upload_samples(n, s.data(), B, n->stream));
    NCK(n, forward_pass(n, B, H, W, true, n->stream));
    NCK(n, backward_pass(n, B, H, W, n->stream));
    ++n->step;
    const double c1 = 1.0 / (1.0 - std::pow(a.beta1, (double)n->step));
    const double c2 = 1.0 / (1.0 - std::pow(a.beta2, (double)n->step));
    NCK(n, launch_adam(n->theta, n->m, n->v, n->grad, kParams, (float)a.lr, (float)a.beta1, (float)a.beta2,
                       (float)a.eps, (float)c1, (float)c2, n->stream));
    NCK(n, launch_pack(n->theta, n->pt, n->stream));
    count_launches(2);
    if (loss) {
        NCK(n, cudaMemcpyAsync(n->loss_h, n->loss_d, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
        NCK(n, cudaStreamSynchronize(n->stream));
        *loss = *n->loss_h;
        return check_err(n);
    }
    return STML_OK;
}

stml_status stml_net_conv3_block(int mode, const float* x, const float* a, const float* W, const float* b,
                                 float* y, int B, int H, int W_, int Cin, int Cout, void* cuda_stream) {
    if (mode < 0 || mode > 2 || !x || !W || !y || (mode != 1 && !b) || (mode == 2 && !a) || B < 1 || H < 1 ||
        W_ < 1 || Cin < 32 || Cout < 32 || Cin % 32 || Cout % 32 || Cin > 256 || Cout > 256)
        return net_fail(nullptr, STML_EINVAL, "stml_net_conv3_block: bad arguments");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const long long P = (long long)B * H * W_;
    const long long nw = 9LL * Cin * Cout;
    bf16 *xb = nullptr, *ab = nullptr, *yb = nullptr, *wf = nullptr, *wd = nullptr;
    float *wpart = nullptr, *bpart = nullptr;
    int* errd = nullptr;
    int errh = 0;
    const size_t wcap = (size_t)nw * 64, bcap = 256 * 256;
    cudaError_t e = cudaSuccess;
    auto run = [&]() -> cudaError_t {
        ECK(nalloc(&xb, (size_t)(P * (mode == 0 ? Cin : Cout))));
        ECK(nalloc(&wf, (size_t)nw));
        ECK(nalloc(&wd, (size_t)nw));
        ECK(nalloc(&errd, 1));
        ECK(cudaMemsetAsync(errd, 0, sizeof(int), s));
        PackTable t{};
        t.n = 1;
        t.cin_real[0] = Cin;
        t.cin[0] = Cin;
        t.cout[0] = Cout;
        t.w_off[0] = 0;
        t.wf[0] = wf;
        t.wd[0] = wd;
        ECK(launch_pack(W, t, s));
        ECK(launch_to_bf16(x, xb, P * (mode == 0 ? Cin : Cout), s));
        if (mode == 0) {
            ECK(nalloc(&yb, (size_t)(P * Cout)));
            ConvOut o{CONV_FWD, b, yb, nullptr, nullptr, nullptr, 0};
            ECK(launch_conv3(cin1(xb, Cin), wf, Cin, Cout, B, H, W_, o, errd, s));
            ECK(launch_from_bf16(yb, y, P * Cout, s));
        } else if (mode == 1) {
            ECK(launch_conv3(cin1(xb, Cout), wd, Cout, Cin, B, H, W_, split_out(y, Cin, nullptr), errd, s));
        } else {
            ECK(nalloc(&ab, (size_t)(P * Cin)));
            ECK(launch_to_bf16(a, ab, P * Cin, s));
            ECK(nalloc(&wpart, wcap));
            ECK(nalloc(&bpart, bcap));
            int ws = 0, bs = 0;
            ECK(launch_wgrad3(cin1(ab, Cin), xb, Cin, Cout, B, H, W_, wpart, wcap, &ws, errd, s));
            ECK(launch_colsum(xb, P, Cout, bpart, bcap, &bs, s));
            ECK(launch_reduce_grad(wpart, ws, Cin, Cin, Cout, bpart, bs, y, 0, nw, s));
        }
        ECK(cudaStreamSynchronize(s));
        if (errd) ECK(cudaMemcpy(&errh, errd, sizeof(int), cudaMemcpyDeviceToHost));
        return cudaSuccess;
    };
    e = run();
    for (void* p : {(void*)xb, (void*)ab, (void*)yb, (void*)wf, (void*)wd, (void*)wpart, (void*)bpart, (void*)errd})
        if (p) cudaFree(p);
    if (e != cudaSuccess) return net_fail(nullptr, STML_ECUDA, std::string("stml_net_conv3_block: ") + cudaGetErrorString(e));
    if (errh) return net_fail(nullptr, STML_ETIMEOUT, "stml_net_conv3_block: a bounded wait expired");
    return STML_OK;
}

stml_status stml_check_bounded_wait(void* cuda_stream, int* expired) {
    if (!expired) return net_fail(nullptr, STML_EINVAL, "expired is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int* d = nullptr;
    cudaError_t e = nalloc(&d, 1);
    if (e == cudaSuccess) e = cudaMemsetAsync(d, 0, sizeof(int), s);
    if (e == cudaSuccess) e = launch_wait_probe(d, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
    if (d) cudaFree(d);
    if (e != cudaSuccess) return net_fail(nullptr, STML_ECUDA, std::string("stml_check_bounded_wait: ") + cudaGetErrorString(e));
    *expired = h;
    return STML_OK;
}

}  // extern "C"
