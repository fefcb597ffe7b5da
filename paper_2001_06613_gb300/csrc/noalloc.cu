// Gauss-Newton Hessian product for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running under a host framework
// that owns all device memory through its own pool, code that may only touch
// buffers handed to it, or code whose set-up must not change the device's
// allocation state.  stml_hessvec_noalloc serves them: the caller passes the
// inputs and the output, and every scratch buffer the kernels need (per-pixel
// frame sums, per-CTA partial sums, the reduction ticket, the frame weights)
// lives in the fixed array below.
//
// The array is a file-scope __device__ variable of kScratchBytes; every GPU
// that loads this library holds it until the process exits.  Its name is a
// host-side stand-in in host code, so the device address is fetched with
// cudaGetSymbolAddress once per device (on the first call made with that
// device current) and passed to the kernels.  That first call should come
// before any stream capture.  All calls share the array and it keeps the last
// call's contents: the reduction ticket is cleared on every call, and calls
// that overlap on the GPU (other streams, other threads) race on it.
#include <mutex>
#include <vector>

#include "../../include/stml.h"
#include "kernels.h"

namespace {

constexpr size_t kScratchBytes = 24u << 20;   // 24 MiB per device
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_dev[kMaxDevices] = {};

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Errors are reported through stml_last_error(NULL), like the other
// context-free calls.
stml_status err(stml_status s, const std::string& m) {
    stml::set_context_free_error(m);
    return s;
}

}  // namespace

extern "C" stml_status stml_hessvec_noalloc(const float* dT, const float* v, float* Hv, int dim,
                                            const int* shape, double h, const int* frames, int nK,
                                            const stml_params* p, double* vHv, void* cuda_stream) {
    using namespace stml;
    if (!dT || !v || !Hv || !shape || !frames || !p || nK < 1 || (dim != 2 && dim != 3) || !(h > 0))
        return err(STML_EINVAL, "stml_hessvec_noalloc: bad arguments");
    int sh3[3] = {1, 1, 1};
    for (int i = 0; i < dim; ++i) {
        if (shape[i] < 1) return err(STML_EINVAL, "stml_hessvec_noalloc: bad shape");
        sh3[3 - dim + i] = shape[i];
    }
    if (((uintptr_t)dT | (uintptr_t)v | (uintptr_t)Hv) & 15u)
        return err(STML_EINVAL, "stml_hessvec_noalloc: device arrays must be 16-byte aligned");
    for (int j = 1; j < nK; ++j)
        if (frames[j] <= frames[j - 1]) return err(STML_EINVAL, "stml_hessvec_noalloc: frames must increase");
    const Geom g = make_geom(sh3, dim, (float)h);

    // scratch layout: ticket (0), result (8) | frames | w_next | partials | mean_s | sum_v
    const size_t off_frames = 256;
    const size_t off_w = off_frames + align256((size_t)nK * sizeof(int));
    const size_t off_part = off_w + align256((size_t)nK * sizeof(float));
    const size_t off_ms = off_part + align256(gn_partials(g, nK) * sizeof(double));
    const size_t off_sv = off_ms + align256((size_t)g.N * sizeof(float));
    const size_t need = off_sv + align256((size_t)dim * g.N * sizeof(float));
    if (need > kScratchBytes)
        return err(STML_EINVAL, "stml_hessvec_noalloc: problem needs " + std::to_string(need) +
                                    " scratch bytes, the static array holds " + std::to_string(kScratchBytes));

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return err(STML_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return err(STML_EINVAL, "device ordinal out of range");
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_dev[dev]) {
            void* ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_scratch);
            if (e != cudaSuccess || !ptr) return err(STML_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_scratch_dev[dev] = ptr;
        }
        base = (unsigned char*)g_scratch_dev[dev];
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    std::vector<float> w(nK, 0.f);
    for (int j = 0; j + 1 < nK; ++j) {
        const double dk = (double)(frames[j + 1] - frames[j]);
        w[j] = (float)(1.0 / (dk * dk));
    }
    unsigned int* ticket = (unsigned int*)base;
    double* out = (double*)(base + 8);
    e = cudaMemsetAsync(base, 0, 256, s);                       // ticket and result start at zero
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + off_frames, frames, (size_t)nK * sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + off_w, w.data(), (size_t)nK * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return err(STML_ECUDA, cudaGetErrorString(e));

    FrameSet fs{(const int*)(base + off_frames), (const float*)(base + off_w), nK};
    Coef cf;
    const double hd = g.hd;
    cf.alpha_hd = (float)(p->alpha * hd);
    cf.alphat_hd = (float)(p->alpha_t * hd);
    cf.pen_g = (float)(2.0 * p->lambda * hd / nK);
    cf.pen_h = (float)(2.0 * p->lambda * hd / ((double)nK * nK));
    cf.lam_hd = (float)(p->lambda * hd);
    cf.half_hd = (float)(0.5 * hd);
    cf.hd = (float)hd;
    cf.inv_h2 = (float)(1.0 / (h * h));
    cf.inv_nK = (float)(1.0 / nK);
    cf.diag_D = (float)(hd * (1.0 - 1.0 / nK));
    HessWork hw{(float*)(base + off_ms), (float*)(base + off_sv), (double*)(base + off_part), gn_partials(g, nK)};
    e = launch_hessvec(g, fs, cf, dT, v, Hv, hw, ticket, out, nullptr, s);
    if (e != cudaSuccess) return err(STML_ECUDA, cudaGetErrorString(e));
    if (vHv) {
        e = cudaMemcpyAsync(vHv, out, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return err(STML_ECUDA, cudaGetErrorString(e));
    }
    return STML_OK;
}
