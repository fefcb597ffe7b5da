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
// cudaGetSymbolAddress on the first call made with that device current, and
// passed to the kernels.  The address is kept per CUDA context, so a context
// that replaces the device's (after cudaDeviceReset, say) looks it up again on
// its first call.  That first call should come before any stream capture.
// The frame numbers and temporal weights reach the array through the
// arguments of small set-up kernels, not through copies from host memory.
// All calls share the array and it keeps the last call's contents: the
// reduction ticket is cleared on every call, and calls that overlap on the
// GPU (other streams, other threads) race on it.
#include <cuda.h>   // driver API types; the two functions used come from cudaGetDriverEntryPointByVersion

#include <map>
#include <mutex>
#include <utility>

#include "../../include/stml.h"
#include "kernels.h"

namespace {

constexpr size_t kScratchBytes = 24u << 20;   // 24 MiB per device
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
std::map<std::pair<int, unsigned long long>, void*> g_scratch_dev;   // (device, context id) -> address

// Identity of the calling thread's current CUDA context (0 when none is
// current or the driver entry points are unavailable).
unsigned long long current_context_id() {
    using GetCurrent = CUresult (*)(CUcontext*);
    using GetId = CUresult (*)(CUcontext, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {   // under g_mu
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
        looked_up = true;
    }
    CUcontext c = nullptr;
    if (!get_current || get_current(&c) != CUDA_SUCCESS || !c) return 0;
    unsigned long long id = 0;
    if (get_id && get_id(c, &id) == CUDA_SUCCESS) return id + 1;
    return (unsigned long long)(uintptr_t)c;
}

// Frame numbers and temporal weights of up to kSetupChunk frames, passed by
// value as kernel arguments.
constexpr int kSetupChunk = 256;
struct SetupChunk {
    int first, count;
    int frames[kSetupChunk];
    float w_next[kSetupChunk];
};

__global__ void noalloc_setup_kernel(SetupChunk c, int* frames, float* w_next) {
    for (int i = threadIdx.x; i < c.count; i += blockDim.x) {
        frames[c.first + i] = c.frames[i];
        w_next[c.first + i] = c.w_next[i];
    }
}

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
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        unsigned long long ctx = current_context_id();
        auto it = ctx ? g_scratch_dev.find({dev, ctx}) : g_scratch_dev.end();
        if (it != g_scratch_dev.end()) {
            base = (unsigned char*)it->second;
        } else {
            void* ptr = nullptr;   // also makes the runtime's context current if it was not yet
            e = cudaGetSymbolAddress(&ptr, g_scratch);
            if (e != cudaSuccess || !ptr) return err(STML_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            if (!ctx) ctx = current_context_id();
            if (ctx) g_scratch_dev[{dev, ctx}] = ptr;
            base = (unsigned char*)ptr;
        }
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    unsigned int* ticket = (unsigned int*)base;
    double* out = (double*)(base + 8);
    e = cudaMemsetAsync(base, 0, 256, s);                       // ticket and result start at zero
    // frames and w_next = 1 / (k_{j+1} - k_j)^2 (0 for the last frame of K)
    SetupChunk chunk;
    for (int j0 = 0; e == cudaSuccess && j0 < nK; j0 += kSetupChunk) {
        chunk.first = j0;
        chunk.count = nK - j0 < kSetupChunk ? nK - j0 : kSetupChunk;
        for (int i = 0; i < chunk.count; ++i) {
            const int j = j0 + i;
            chunk.frames[i] = frames[j];
            const double dk = j + 1 < nK ? (double)(frames[j + 1] - frames[j]) : 0.0;
            chunk.w_next[i] = j + 1 < nK ? (float)(1.0 / (dk * dk)) : 0.f;
        }
        noalloc_setup_kernel<<<1, 256, 0, s>>>(chunk, (int*)(base + off_frames), (float*)(base + off_w));
        count_launches(1);
        e = cudaGetLastError();
    }
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
