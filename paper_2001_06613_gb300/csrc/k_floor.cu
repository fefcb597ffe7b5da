// Latency floor of a CG step of the cooperative PCG solve.
//
// pcg_coop_kernel spends each CG step in two rounds of: CTA partial sums ->
// grid-wide barrier -> the fixed-order total of all partials, formed in every
// CTA (once for <p, Hp>, once for <r, z> and |r|^2), around its two vector
// passes.  On the small levels, where the vectors are a few hundred KB to a
// few MB and stay in L2, those rounds and not the bytes bound a step.
// coop_floor_kernel runs only the rounds, with the same reductions and the
// same barrier, so that timing it on the solve's grid gives the part of a CG
// step that no faster vector pass can remove.
#include <cooperative_groups.h>

#include <string>

#include "../../include/stml.h"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace stml {
namespace {

__global__ void __launch_bounds__(kThreads) coop_floor_kernel(double* partials, int iters, float* sink) {
    cg::grid_group grid = cg::this_grid();
    // the solve's two partial-sum buffers, each rewritten only after a
    // barrier that follows every CTA's read of it
    float2* partA = reinterpret_cast<float2*>(partials);
    float2* partB = partA + 2 * (size_t)gridDim.x;
    float carry = 0.f;
    for (int k = 0; k < iters; ++k) {
        const float v1[1] = {carry + (float)threadIdx.x};
        cta_partials<1>(v1, partA, blockIdx.x);
        grid.sync();
        dfloat t1[1];
        cta_total<1>(partA, gridDim.x, t1);
        const float v2[2] = {t1[0].hi * 1e-30f, (float)blockIdx.x};
        cta_partials<2>(v2, partB, blockIdx.x);
        grid.sync();
        dfloat t2[2];
        cta_total<2>(partB, gridDim.x, t2);
        carry = 1e-30f * (t2[0].hi + t2[1].hi);   // each round depends on the one before
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *sink = carry;
}

// Dynamic shared memory (unused) that leaves room for at most two CTAs per
// SM, the residency of the solve (whose registers allow two): the CTAs of a
// grid are spread over the SMs as the solve's are.
constexpr int kFloorSmem = 96 * 1024;

stml_status floor_err(stml_status s, const std::string& m) {
    set_context_free_error("stml_coop_sync_floor: " + m);
    return s;
}

}  // namespace
}  // namespace stml

extern "C" stml_status stml_coop_sync_floor(int blocks, int iters, double* us_per_iter) {
    using namespace stml;
    if (blocks < 1 || iters < 1 || !us_per_iter) return floor_err(STML_EINVAL, "bad arguments");
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void*)coop_floor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kFloorSmem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)coop_floor_kernel, kThreads,
                                                          kFloorSmem);
    if (e != cudaSuccess) return floor_err(STML_ECUDA, cudaGetErrorString(e));
    if ((long long)blocks > (long long)sms * per_sm)
        return floor_err(STML_EINVAL, std::to_string(blocks) + " CTAs cannot all be resident (at most " +
                                          std::to_string((long long)sms * per_sm) + ")");
    double* partials = nullptr;
    float* sink = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    auto release = [&]() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
        if (s) cudaStreamDestroy(s);
        cudaFree(partials);
        cudaFree(sink);
    };
    // the two buffers: 1 + 2 float2 per CTA
    e = cudaMalloc(&partials, (size_t)blocks * 4 * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(float));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    float ms = 0.f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // a warm-up launch, then the timed one
        void* args[] = {(void*)&partials, (void*)&iters, (void*)&sink};
        if (rep == 1) e = cudaEventRecord(a, s);
        if (e == cudaSuccess) {
            e = cudaLaunchCooperativeKernel((const void*)coop_floor_kernel, dim3(blocks), dim3(kThreads), args,
                                            kFloorSmem, s);
            if (e == cudaSuccess) count_launches(1);
        }
        if (e == cudaSuccess && rep == 1) e = cudaEventRecord(b, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    release();
    if (e != cudaSuccess) {
        cudaGetLastError();   // a refused launch leaves no error behind for later calls
        return floor_err(STML_ECUDA, cudaGetErrorString(e));
    }
    *us_per_iter = 1e3 * (double)ms / iters;
    return STML_OK;
}
