// The directional derivative <g, d> of a Gauss-Newton step with |d|^2, as
// one deterministic FP64 reduction over flat arrays (float4 when the length
// allows).
#include "kernels.h"

namespace stml {

namespace {

constexpr int kVecBlocks = 152 * 8;   // grid-stride launch: 8 CTAs per SM of a GB300

inline unsigned flat_blocks(size_t n4) {
    size_t b = (n4 + kThreads - 1) / kThreads;
    if (b < 1) b = 1;
    if (b > (size_t)kVecBlocks) b = kVecBlocks;
    return (unsigned)b;
}

__device__ __forceinline__ float4 ld4(const float* p, size_t i) { return __ldg(reinterpret_cast<const float4*>(p) + i); }

}  // namespace

__global__ void __launch_bounds__(kThreads)
dot2_kernel(const float* __restrict__ a, const float* __restrict__ b, size_t n,
            double* __restrict__ partials, unsigned int* ticket, double* out) {
    float acc[2] = {0.f, 0.f};
    const size_t n4 = n / 4;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += stride) {
        const float4 av = ld4(a, i), bv = ld4(b, i);
        acc[0] += av.x * bv.x + av.y * bv.y + av.z * bv.z + av.w * bv.w;
        acc[1] += bv.x * bv.x + bv.y * bv.y + bv.z * bv.z + bv.w * bv.w;
    }
    for (size_t i = n4 * 4 + blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        const float bv = __ldg(b + i);
        acc[0] = fmaf(__ldg(a + i), bv, acc[0]);
        acc[1] = fmaf(bv, bv, acc[1]);
    }
    grid_reduce<2>(acc, partials, ticket, out);
}

cudaError_t launch_dot2(const float* a, const float* b, size_t n, double* partials,
                        unsigned int* ticket, double* out, cudaStream_t s) {
    dot2_kernel<<<flat_blocks(n / 4 + 1), kThreads, 0, s>>>(a, b, n, partials, ticket, out);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace stml
