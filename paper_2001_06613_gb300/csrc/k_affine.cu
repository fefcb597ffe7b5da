// Affine-linear transformations per frame (Sec. 4) for the L-BFGS solver of
// Sec. 2: the displacement of frame k is u_k(x) = W_k (x - c) / rho + b_k,
// x the cell centre in finest-level pixel units, c the domain centre and rho
// half of its largest extent; theta_k = (W_k row by row, b_k), d (d + 1)
// values.  The objective and its field gradient come from the registration's
// own objective and gradient passes on the field these kernels write; the
// projection below turns the field gradient into dJ/dtheta.
#include "kernels.h"

namespace stml {

namespace {

// (x - c) / rho of the cell with indices (iz, iy, ix): component i of xhat
// belongs to array axis i (z, y, x in 3-D; y, x in 2-D).
template <int D>
__device__ __forceinline__ void cell_xhat(const Geom& g, const AffineFrame& af, long long p, float (&xh)[D]) {
    const int ix = (int)(p % g.nx);
    const long long q = p / g.nx;
    const int iy = (int)(q % g.ny);
    const int iz = (int)(q / g.ny);
    const float xs[3] = {((float)iz + 0.5f) * g.h, ((float)iy + 0.5f) * g.h, ((float)ix + 0.5f) * g.h};
#pragma unroll
    for (int i = 0; i < D; ++i) xh[i] = (xs[3 - D + i] - af.c[i]) * af.inv_rho;
}

template <int D>
__global__ void affine_field_kernel(Geom g, AffineFrame af, const float* __restrict__ theta, int nK,
                                    float* __restrict__ u) {
    constexpr int P = D * (D + 1);
    const int k = blockIdx.y;
    if (k >= nK) return;
    float th[P];
#pragma unroll
    for (int j = 0; j < P; ++j) th[j] = theta[k * P + j];
    float* uk = u + (size_t)k * D * g.N;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < g.N;
         p += (long long)gridDim.x * blockDim.x) {
        float xh[D];
        cell_xhat<D>(g, af, p, xh);
#pragma unroll
        for (int c = 0; c < D; ++c) {
            float v = th[D * D + c];
#pragma unroll
            for (int i = 0; i < D; ++i) v = fmaf(th[c * D + i], xh[i], v);
            uk[(size_t)c * g.N + p] = v;
        }
    }
}

// Per-CTA sums of g_{k,c}(x) xhat_i(x) and g_{k,c}(x) (FP32 per thread over
// its few cells, FP64 across the CTA), written to part[k][block][P].
template <int D>
__global__ void __launch_bounds__(256) affine_project_kernel(Geom g, AffineFrame af, const float* __restrict__ gu,
                                                             int nK, double* __restrict__ part) {
    constexpr int P = D * (D + 1);
    __shared__ double red[8][P];
    const int k = blockIdx.y;
    float acc[P];
#pragma unroll
    for (int j = 0; j < P; ++j) acc[j] = 0.f;
    const float* gk = gu + (size_t)k * D * g.N;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < g.N;
         p += (long long)gridDim.x * blockDim.x) {
        float xh[D];
        cell_xhat<D>(g, af, p, xh);
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const float gc = gk[(size_t)c * g.N + p];
#pragma unroll
            for (int i = 0; i < D; ++i) acc[c * D + i] = fmaf(gc, xh[i], acc[c * D + i]);
            acc[D * D + c] += gc;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < P; ++j) {
        double v = (double)acc[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][j] = v;
    }
    __syncthreads();
    if (threadIdx.x < P) {
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v += red[w][threadIdx.x];
        part[((size_t)k * gridDim.x + blockIdx.x) * P + threadIdx.x] = v;
    }
}

__global__ void affine_project_sum_kernel(const double* __restrict__ part, int blocks, int P,
                                          double* __restrict__ out) {
    const int k = blockIdx.x;
    for (int j = threadIdx.x; j < P; j += blockDim.x) {
        double v = 0.0;
        for (int b = 0; b < blocks; ++b) v += part[((size_t)k * blocks + b) * P + j];
        out[(size_t)k * P + j] = v;
    }
}

}  // namespace

int affine_project_blocks(const Geom& g) {
    long long b = (g.N + 256 * 8 - 1) / (256 * 8);
    if (b < 1) b = 1;
    if (b > 256) b = 256;
    return (int)b;
}

cudaError_t launch_affine_field(const Geom& g, const AffineFrame& af, const float* theta, int nK, float* u,
                                cudaStream_t s) {
    if (nK <= 0) return cudaErrorInvalidValue;
    long long bx = (g.N + 255) / 256;
    if (bx > 1024) bx = 1024;
    dim3 grid((unsigned)bx, (unsigned)nK);
    if (g.d == 2)
        affine_field_kernel<2><<<grid, 256, 0, s>>>(g, af, theta, nK, u);
    else
        affine_field_kernel<3><<<grid, 256, 0, s>>>(g, af, theta, nK, u);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_affine_project(const Geom& g, const AffineFrame& af, const float* gu, int nK, double* part,
                                  double* out, cudaStream_t s) {
    if (nK <= 0) return cudaErrorInvalidValue;
    const int blocks = affine_project_blocks(g);
    const int P = g.d * (g.d + 1);
    dim3 grid((unsigned)blocks, (unsigned)nK);
    if (g.d == 2)
        affine_project_kernel<2><<<grid, 256, 0, s>>>(g, af, gu, nK, part);
    else
        affine_project_kernel<3><<<grid, 256, 0, s>>>(g, af, gu, nK, part);
    affine_project_sum_kernel<<<nK, 32, 0, s>>>(part, blocks, P, out);
    count_launches(2);
    return cudaGetLastError();
}

}  // namespace stml
