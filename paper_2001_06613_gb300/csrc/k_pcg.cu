// Vector kernels of the Jacobi-preconditioned conjugate-gradient solve of
// H d = -g inside each Gauss-Newton step.  The CG coefficients live in device
// memory (DevScalars): the last CTA of each reducing kernel computes them, so
// the host only looks at the solver state between chunks of iterations.
//
// The Jacobi diagonal is recomputed from grad T on the fly:
//   diag = hd (1 - 1/|K|) (d_c T_k)^2 + alpha hd nnb / h^2
//          + alpha_t hd (w_prev + w_next) + 2 lambda hd / |K|^2,
// nnb = number of in-grid neighbours of the pixel.
#include "kernels.h"

namespace stml {

__device__ __forceinline__ float jacobi_inv(float dt, int nnb, float tdiag, const Coef& cf) {
    const float dg = cf.diag_D * dt * dt + cf.alpha_hd * cf.inv_h2 * (float)nnb +
                     cf.alphat_hd * tdiag + cf.pen_h;
    return dg > 0.f ? 1.0f / dg : 1.0f;   // zero only when alpha = lambda = 0 and grad T = 0
}

static unsigned vec_blocks_x(const Geom& g) {
    long long per = (g.N + (long long)kThreads * 4 - 1) / ((long long)kThreads * 4);
    if (per < 1) per = 1;
    if (per > 65535) per = 65535;
    return (unsigned)per;
}

template <int D>
__global__ void __launch_bounds__(kThreads)
pcg_init_kernel(Geom g, FrameSet fs, Coef cf, const float* __restrict__ grad,
                const float* __restrict__ dT, float* __restrict__ x, float* __restrict__ r,
                float* __restrict__ p, double* __restrict__ partials, DevScalars* S, PcgArgs a) {
    const int plane = blockIdx.y, j = plane / D;
    const float tdiag = __ldg(fs.w_next + j) + (j > 0 ? __ldg(fs.w_next + j - 1) : 0.f);
    float acc[2] = {0.f, 0.f};
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < g.N;
         q += (long long)gridDim.x * blockDim.x) {
        int ix, iy, iz;
        unflatten(g, q, ix, iy, iz);
        const size_t e = (size_t)plane * g.N + q;
        const float rv = -__ldg(grad + e);
        const float zv = jacobi_inv(__ldg(dT + e), neighbour_count(g, ix, iy, iz), tdiag, cf) * rv;
        r[e] = rv;
        p[e] = zv;
        x[e] = 0.f;
        acc[0] = fmaf(rv, zv, acc[0]);
        acc[1] = fmaf(rv, rv, acc[1]);
    }
    double tot[2];
    if (grid_reduce<2>(acc, partials, &S->ticket[2], tot) && threadIdx.x == 0) {
        S->rho = tot[0];
        S->bnorm2 = tot[1];
        S->rnorm2 = tot[1];
        S->cg_iter = 0;
        if (!(tot[1] > 0.0)) {
            S->cg_flag = CG_ZERO;
            S->cg_active = 0;
        } else if (a.max_cg <= 0) {
            S->cg_flag = CG_MAXIT;
            S->cg_active = 0;
        } else {
            S->cg_flag = CG_RUNNING;
            S->cg_active = 1;
        }
    }
}

template <int D>
__global__ void __launch_bounds__(kThreads)
pcg_update_kernel(Geom g, FrameSet fs, Coef cf, const float* __restrict__ dT,
                  float* __restrict__ x, float* __restrict__ r, const float* __restrict__ p,
                  const float* __restrict__ q, double* __restrict__ partials, DevScalars* S,
                  PcgArgs a) {
    if (!S->cg_active) return;
    const float alpha = (float)S->alpha;
    const int plane = blockIdx.y, j = plane / D;
    const float tdiag = __ldg(fs.w_next + j) + (j > 0 ? __ldg(fs.w_next + j - 1) : 0.f);
    float acc[2] = {0.f, 0.f};
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < g.N;
         k += (long long)gridDim.x * blockDim.x) {
        int ix, iy, iz;
        unflatten(g, k, ix, iy, iz);
        const size_t e = (size_t)plane * g.N + k;
        x[e] = fmaf(alpha, __ldg(p + e), x[e]);
        const float rv = fmaf(-alpha, __ldg(q + e), r[e]);
        r[e] = rv;
        const float zv = jacobi_inv(__ldg(dT + e), neighbour_count(g, ix, iy, iz), tdiag, cf) * rv;
        acc[0] = fmaf(rv, zv, acc[0]);
        acc[1] = fmaf(rv, rv, acc[1]);
    }
    double tot[2];
    if (grid_reduce<2>(acc, partials, &S->ticket[2], tot) && threadIdx.x == 0) {
        S->cg_iter += 1;
        S->rnorm2 = tot[1];
        if (sqrt(tot[1]) <= (double)a.tol_cg * sqrt(S->bnorm2)) {
            S->cg_flag = CG_CONVERGED;
            S->cg_active = 0;
        } else if (S->cg_iter >= a.max_cg) {
            S->cg_flag = CG_MAXIT;
            S->cg_active = 0;
        } else {
            S->beta = tot[0] / S->rho;
            S->rho = tot[0];
        }
    }
}

template <int D>
__global__ void __launch_bounds__(kThreads)
pcg_pupdate_kernel(Geom g, FrameSet fs, Coef cf, const float* __restrict__ dT,
                   const float* __restrict__ r, float* __restrict__ p, DevScalars* S) {
    if (!S->cg_active) return;
    const float beta = (float)S->beta;
    const int plane = blockIdx.y, j = plane / D;
    const float tdiag = __ldg(fs.w_next + j) + (j > 0 ? __ldg(fs.w_next + j - 1) : 0.f);
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < g.N;
         k += (long long)gridDim.x * blockDim.x) {
        int ix, iy, iz;
        unflatten(g, k, ix, iy, iz);
        const size_t e = (size_t)plane * g.N + k;
        const float zv = jacobi_inv(__ldg(dT + e), neighbour_count(g, ix, iy, iz), tdiag, cf) * __ldg(r + e);
        p[e] = fmaf(beta, p[e], zv);
    }
}

cudaError_t launch_pcg_init(const Geom& g, const FrameSet& fs, const Coef& cf, const float* grad,
                            const float* dT, float* x, float* r, float* p, double* partials,
                            DevScalars* S, PcgArgs a, cudaStream_t s) {
    dim3 grid(vec_blocks_x(g), fs.nK * g.d);
    if (g.d == 2)
        pcg_init_kernel<2><<<grid, kThreads, 0, s>>>(g, fs, cf, grad, dT, x, r, p, partials, S, a);
    else
        pcg_init_kernel<3><<<grid, kThreads, 0, s>>>(g, fs, cf, grad, dT, x, r, p, partials, S, a);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_pcg_update(const Geom& g, const FrameSet& fs, const Coef& cf, const float* dT,
                              float* x, float* r, const float* p, const float* q,
                              double* partials, DevScalars* S, PcgArgs a, cudaStream_t s) {
    dim3 grid(vec_blocks_x(g), fs.nK * g.d);
    if (g.d == 2)
        pcg_update_kernel<2><<<grid, kThreads, 0, s>>>(g, fs, cf, dT, x, r, p, q, partials, S, a);
    else
        pcg_update_kernel<3><<<grid, kThreads, 0, s>>>(g, fs, cf, dT, x, r, p, q, partials, S, a);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_pcg_pupdate(const Geom& g, const FrameSet& fs, const Coef& cf, const float* dT,
                               const float* r, float* p, DevScalars* S, cudaStream_t s) {
    dim3 grid(vec_blocks_x(g), fs.nK * g.d);
    if (g.d == 2)
        pcg_pupdate_kernel<2><<<grid, kThreads, 0, s>>>(g, fs, cf, dT, r, p, S);
    else
        pcg_pupdate_kernel<3><<<grid, kThreads, 0, s>>>(g, fs, cf, dT, r, p, S);
    count_launches(1);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(kThreads)
dot2_kernel(const float* __restrict__ a, const float* __restrict__ b, size_t n,
            double* __restrict__ partials, unsigned int* ticket, double* out) {
    float acc[2] = {0.f, 0.f};
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const float bv = __ldg(b + i);
        acc[0] = fmaf(__ldg(a + i), bv, acc[0]);
        acc[1] = fmaf(bv, bv, acc[1]);
    }
    grid_reduce<2>(acc, partials, ticket, out);
}

cudaError_t launch_dot2(const float* a, const float* b, size_t n, double* partials,
                        unsigned int* ticket, double* out, cudaStream_t s) {
    const unsigned blocks = blocks_for((long long)((n + 7) / 8), kThreads, 4096);
    dot2_kernel<<<blocks, kThreads, 0, s>>>(a, b, n, partials, ticket, out);
    count_launches(1);
    return cudaGetLastError();
}

__global__ void axpy_kernel(const float* __restrict__ x, const float* __restrict__ d, float t,
                            float* __restrict__ y, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        y[i] = fmaf(t, __ldg(d + i), __ldg(x + i));
}

cudaError_t launch_axpy(const float* x, const float* d, float t, float* y, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    axpy_kernel<<<blocks_for((long long)n, kThreads, 8192), kThreads, 0, s>>>(x, d, t, y, n);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace stml
