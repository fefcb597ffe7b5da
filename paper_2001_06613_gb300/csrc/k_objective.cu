// Objective of eq. (1) with the regulariser S and the penalty P of Sec. 2,
// its gradient, and the warped-image derivatives the Gauss-Newton model needs.
//
// Two passes over the frames of K:
//  1. warp_mean: for every pixel, loop over the frames: a_k = T_k(x + u_k(x))
//     and grad T_k there (linear interpolation, zero outside); per-pixel
//     means abar = mean_k a_k and ubar = mean_k u_k (compensated sums);
//  2. residual_grad: for every (frame, pixel): r_k = a_k - abar,
//     g_k = hd r_k grad T_k + alpha hd B^T B u_k + alpha_t hd (L_t u)_k
//           + 2 lambda hd ubar / |K|,
//     and the FP64 totals of D, S, P, |g|^2, |u|^2.
// The fields may be given as u + t du (an Armijo trial point) without
// forming that array.
#include "kernels.h"

namespace stml {

struct FieldView {
    const float* __restrict__ u;
    const float* __restrict__ du;
    float t;
    __device__ __forceinline__ float operator()(size_t i) const {
        return du ? fmaf(t, __ldg(du + i), __ldg(u + i)) : __ldg(u + i);
    }
};

// Compensated (Neumaier) running sum in float.
struct KSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float t = s + v;
        if (fabsf(s) >= fabsf(v))
            c += (s - t) + v;
        else
            c += (v - t) + s;
        s = t;
    }
    __device__ __forceinline__ float value() const { return s + c; }
};

// CTA = 32 consecutive pixels x 8 frame groups (one warp each); warp w
// visits the frames j = w, w + 8, ...; the per-pixel sums of the 8 warps are
// combined in warp order.
template <int D, bool WRITE_DT>
__global__ void __launch_bounds__(kThreads)
warp_mean_kernel(const float* __restrict__ T, Geom g, FrameSet fs, FieldView U,
                 float* __restrict__ a, float* __restrict__ dT, float* __restrict__ mean_a,
                 float* __restrict__ mean_u) {
    __shared__ float sh[kFrameGroups][1 + D][kPixPerCta];
    const int tx = threadIdx.x % kPixPerCta, fg = threadIdx.x / kPixPerCta;
    const long long p = (long long)blockIdx.x * kPixPerCta + tx;
    const bool valid = p < g.N;
    KSum sa;
    KSum su[D];
    if (valid) {
        int x, y, z;
        unflatten(g, p, x, y, z);
        for (int j = fg; j < fs.nK; j += kFrameGroups) {
            const float* Tk = T + (size_t)__ldg(fs.frames + j) * g.N;
            float uv[D];
#pragma unroll
            for (int c = 0; c < D; ++c) uv[c] = U(((size_t)j * D + c) * g.N + p);
            float val, gr[D];
            if constexpr (D == 2)
                interp2(Tk, g, x, y, uv[0], uv[1], val, gr[0], gr[1]);
            else
                interp3(Tk, g, x, y, z, uv[0], uv[1], uv[2], val, gr[0], gr[1], gr[2]);
            a[(size_t)j * g.N + p] = val;
            if constexpr (WRITE_DT) {
#pragma unroll
                for (int c = 0; c < D; ++c) dT[((size_t)j * D + c) * g.N + p] = gr[c];
            }
            sa.add(val);
#pragma unroll
            for (int c = 0; c < D; ++c) su[c].add(uv[c]);
        }
    }
    sh[fg][0][tx] = sa.value();
#pragma unroll
    for (int c = 0; c < D; ++c) sh[fg][1 + c][tx] = su[c].value();
    __syncthreads();
    if (valid && fg < 1 + D) {
        // warp fg combines quantity fg (0: a, 1..D: u components)
        KSum tot;
        for (int w = 0; w < kFrameGroups; ++w) tot.add(sh[w][fg][tx]);
        const float m = tot.value() / (float)fs.nK;
        if (fg == 0)
            mean_a[p] = m;
        else
            mean_u[(size_t)(fg - 1) * g.N + p] = m;
    }
}

// (B^T B w)(p) h^2 and the forward-difference energy from p (h^2 units) for
// a plane read through the field view.
template <int D>
__device__ __forceinline__ void stencil_terms(const FieldView& U, size_t base, const Geom& g,
                                              long long p, int x, int y, int z, float& lap,
                                              float& fwd2) {
    const float c = U(base + p);
    lap = 0.f;
    fwd2 = 0.f;
    if (x > 0) lap += c - U(base + p - 1);
    if (x < g.nx - 1) {
        const float n = U(base + p + 1);
        lap += c - n;
        fwd2 += (n - c) * (n - c);
    }
    if (y > 0) lap += c - U(base + p - g.nx);
    if (y < g.ny - 1) {
        const float n = U(base + p + g.nx);
        lap += c - n;
        fwd2 += (n - c) * (n - c);
    }
    if constexpr (D == 3) {
        const long long s = (long long)g.nx * g.ny;
        if (z > 0) lap += c - U(base + p - s);
        if (z < g.nz - 1) {
            const float n = U(base + p + s);
            lap += c - n;
            fwd2 += (n - c) * (n - c);
        }
    }
}

// Element (j, p) per thread; blockIdx.y = j.  Values reduced:
// 0 D, 1 S_x, 2 S_t, 3 P, 4 |g|^2, 5 |u|^2.
template <int D, bool GRAD>
__global__ void __launch_bounds__(kThreads)
residual_grad_kernel(Geom g, FrameSet fs, Coef cf, FieldView U, const float* __restrict__ a,
                     const float* __restrict__ mean_a, const float* __restrict__ mean_u,
                     const float* __restrict__ dT, float* __restrict__ grad,
                     double* __restrict__ partials, unsigned int* ticket, double* out) {
    const int j = blockIdx.y;
    float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const float w_next = __ldg(fs.w_next + j);
    const float w_prev = j > 0 ? __ldg(fs.w_next + j - 1) : 0.f;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < g.N;
         p += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        unflatten(g, p, x, y, z);
        const float r = __ldg(a + (size_t)j * g.N + p) - __ldg(mean_a + p);
        acc[0] += cf.half_hd * r * r;
        float pen = 0.f;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const size_t base = ((size_t)j * D + c) * g.N;
            float lap, fwd2;
            stencil_terms<D>(U, base, g, p, x, y, z, lap, fwd2);
            acc[1] += 0.5f * cf.alpha_hd * cf.inv_h2 * fwd2;
            const float uc = U(base + p);
            float tgrad = 0.f;
            if (cf.alphat_hd != 0.f) {
                if (j + 1 < fs.nK) {
                    const float un = U(base + (size_t)D * g.N + p);
                    acc[2] += 0.5f * cf.alphat_hd * w_next * (un - uc) * (un - uc);
                    tgrad += w_next * (uc - un);
                }
                if (j > 0) tgrad += w_prev * (uc - U(base - (size_t)D * g.N + p));
            }
            const float ub = __ldg(mean_u + (size_t)c * g.N + p);
            pen += ub * ub;
            if constexpr (GRAD) {
                const float gv = cf.hd * r * __ldg(dT + base + p) + cf.alpha_hd * cf.inv_h2 * lap +
                                 cf.alphat_hd * tgrad + cf.pen_g * ub;
                grad[base + p] = gv;
                acc[4] += gv * gv;
            }
            acc[5] += uc * uc;
        }
        if (j == 0) acc[3] += cf.lam_hd * pen;
    }
    if (grid_reduce<6>(acc, partials, ticket, out) && threadIdx.x == 0) {
        // out: D, Sx, St, P, |g|^2, |u|^2  ->  J, D, S, P, |g|^2, |u|^2
        const double Dv = out[0], Sx = out[1], St = out[2], Pv = out[3];
        out[0] = Dv + Sx + St + Pv;
        out[1] = Dv;
        out[2] = Sx + St;
        out[3] = Pv;
    }
}

static unsigned eval_blocks_x(const Geom& g, int nK) {
    // about 4 elements per thread, at least one CTA per frame row
    long long per = (g.N + (long long)kThreads * 4 - 1) / ((long long)kThreads * 4);
    if (per < 1) per = 1;
    if (per > 65535) per = 65535;
    (void)nK;
    return (unsigned)per;
}

size_t partials_needed(const Geom& g, int nK) {
    return (size_t)eval_blocks_x(g, nK) * nK * kMaxRed + 1024 * kMaxRed;
}

cudaError_t launch_eval(const float* T, const Geom& g, const FrameSet& fs, const Coef& cf,
                        const float* u, const float* du, float t, float* dT, float* grad,
                        EvalWork& w, unsigned int* ticket, double* out, cudaStream_t s) {
    if (fs.nK <= 0) return cudaErrorInvalidValue;
    FieldView U{u, du, t};
    const unsigned gx = (unsigned)((g.N + kPixPerCta - 1) / kPixPerCta);
    const bool want = grad != nullptr;
    if (g.d == 2) {
        if (want)
            warp_mean_kernel<2, true><<<gx, kThreads, 0, s>>>(T, g, fs, U, w.a, dT, w.mean_a, w.mean_u);
        else
            warp_mean_kernel<2, false><<<gx, kThreads, 0, s>>>(T, g, fs, U, w.a, dT, w.mean_a, w.mean_u);
    } else {
        if (want)
            warp_mean_kernel<3, true><<<gx, kThreads, 0, s>>>(T, g, fs, U, w.a, dT, w.mean_a, w.mean_u);
        else
            warp_mean_kernel<3, false><<<gx, kThreads, 0, s>>>(T, g, fs, U, w.a, dT, w.mean_a, w.mean_u);
    }
    dim3 grid(eval_blocks_x(g, fs.nK), fs.nK);
    if ((size_t)grid.x * grid.y * kMaxRed > w.partials_cap) return cudaErrorInvalidValue;
    if (g.d == 2) {
        if (want)
            residual_grad_kernel<2, true><<<grid, kThreads, 0, s>>>(g, fs, cf, U, w.a, w.mean_a, w.mean_u, dT, grad, w.partials, ticket, out);
        else
            residual_grad_kernel<2, false><<<grid, kThreads, 0, s>>>(g, fs, cf, U, w.a, w.mean_a, w.mean_u, dT, grad, w.partials, ticket, out);
    } else {
        if (want)
            residual_grad_kernel<3, true><<<grid, kThreads, 0, s>>>(g, fs, cf, U, w.a, w.mean_a, w.mean_u, dT, grad, w.partials, ticket, out);
        else
            residual_grad_kernel<3, false><<<grid, kThreads, 0, s>>>(g, fs, cf, U, w.a, w.mean_a, w.mean_u, dT, grad, w.partials, ticket, out);
    }
    count_launches(2);
    return cudaGetLastError();
}

}  // namespace stml
