// Gauss-Newton Hessian product of the groupwise objective:
//   (Hv)_k = hd grad T_k (s_k - sbar) + alpha hd B^T B v_k + alpha_t hd (L_t v)_k
//            + 2 lambda hd / |K|^2 sum_j v_j,          s_k = grad T_k . v_k,
// i.e. J^T J v for the residual r = (I - 11^T/|K|) a plus the quadratic terms.
// The frame mean sbar and the frame sum of v couple all frames of a pixel.
//
// Two-pass form: hv_sums computes sbar and sum_j v_j per pixel (CTA = 32
// pixels x 8 frame groups), hv_apply writes Hv per (frame, pixel) with the
// 2d+1-point stencil of B^T B and reduces <v, Hv> in FP64.
#include "kernels.h"

namespace stml {

namespace {
struct KSumH {
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
}  // namespace

template <int D>
__global__ void __launch_bounds__(kThreads)
hv_sums_kernel(Geom g, int nK, const float* __restrict__ dT, const float* __restrict__ v,
               float* __restrict__ mean_s, float* __restrict__ sum_v, const DevScalars* pcg) {
    if (pcg && !pcg->cg_active) return;
    __shared__ float sh[kFrameGroups][1 + D][kPixPerCta];
    const int tx = threadIdx.x % kPixPerCta, fg = threadIdx.x / kPixPerCta;
    const long long p = (long long)blockIdx.x * kPixPerCta + tx;
    const bool valid = p < g.N;
    KSumH ss;
    KSumH sv[D];
    if (valid) {
        for (int j = fg; j < nK; j += kFrameGroups) {
            float s = 0.f;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const size_t e = ((size_t)j * D + c) * g.N + p;
                const float vv = __ldg(v + e);
                s = fmaf(__ldg(dT + e), vv, s);
                sv[c].add(vv);
            }
            ss.add(s);
        }
    }
    sh[fg][0][tx] = ss.value();
#pragma unroll
    for (int c = 0; c < D; ++c) sh[fg][1 + c][tx] = sv[c].value();
    __syncthreads();
    if (valid && fg < 1 + D) {
        KSumH tot;
        for (int w = 0; w < kFrameGroups; ++w) tot.add(sh[w][fg][tx]);
        if (fg == 0)
            mean_s[p] = tot.value() / (float)nK;
        else
            sum_v[(size_t)(fg - 1) * g.N + p] = tot.value();
    }
}

template <int D>
__global__ void __launch_bounds__(kThreads)
hv_apply_kernel(Geom g, FrameSet fs, Coef cf, const float* __restrict__ dT,
                const float* __restrict__ v, const float* __restrict__ mean_s,
                const float* __restrict__ sum_v, float* __restrict__ Hv,
                double* __restrict__ partials, unsigned int* ticket, double* out,
                DevScalars* pcg) {
    if (pcg && !pcg->cg_active) return;
    const int j = blockIdx.y;
    const float w_next = __ldg(fs.w_next + j);
    const float w_prev = j > 0 ? __ldg(fs.w_next + j - 1) : 0.f;
    float acc[1] = {0.f};
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < g.N;
         p += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        unflatten(g, p, x, y, z);
        float dTv[D], vv[D];
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const size_t e = ((size_t)j * D + c) * g.N + p;
            dTv[c] = __ldg(dT + e);
            vv[c] = __ldg(v + e);
            s = fmaf(dTv[c], vv[c], s);
        }
        const float ds = cf.hd * (s - __ldg(mean_s + p));
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const size_t base = ((size_t)j * D + c) * g.N;
            const float lap = neg_laplacian_h2(v + base, g, p, x, y, z);
            float h = fmaf(ds, dTv[c], cf.alpha_hd * cf.inv_h2 * lap);
            if (cf.alphat_hd != 0.f) {
                float tl = 0.f;
                if (j + 1 < fs.nK) tl += w_next * (vv[c] - __ldg(v + base + (size_t)D * g.N + p));
                if (j > 0) tl += w_prev * (vv[c] - __ldg(v + base - (size_t)D * g.N + p));
                h = fmaf(cf.alphat_hd, tl, h);
            }
            h = fmaf(cf.pen_h, __ldg(sum_v + (size_t)c * g.N + p), h);
            Hv[base + p] = h;
            acc[0] = fmaf(vv[c], h, acc[0]);
        }
    }
    if (grid_reduce<1>(acc, partials, ticket, out) && threadIdx.x == 0 && pcg) {
        const double pq = out[0];
        pcg->pq = pq;
        if (!(pq > 0.0)) {
            pcg->cg_flag = CG_BREAKDOWN;
            pcg->cg_active = 0;
        } else {
            pcg->alpha = pcg->rho / pq;
        }
    }
}

static unsigned apply_blocks_x(const Geom& g) {
    long long per = (g.N + (long long)kThreads * 4 - 1) / ((long long)kThreads * 4);
    if (per < 1) per = 1;
    if (per > 65535) per = 65535;
    return (unsigned)per;
}

size_t hessvec_partials(const Geom& g, int nK) { return (size_t)apply_blocks_x(g) * (size_t)nK; }

cudaError_t launch_hessvec(const Geom& g, const FrameSet& fs, const Coef& cf, const float* dT,
                           const float* v, float* Hv, HessWork& w, unsigned int* ticket,
                           double* out, DevScalars* pcg, cudaStream_t s) {
    if (fs.nK <= 0) return cudaErrorInvalidValue;
    const unsigned gx = (unsigned)((g.N + kPixPerCta - 1) / kPixPerCta);
    dim3 grid(apply_blocks_x(g), fs.nK);
    if ((size_t)grid.x * grid.y > w.partials_cap) return cudaErrorInvalidValue;
    if (g.d == 2) {
        hv_sums_kernel<2><<<gx, kThreads, 0, s>>>(g, fs.nK, dT, v, w.mean_s, w.sum_v, pcg);
        hv_apply_kernel<2><<<grid, kThreads, 0, s>>>(g, fs, cf, dT, v, w.mean_s, w.sum_v, Hv,
                                                     w.partials, ticket, out, pcg);
    } else {
        hv_sums_kernel<3><<<gx, kThreads, 0, s>>>(g, fs.nK, dT, v, w.mean_s, w.sum_v, pcg);
        hv_apply_kernel<3><<<grid, kThreads, 0, s>>>(g, fs, cf, dT, v, w.mean_s, w.sum_v, Hv,
                                                     w.partials, ticket, out, pcg);
    }
    count_launches(2);
    return cudaGetLastError();
}

}  // namespace stml
