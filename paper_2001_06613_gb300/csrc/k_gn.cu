// Gauss-Newton Hessian product and the PCG vector kernels around it.
//
//   (Hv)_k = hd grad T_k (s_k - sbar) + alpha hd B^T B v_k + alpha_t hd (L_t v)_k
//            + 2 lambda hd / |K|^2 sum_j v_j,          s_k = grad T_k . v_k
//
// The Hessian product needs two per-pixel sums over all frames of K (sbar and
// sum_j v_j).  They are produced by the kernel that writes v: in the PCG loop
// the search direction p is written by `dir_kernel`, which visits all frames
// of a pixel anyway (p = M^-1 r + beta p); it reduces sbar and sum_j p_j over
// the frames in the same pass.  The Hessian product itself (`apply_kernel`) is
// then an element-wise stencil stream: it reads v (and its stencil
// neighbours, served from L1/L2), grad T and the sums, writes Hv and reduces
// <v, Hv>.  Per PCG iteration and pixel-frame: apply 12d bytes, update 28d,
// direction 16d -- every array read or written once.
//
// The Jacobi preconditioner is computed from grad T where it is needed
// (`jacobi_inv`, one rounding sequence everywhere), so no M^-1 array exists.
#include "kernels.h"

namespace stml {

namespace {

__device__ __forceinline__ float4 ld4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float4 ld4rw(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

template <int VEC>
struct V;
template <>
struct V<4> {
    float a[4];
    __device__ __forceinline__ void load(const float* p) {
        const float4 q = ld4(p);
        a[0] = q.x; a[1] = q.y; a[2] = q.z; a[3] = q.w;
    }
    __device__ __forceinline__ void load_rw(const float* p) {
        const float4 q = ld4rw(p);
        a[0] = q.x; a[1] = q.y; a[2] = q.z; a[3] = q.w;
    }
    __device__ __forceinline__ void store(float* p) const { st4(p, make_float4(a[0], a[1], a[2], a[3])); }
    __device__ __forceinline__ void zero() { a[0] = a[1] = a[2] = a[3] = 0.f; }
};
template <>
struct V<1> {
    float a[1];
    __device__ __forceinline__ void load(const float* p) { a[0] = __ldg(p); }
    __device__ __forceinline__ void load_rw(const float* p) { a[0] = *p; }
    __device__ __forceinline__ void store(float* p) const { *p = a[0]; }
    __device__ __forceinline__ void zero() { a[0] = 0.f; }
};

// Position of pixel p: x, y, z via multiply-high division.
__device__ __forceinline__ void pix_pos(const PixIndex& pi, unsigned p, int& x, int& y, int& z) {
    const unsigned r = pi.nx.div(p);
    x = (int)(p - r * pi.nx.d);
    const unsigned zz = pi.ny.div(r);
    y = (int)(r - zz * pi.ny.d);
    z = (int)zz;
}

}  // namespace

// Inverse of the Jacobi diagonal of the Gauss-Newton Hessian at one element:
// hd (1 - 1/|K|) (d_c T_k)^2 + alpha hd nnb / h^2 + alpha_t hd (w_prev + w_next)
// + 2 lambda hd / |K|^2 (explicit roundings: every kernel gets the same value).
__device__ __forceinline__ float jacobi_inv(float dt, int nnb, float tdiag, const Coef& cf) {
    float dg = __fmul_rn(__fmul_rn(cf.diag_D, dt), dt);
    dg = __fadd_rn(dg, __fmul_rn(__fmul_rn(cf.alpha_hd, cf.inv_h2), (float)nnb));
    dg = __fadd_rn(dg, __fmul_rn(cf.alphat_hd, tdiag));
    dg = __fadd_rn(dg, cf.pen_h);
    return dg > 0.f ? __frcp_rn(dg) : 1.0f;   // zero only when alpha = lambda = 0 and grad T = 0
}

// ----------------------------------------------------------------- direction
// MODE 0: sums of a given v.  MODE 1: p = M^-1 r + beta p (PCG step), sums of
// the new p.  MODE 2: r = -g, p = M^-1 r, x = 0, <r, M^-1 r>, |r|^2 (PCG start),
// sums of p.  CTA = SEG consecutive pixels x FG frame groups; group f visits
// the frames f, f + FG, ...; the per-pixel sums of the groups are combined in
// group order.  Writes mean_s[p] = sum_k s_k / |K| and sum_v[c][p].
template <int D, int VEC, int MODE>
__global__ void __launch_bounds__(kThreads)
dir_kernel(Geom g, PixIndex pi, FrameSet fs, Coef cf, const float* __restrict__ dT, float* __restrict__ v,
           float* __restrict__ r, const float* __restrict__ grad, float* __restrict__ x,
           float* __restrict__ mean_s, float* __restrict__ sum_v, double* __restrict__ partials,
           DevScalars* S, PcgArgs a) {
    if (MODE == 1 && !S->cg_active) return;
    constexpr int TPR = VEC == 4 ? 16 : 32, SEG = TPR * VEC, FG = kThreads / TPR, NR = 1 + D;
    __shared__ float sh[FG][NR][SEG];
    const int lane = threadIdx.x % TPR, fg = threadIdx.x / TPR;
    const unsigned p = blockIdx.x * SEG + lane * VEC;
    const bool valid = p < (unsigned)g.N;
    const size_t N = (size_t)g.N;
    float beta = 0.f;
    if constexpr (MODE == 1) beta = (float)S->beta;
    int nnb[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) nnb[e] = 0;
    if (MODE != 0 && valid) {
        int px, py, pz;
        pix_pos(pi, p, px, py, pz);
#pragma unroll
        for (int e = 0; e < VEC; ++e) nnb[e] = neighbour_count(g, px + e, py, pz);
    }
    float as[VEC], av[D][VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
        as[e] = 0.f;
#pragma unroll
        for (int c = 0; c < D; ++c) av[c][e] = 0.f;
    }
    float rz = 0.f, rr = 0.f;
    if (valid) {
        for (int j = fg; j < fs.nK; j += FG) {
            float tdiag = 0.f;
            if (MODE != 0)
                tdiag = (j + 1 < fs.nK ? __ldg(fs.w_next + j) : 0.f) + (j > 0 ? __ldg(fs.w_next + j - 1) : 0.f);
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const size_t e0 = ((size_t)j * D + c) * N + p;
                V<VEC> dt, pv;
                dt.load(dT + e0);
                if constexpr (MODE == 0) {
                    pv.load(v + e0);
                } else if constexpr (MODE == 1) {
                    V<VEC> rv;
                    rv.load(r + e0);
                    pv.load_rw(v + e0);
#pragma unroll
                    for (int e = 0; e < VEC; ++e)
                        pv.a[e] = fmaf(beta, pv.a[e], jacobi_inv(dt.a[e], nnb[e], tdiag, cf) * rv.a[e]);
                    pv.store(v + e0);
                } else {
                    V<VEC> gv, rv, zero;
                    gv.load(grad + e0);
                    zero.zero();
#pragma unroll
                    for (int e = 0; e < VEC; ++e) {
                        rv.a[e] = -gv.a[e];
                        pv.a[e] = jacobi_inv(dt.a[e], nnb[e], tdiag, cf) * rv.a[e];
                        rz = fmaf(rv.a[e], pv.a[e], rz);
                        rr = fmaf(rv.a[e], rv.a[e], rr);
                    }
                    rv.store(r + e0);
                    pv.store(v + e0);
                    zero.store(x + e0);
                }
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    as[e] = fmaf(dt.a[e], pv.a[e], as[e]);
                    av[c][e] += pv.a[e];
                }
            }
        }
    }
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
        sh[fg][0][lane * VEC + e] = as[e];
#pragma unroll
        for (int c = 0; c < D; ++c) sh[fg][1 + c][lane * VEC + e] = av[c][e];
    }
    __syncthreads();
    const float invK = 1.0f / (float)fs.nK;
    for (int i = threadIdx.x; i < NR * SEG; i += blockDim.x) {
        const int q = i / SEG, k = i - q * SEG;
        const unsigned pp = blockIdx.x * SEG + k;
        if (pp >= (unsigned)g.N) continue;
        float s = 0.f;
#pragma unroll
        for (int w = 0; w < FG; ++w) s += sh[w][q][k];
        if (q == 0)
            mean_s[pp] = s * invK;
        else
            sum_v[(size_t)(q - 1) * N + pp] = s;
    }
    if constexpr (MODE == 2) {
        float acc[2] = {rz, rr};
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
}

// ----------------------------------------------------------------- apply
// Element = (frame j = blockIdx.y, VEC pixels); all D components.
template <int D, int VEC>
__global__ void __launch_bounds__(kThreads)
apply_kernel(Geom g, PixIndex pi, FastDiv chunks, long long items, FrameSet fs, Coef cf,
             const float* __restrict__ dT, const float* __restrict__ v, const float* __restrict__ mean_s,
             const float* __restrict__ sum_v, float* __restrict__ Hv, double* __restrict__ partials,
             unsigned int* ticket, double* out, DevScalars* pcg) {
    if (pcg && !pcg->cg_active) return;
    const size_t N = (size_t)g.N;
    const int lane = threadIdx.x & 31;
    float acc[1] = {0.f};
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
    const int j = (int)chunks.div((unsigned)it);
    const unsigned ch = (unsigned)it - (unsigned)j * chunks.d;
    const unsigned p = (ch * kThreads + threadIdx.x) * VEC;
    const bool valid = p < (unsigned)g.N;
    const float w_next = (cf.alphat_hd != 0.f && j + 1 < fs.nK) ? __ldg(fs.w_next + j) : 0.f;
    const float w_prev = (cf.alphat_hd != 0.f && j > 0) ? __ldg(fs.w_next + j - 1) : 0.f;
    int x = 0, y = 0, z = 0;
    if (valid) pix_pos(pi, p, x, y, z);
    V<VEC> vc[D], dt[D];
    float s[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) s[e] = 0.f;
#pragma unroll
    for (int c = 0; c < D; ++c) {
        const size_t e0 = ((size_t)j * D + c) * N + p;
        if (valid) {
            vc[c].load(v + e0);
            dt[c].load(dT + e0);
        } else {
            vc[c].zero();
            dt[c].zero();
        }
#pragma unroll
        for (int e = 0; e < VEC; ++e) s[e] = fmaf(dt[c].a[e], vc[c].a[e], s[e]);
    }
    float ds[VEC], sv[D][VEC];
    if (valid) {
        V<VEC> ms;
        ms.load(mean_s + p);
#pragma unroll
        for (int e = 0; e < VEC; ++e) ds[e] = cf.hd * (s[e] - ms.a[e]);
#pragma unroll
        for (int c = 0; c < D; ++c) {
            V<VEC> t;
            t.load(sum_v + (size_t)c * N + p);
#pragma unroll
            for (int e = 0; e < VEC; ++e) sv[c][e] = t.a[e];
        }
    }
#pragma unroll
    for (int c = 0; c < D; ++c) {
        const size_t e0 = ((size_t)j * D + c) * N + p;
        // x neighbours: the neighbouring lane's value when it holds the same row
        const float up_l = __shfl_up_sync(0xffffffffu, vc[c].a[VEC - 1], 1);
        const float dn_r = __shfl_down_sync(0xffffffffu, vc[c].a[0], 1);
        if (!valid) continue;
        float left = 0.f, right = 0.f;
        if (x > 0) left = (lane > 0) ? up_l : __ldg(v + e0 - 1);
        if (x + VEC < g.nx) right = (lane < 31) ? dn_r : __ldg(v + e0 + VEC);
        float lap[VEC];
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
            const float ce = vc[c].a[e];
            const float le = e == 0 ? left : vc[c].a[e - 1];
            const float re = e == VEC - 1 ? right : vc[c].a[e + 1];
            float lp = 0.f;
            if (x + e > 0) lp += ce - le;
            if (x + e < g.nx - 1) lp += ce - re;
            lap[e] = lp;
        }
        V<VEC> nb;
        if (y > 0) {
            nb.load(v + e0 - g.nx);
#pragma unroll
            for (int e = 0; e < VEC; ++e) lap[e] += vc[c].a[e] - nb.a[e];
        }
        if (y < g.ny - 1) {
            nb.load(v + e0 + g.nx);
#pragma unroll
            for (int e = 0; e < VEC; ++e) lap[e] += vc[c].a[e] - nb.a[e];
        }
        if constexpr (D == 3) {
            const size_t sz = (size_t)g.nx * g.ny;
            if (z > 0) {
                nb.load(v + e0 - sz);
#pragma unroll
                for (int e = 0; e < VEC; ++e) lap[e] += vc[c].a[e] - nb.a[e];
            }
            if (z < g.nz - 1) {
                nb.load(v + e0 + sz);
#pragma unroll
                for (int e = 0; e < VEC; ++e) lap[e] += vc[c].a[e] - nb.a[e];
            }
        }
        V<VEC> h;
#pragma unroll
        for (int e = 0; e < VEC; ++e) h.a[e] = fmaf(ds[e], dt[c].a[e], fmaf(cf.alpha_hd * cf.inv_h2, lap[e], cf.pen_h * sv[c][e]));
        if (w_next != 0.f) {
            nb.load(v + e0 + (size_t)D * N);
#pragma unroll
            for (int e = 0; e < VEC; ++e) h.a[e] = fmaf(cf.alphat_hd * w_next, vc[c].a[e] - nb.a[e], h.a[e]);
        }
        if (w_prev != 0.f) {
            nb.load(v + e0 - (size_t)D * N);
#pragma unroll
            for (int e = 0; e < VEC; ++e) h.a[e] = fmaf(cf.alphat_hd * w_prev, vc[c].a[e] - nb.a[e], h.a[e]);
        }
        h.store(Hv + e0);
#pragma unroll
        for (int e = 0; e < VEC; ++e) acc[0] = fmaf(vc[c].a[e], h.a[e], acc[0]);
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

// ----------------------------------------------------------------- update
// x += alpha p, r -= alpha q, z = M^-1 r; <r, z>, |r|^2 -> convergence, beta.
// Element = (plane = blockIdx.y, VEC pixels).
template <int D, int VEC>
__global__ void __launch_bounds__(kThreads)
update_kernel(Geom g, PixIndex pi, FastDiv chunks, long long items, FrameSet fs, Coef cf,
              const float* __restrict__ dT, float* __restrict__ x, float* __restrict__ r,
              const float* __restrict__ p, const float* __restrict__ q, double* __restrict__ partials,
              DevScalars* S, PcgArgs a) {
    if (!S->cg_active) return;
    const float al = (float)S->alpha;
    float acc[2] = {0.f, 0.f};
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
    const int plane = (int)chunks.div((unsigned)it);
    const unsigned ch = (unsigned)it - (unsigned)plane * chunks.d;
    const int j = plane / D;
    const float tdiag = (j + 1 < fs.nK ? __ldg(fs.w_next + j) : 0.f) + (j > 0 ? __ldg(fs.w_next + j - 1) : 0.f);
    const unsigned px = (ch * kThreads + threadIdx.x) * VEC;
    if (px < (unsigned)g.N) {
        int xx, yy, zz;
        pix_pos(pi, px, xx, yy, zz);
        const size_t e0 = (size_t)plane * g.N + px;
        V<VEC> dt, pv, qv, xv, rv;
        dt.load(dT + e0);
        pv.load(p + e0);
        qv.load(q + e0);
        xv.load_rw(x + e0);
        rv.load_rw(r + e0);
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
            xv.a[e] = fmaf(al, pv.a[e], xv.a[e]);
            rv.a[e] = fmaf(-al, qv.a[e], rv.a[e]);
            const float zv = jacobi_inv(dt.a[e], neighbour_count(g, xx + e, yy, zz), tdiag, cf) * rv.a[e];
            acc[0] = fmaf(rv.a[e], zv, acc[0]);
            acc[1] = fmaf(rv.a[e], rv.a[e], acc[1]);
        }
        xv.store(x + e0);
        rv.store(r + e0);
    }
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

// ----------------------------------------------------------------- launchers
PixIndex make_pix_index(const Geom& g) {
    PixIndex pi;
    pi.nx = FastDiv::make((unsigned)g.nx);
    pi.ny = FastDiv::make((unsigned)g.ny);
    return pi;
}

static bool vec4_ok(const Geom& g, std::initializer_list<const void*> ptrs) {
    if (g.nx % 4) return false;
    for (const void* q : ptrs)
        if (q && ((uintptr_t)q & 15u)) return false;
    return true;
}

template <int MODE>
static cudaError_t dir_launch(const Geom& g, const FrameSet& fs, const Coef& cf, const float* dT, float* v, float* r,
                              const float* grad, float* x, float* mean_s, float* sum_v, double* partials,
                              DevScalars* S, PcgArgs a, cudaStream_t s) {
    const PixIndex pi = make_pix_index(g);
    const bool v4 = vec4_ok(g, {dT, v, r, grad, x});
    const int seg = v4 ? 64 : 32;
    const unsigned blocks = (unsigned)((g.N + seg - 1) / seg);
    if (g.d == 2) {
        if (v4)
            dir_kernel<2, 4, MODE><<<blocks, kThreads, 0, s>>>(g, pi, fs, cf, dT, v, r, grad, x, mean_s, sum_v, partials, S, a);
        else
            dir_kernel<2, 1, MODE><<<blocks, kThreads, 0, s>>>(g, pi, fs, cf, dT, v, r, grad, x, mean_s, sum_v, partials, S, a);
    } else {
        if (v4)
            dir_kernel<3, 4, MODE><<<blocks, kThreads, 0, s>>>(g, pi, fs, cf, dT, v, r, grad, x, mean_s, sum_v, partials, S, a);
        else
            dir_kernel<3, 1, MODE><<<blocks, kThreads, 0, s>>>(g, pi, fs, cf, dT, v, r, grad, x, mean_s, sum_v, partials, S, a);
    }
    count_launches(1);
    return cudaGetLastError();
}

constexpr int kGridStride = 152 * 8;   // CTAs of the grid-stride launches (8 per SM of a GB300)

size_t gn_partials(const Geom& g, int nK) {
    const size_t dir = (size_t)((g.N + 31) / 32) * 2;
    const size_t gs = (size_t)kGridStride * 2;
    (void)nK;
    return dir > gs ? dir : gs;
}

cudaError_t launch_hess_sums(const Geom& g, const FrameSet& fs, const float* dT, const float* v, float* mean_s,
                             float* sum_v, cudaStream_t s) {
    Coef cf{};
    return dir_launch<0>(g, fs, cf, dT, const_cast<float*>(v), nullptr, nullptr, nullptr, mean_s, sum_v, nullptr,
                         nullptr, PcgArgs{0.f, 0}, s);
}

cudaError_t launch_hess_apply(const Geom& g, const FrameSet& fs, const Coef& cf, const float* dT, const float* v,
                              const float* mean_s, const float* sum_v, float* Hv, double* partials,
                              size_t partials_cap, unsigned int* ticket, double* out, DevScalars* pcg,
                              cudaStream_t s) {
    const PixIndex pi = make_pix_index(g);
    const bool v4 = vec4_ok(g, {dT, v, Hv, mean_s, sum_v});
    const int vec = v4 ? 4 : 1;
    const long long cpf = (g.N + (long long)kThreads * vec - 1) / ((long long)kThreads * vec);
    const long long items = cpf * fs.nK;
    const unsigned grid = (unsigned)(items < kGridStride ? items : kGridStride);
    if ((size_t)grid > partials_cap) return cudaErrorInvalidValue;
    const FastDiv chunks = FastDiv::make((unsigned)cpf);
    if (g.d == 2) {
        if (v4)
            apply_kernel<2, 4><<<grid, kThreads, 0, s>>>(g, pi, chunks, items, fs, cf, dT, v, mean_s, sum_v, Hv, partials, ticket, out, pcg);
        else
            apply_kernel<2, 1><<<grid, kThreads, 0, s>>>(g, pi, chunks, items, fs, cf, dT, v, mean_s, sum_v, Hv, partials, ticket, out, pcg);
    } else {
        if (v4)
            apply_kernel<3, 4><<<grid, kThreads, 0, s>>>(g, pi, chunks, items, fs, cf, dT, v, mean_s, sum_v, Hv, partials, ticket, out, pcg);
        else
            apply_kernel<3, 1><<<grid, kThreads, 0, s>>>(g, pi, chunks, items, fs, cf, dT, v, mean_s, sum_v, Hv, partials, ticket, out, pcg);
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_pcg_init(const Geom& g, const FrameSet& fs, const Coef& cf, const float* grad, const float* dT,
                            float* x, float* r, float* p, float* mean_s, float* sum_v, double* partials,
                            size_t partials_cap, DevScalars* S, PcgArgs a, cudaStream_t s) {
    if ((size_t)((g.N + 31) / 32) * 2 > partials_cap) return cudaErrorInvalidValue;
    return dir_launch<2>(g, fs, cf, dT, p, r, grad, x, mean_s, sum_v, partials, S, a, s);
}

cudaError_t launch_pcg_direction(const Geom& g, const FrameSet& fs, const Coef& cf, const float* dT, const float* r,
                                 float* p, float* mean_s, float* sum_v, DevScalars* S, cudaStream_t s) {
    return dir_launch<1>(g, fs, cf, dT, p, const_cast<float*>(r), nullptr, nullptr, mean_s, sum_v, nullptr, S,
                         PcgArgs{0.f, 0}, s);
}

cudaError_t launch_pcg_update(const Geom& g, const FrameSet& fs, const Coef& cf, const float* dT, float* x, float* r,
                              const float* p, const float* q, double* partials, size_t partials_cap, DevScalars* S,
                              PcgArgs a, cudaStream_t s) {
    const PixIndex pi = make_pix_index(g);
    const bool v4 = vec4_ok(g, {dT, x, r, p, q});
    const int vec = v4 ? 4 : 1;
    const long long cpf = (g.N + (long long)kThreads * vec - 1) / ((long long)kThreads * vec);
    const long long items = cpf * fs.nK * g.d;
    const unsigned grid = (unsigned)(items < kGridStride ? items : kGridStride);
    if ((size_t)grid * 2 > partials_cap) return cudaErrorInvalidValue;
    const FastDiv chunks = FastDiv::make((unsigned)cpf);
    if (g.d == 2) {
        if (v4)
            update_kernel<2, 4><<<grid, kThreads, 0, s>>>(g, pi, chunks, items, fs, cf, dT, x, r, p, q, partials, S, a);
        else
            update_kernel<2, 1><<<grid, kThreads, 0, s>>>(g, pi, chunks, items, fs, cf, dT, x, r, p, q, partials, S, a);
    } else {
        if (v4)
            update_kernel<3, 4><<<grid, kThreads, 0, s>>>(g, pi, chunks, items, fs, cf, dT, x, r, p, q, partials, S, a);
        else
            update_kernel<3, 1><<<grid, kThreads, 0, s>>>(g, pi, chunks, items, fs, cf, dT, x, r, p, q, partials, S, a);
    }
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace stml
