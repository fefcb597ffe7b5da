// Gauss-Newton Hessian product and the PCG solve around it.
//
//   (Hv)_k = hd grad T_k (s_k - sbar) + alpha hd B^T B v_k + alpha_t hd (L_t v)_k
//            + 2 lambda hd / |K|^2 sum_j v_j,          s_k = grad T_k . v_k
//
// The Hessian product needs two per-pixel sums over all frames of K (sbar and
// sum_j v_j).  They are produced by the step that writes v: in the PCG loop the
// search direction p is written by the direction step, which visits all frames
// of a pixel anyway (p = M^-1 r + beta p) and reduces sbar and sum_j p_j over
// the frames in the same pass.  The Hessian product itself is then an
// element-wise stencil stream: it reads v (stencil neighbours come from L1/L2),
// grad T and the sums, writes Hv and reduces <v, Hv>.  Per PCG iteration and
// pixel-frame: Hessian product 12d bytes, update 28d, direction 16d -- every
// array read or written once.
//
// Two ways to run a solve: three stream kernels per iteration whose CG
// coefficients stay in device memory (large levels), or one cooperative
// kernel that runs the whole solve with grid-wide barriers between the steps
// (small levels, where launch latency would dominate).  Both use the same
// per-item code below.  The Jacobi preconditioner is computed from grad T
// where it is needed (`jacobi_inv`, one rounding sequence everywhere).
#include <cooperative_groups.h>

#include "kernels.h"

namespace cg = cooperative_groups;

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

__device__ __forceinline__ float tdiag_of(const FrameSet& fs, int j) {
    return (j + 1 < fs.nK ? __ldg(fs.w_next + j) : 0.f) + (j > 0 ? __ldg(fs.w_next + j - 1) : 0.f);
}

// ------------------------------------------------------------- per-item bodies
// Direction step on one pixel tile (SEG pixels, all frames; CTA = SEG/VEC
// threads per row x FG frame groups).  MODE 0: sums of a given v.  MODE 1:
// p = M^-1 r + beta p and sums of the new p.  MODE 2: r = -g, p = M^-1 r,
// x = 0, the sums, and rz += <r, M^-1 r>, rr += |r|^2.  Writes
// mean_s = sum_k s_k / |K| and sum_v[c]; the frame groups are combined in
// group order.  Every thread of the CTA must call it (it synchronises).
template <int D, int VEC, int MODE, int TPR>
__device__ __forceinline__ void dir_tile(const Geom& g, const PixIndex& pi, const FrameSet& fs, const Coef& cf,
                                         const float* __restrict__ dT, float* __restrict__ v,
                                         float* __restrict__ r, const float* __restrict__ grad,
                                         float* __restrict__ x, float* __restrict__ mean_s,
                                         float* __restrict__ sum_v, float beta, unsigned tile, float* sh,
                                         float& rz, float& rr) {
    constexpr int SEG = TPR * VEC, FG = kThreads / TPR, NR = 1 + D;
    const int lane = threadIdx.x % TPR, fg = threadIdx.x / TPR;
    const unsigned p = tile * SEG + lane * VEC;
    const bool valid = p < (unsigned)g.N;
    const size_t N = (size_t)g.N;
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
    if (valid) {
        for (int j = fg; j < fs.nK; j += FG) {
            const float tdiag = MODE != 0 ? tdiag_of(fs, j) : 0.f;
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
        sh[(fg * NR + 0) * SEG + lane * VEC + e] = as[e];
#pragma unroll
        for (int c = 0; c < D; ++c) sh[(fg * NR + 1 + c) * SEG + lane * VEC + e] = av[c][e];
    }
    __syncthreads();
    const float invK = 1.0f / (float)fs.nK;
    for (int i = threadIdx.x; i < NR * SEG; i += blockDim.x) {
        const int q = i / SEG, k = i - q * SEG;
        const unsigned pp = tile * SEG + k;
        if (pp >= (unsigned)g.N) continue;
        float s = 0.f;
#pragma unroll
        for (int w = 0; w < FG; ++w) s += sh[(w * NR + q) * SEG + k];
        if (q == 0)
            mean_s[pp] = s * invK;
        else
            sum_v[(size_t)(q - 1) * N + pp] = s;
    }
    __syncthreads();
}

// Hessian product on one item: frame j, pixels [ch * kThreads * VEC, +kThreads * VEC).
// Every thread of the warp must call it (warp shuffles).  acc += <v, Hv>.
template <int D, int VEC>
__device__ __forceinline__ void apply_item(const Geom& g, const PixIndex& pi, const FrameSet& fs, const Coef& cf,
                                           const float* __restrict__ dT, const float* __restrict__ v,
                                           const float* __restrict__ mean_s, const float* __restrict__ sum_v,
                                           float* __restrict__ Hv, int j, unsigned ch, float& acc) {
    const size_t N = (size_t)g.N;
    const int lane = threadIdx.x & 31;
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
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
        ds[e] = 0.f;
#pragma unroll
        for (int c = 0; c < D; ++c) sv[c][e] = 0.f;
    }
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
        for (int e = 0; e < VEC; ++e)
            h.a[e] = fmaf(ds[e], dt[c].a[e], fmaf(cf.alpha_hd * cf.inv_h2, lap[e], cf.pen_h * sv[c][e]));
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
        for (int e = 0; e < VEC; ++e) acc = fmaf(vc[c].a[e], h.a[e], acc);
    }
}

// PCG update on one item: plane (frame j, component c), one chunk of pixels.
// x += alpha p, r -= alpha q; rz += <r, M^-1 r>, rr += |r|^2.
template <int D, int VEC>
__device__ __forceinline__ void update_item(const Geom& g, const PixIndex& pi, const FrameSet& fs, const Coef& cf,
                                            const float* __restrict__ dT, float* __restrict__ x,
                                            float* __restrict__ r, const float* __restrict__ p,
                                            const float* __restrict__ q, int plane, unsigned ch, float al,
                                            float& rz, float& rr) {
    const unsigned px = (ch * kThreads + threadIdx.x) * VEC;
    if (px >= (unsigned)g.N) return;
    const float tdiag = tdiag_of(fs, plane / D);
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
        rz = fmaf(rv.a[e], zv, rz);
        rr = fmaf(rv.a[e], rv.a[e], rr);
    }
    xv.store(x + e0);
    rv.store(r + e0);
}

// CG decisions (shared by both solve paths), in float: the step lengths are
// applied in float anyway, and the totals they come from are double-float.
struct CgState {
    float rho, bnorm2, rnorm2, pq, alpha, beta;
    int iter, flag, active;
};

__device__ __forceinline__ float df_val(const dfloat& v) { return v.hi + v.lo; }

__device__ __forceinline__ void cg_after_init(CgState& s, float rz, float rr, int max_cg) {
    s.rho = rz;
    s.bnorm2 = rr;
    s.rnorm2 = rr;
    s.iter = 0;
    if (!(rr > 0.f)) {
        s.flag = CG_ZERO;
        s.active = 0;
    } else if (max_cg <= 0) {
        s.flag = CG_MAXIT;
        s.active = 0;
    } else {
        s.flag = CG_RUNNING;
        s.active = 1;
    }
}

__device__ __forceinline__ void cg_after_apply(CgState& s, float pq) {
    s.pq = pq;
    if (!(pq > 0.f)) {
        s.flag = CG_BREAKDOWN;
        s.active = 0;
    } else {
        s.alpha = s.rho / pq;
    }
}

__device__ __forceinline__ void cg_after_update(CgState& s, float rz, float rr, float tol_cg, int max_cg) {
    s.iter += 1;
    s.rnorm2 = rr;
    if (sqrtf(rr) <= tol_cg * sqrtf(s.bnorm2)) {
        s.flag = CG_CONVERGED;
        s.active = 0;
    } else if (s.iter >= max_cg) {
        s.flag = CG_MAXIT;
        s.active = 0;
    } else {
        s.beta = rz / s.rho;
        s.rho = rz;
    }
}

__device__ __forceinline__ CgState cg_load(const DevScalars* S) {
    CgState s;
    s.rho = S->rho;
    s.bnorm2 = S->bnorm2;
    s.rnorm2 = S->rnorm2;
    s.pq = S->pq;
    s.alpha = S->alpha;
    s.beta = S->beta;
    s.iter = S->cg_iter;
    s.flag = S->cg_flag;
    s.active = S->cg_active;
    return s;
}

__device__ __forceinline__ void cg_store(DevScalars* S, const CgState& s) {
    S->rho = s.rho;
    S->bnorm2 = s.bnorm2;
    S->rnorm2 = s.rnorm2;
    S->pq = s.pq;
    S->alpha = s.alpha;
    S->beta = s.beta;
    S->cg_iter = s.iter;
    S->cg_flag = s.flag;
    S->cg_active = s.active;
}

}  // namespace

// ----------------------------------------------------------------- stream kernels
template <int D, int VEC, int MODE, int TPR>
__global__ void __launch_bounds__(kThreads)
dir_kernel(Geom g, PixIndex pi, FrameSet fs, Coef cf, const float* __restrict__ dT, float* __restrict__ v,
           float* __restrict__ r, const float* __restrict__ grad, float* __restrict__ x,
           float* __restrict__ mean_s, float* __restrict__ sum_v, double* __restrict__ partials,
           DevScalars* S, PcgArgs a) {
    if (MODE == 1 && !S->cg_active) return;
    __shared__ float sh[(kThreads / TPR) * (1 + D) * TPR * VEC];
    const float beta = MODE == 1 ? S->beta : 0.f;
    float rz = 0.f, rr = 0.f;
    dir_tile<D, VEC, MODE, TPR>(g, pi, fs, cf, dT, v, r, grad, x, mean_s, sum_v, beta, blockIdx.x, sh, rz, rr);
    if constexpr (MODE == 2) {
        float acc[2] = {rz, rr};
        double tot[2];
        if (grid_reduce<2>(acc, partials, &S->ticket[2], tot) && threadIdx.x == 0) {
            CgState st = cg_load(S);
            cg_after_init(st, (float)tot[0], (float)tot[1], a.max_cg);
            cg_store(S, st);
        }
    }
}

template <int D, int VEC>
__global__ void __launch_bounds__(kThreads)
apply_kernel(Geom g, PixIndex pi, FastDiv chunks, long long items, FrameSet fs, Coef cf,
             const float* __restrict__ dT, const float* __restrict__ v, const float* __restrict__ mean_s,
             const float* __restrict__ sum_v, float* __restrict__ Hv, double* __restrict__ partials,
             unsigned int* ticket, double* out, DevScalars* pcg) {
    if (pcg && !pcg->cg_active) return;
    float acc[1] = {0.f};
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const int j = (int)chunks.div((unsigned)it);
        apply_item<D, VEC>(g, pi, fs, cf, dT, v, mean_s, sum_v, Hv, j, (unsigned)it - (unsigned)j * chunks.d, acc[0]);
    }
    if (grid_reduce<1>(acc, partials, ticket, out) && threadIdx.x == 0 && pcg) {
        CgState st = cg_load(pcg);
        cg_after_apply(st, (float)out[0]);
        cg_store(pcg, st);
    }
}

template <int D, int VEC>
__global__ void __launch_bounds__(kThreads)
update_kernel(Geom g, PixIndex pi, FastDiv chunks, long long items, FrameSet fs, Coef cf,
              const float* __restrict__ dT, float* __restrict__ x, float* __restrict__ r,
              const float* __restrict__ p, const float* __restrict__ q, double* __restrict__ partials,
              DevScalars* S, PcgArgs a) {
    if (!S->cg_active) return;
    const float al = S->alpha;
    float acc[2] = {0.f, 0.f};
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const int plane = (int)chunks.div((unsigned)it);
        update_item<D, VEC>(g, pi, fs, cf, dT, x, r, p, q, plane, (unsigned)it - (unsigned)plane * chunks.d, al,
                            acc[0], acc[1]);
    }
    double tot[2];
    if (grid_reduce<2>(acc, partials, &S->ticket[2], tot) && threadIdx.x == 0) {
        CgState st = cg_load(S);
        cg_after_update(st, (float)tot[0], (float)tot[1], a.tol_cg, a.max_cg);
        cg_store(S, st);
    }
}

// ----------------------------------------------------------------- cooperative solve
// The whole PCG solve in one cooperative launch: init, then per iteration the
// Hessian product, the update and the direction step, separated by three
// grid-wide barriers.  Every CTA evaluates the same CG decisions from the same
// fixed-order totals, so all CTAs leave the loop together.
template <int D, int VEC, int TPR>
__global__ void __launch_bounds__(kThreads)
pcg_coop_kernel(Geom g, PixIndex pi, FastDiv chunks, long long aitems, long long uitems, unsigned tiles,
                FrameSet fs, Coef cf, const float* __restrict__ grad, const float* __restrict__ dT,
                float* __restrict__ x, float* __restrict__ r, float* __restrict__ p, float* __restrict__ q,
                float* __restrict__ mean_s, float* __restrict__ sum_v, double* __restrict__ partials,
                DevScalars* S, PcgArgs a) {
    cg::grid_group grid = cg::this_grid();
    __shared__ float sh[(kThreads / TPR) * (1 + D) * TPR * VEC];
    // two partial-sum buffers: A for <p, Hp>, B for the update's sums (and the
    // start); a buffer is rewritten only after a barrier that follows every
    // CTA's read of it, so three barriers per iteration suffice
    float2* partA = reinterpret_cast<float2*>(partials);
    float2* partB = partA + 2 * (size_t)gridDim.x;
    CgState st{0, 0, 0, 0, 0, 0, 0, 0, 0};
    {   // r = -g, p = M^-1 r, x = 0, frame sums of p
        float rz = 0.f, rr = 0.f;
        for (unsigned t = blockIdx.x; t < tiles; t += gridDim.x)
            dir_tile<D, VEC, 2, TPR>(g, pi, fs, cf, dT, p, r, grad, x, mean_s, sum_v, 0.f, t, sh, rz, rr);
        const float v2[2] = {rz, rr};
        cta_partials<2>(v2, partB, blockIdx.x);
        grid.sync();
        dfloat tot[2];
        cta_total<2>(partB, gridDim.x, tot);
        cg_after_init(st, df_val(tot[0]), df_val(tot[1]), a.max_cg);
    }
    while (st.active) {
        float pq = 0.f;
        for (long long it = blockIdx.x; it < aitems; it += gridDim.x) {
            const int j = (int)chunks.div((unsigned)it);
            apply_item<D, VEC>(g, pi, fs, cf, dT, p, mean_s, sum_v, q, j, (unsigned)it - (unsigned)j * chunks.d, pq);
        }
        {
            const float v1[1] = {pq};
            cta_partials<1>(v1, partA, blockIdx.x);
        }
        grid.sync();   // q and the <p, Hp> partials are complete
        {
            dfloat tot[1];
            cta_total<1>(partA, gridDim.x, tot);
            cg_after_apply(st, df_val(tot[0]));
        }
        if (!st.active) break;
        const float al = st.alpha;
        float rz = 0.f, rr = 0.f;
        for (long long it = blockIdx.x; it < uitems; it += gridDim.x) {
            const int plane = (int)chunks.div((unsigned)it);
            update_item<D, VEC>(g, pi, fs, cf, dT, x, r, p, q, plane, (unsigned)it - (unsigned)plane * chunks.d, al,
                                rz, rr);
        }
        {
            const float v2[2] = {rz, rr};
            cta_partials<2>(v2, partB, blockIdx.x);
        }
        grid.sync();   // r and the update partials are complete
        {
            dfloat tot[2];
            cta_total<2>(partB, gridDim.x, tot);
            cg_after_update(st, df_val(tot[0]), df_val(tot[1]), a.tol_cg, a.max_cg);
        }
        if (!st.active) break;
        const float be = st.beta;
        float d0 = 0.f, d1 = 0.f;
        for (unsigned t = blockIdx.x; t < tiles; t += gridDim.x)
            dir_tile<D, VEC, 1, TPR>(g, pi, fs, cf, dT, p, r, nullptr, nullptr, mean_s, sum_v, be, t, sh, d0, d1);
        grid.sync();   // p and its frame sums are complete
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) cg_store(S, st);
}

// ----------------------------------------------------------------- launchers
PixIndex make_pix_index(const Geom& g) {
    PixIndex pi;
    pi.nx = FastDiv::make((unsigned)g.nx);
    pi.ny = FastDiv::make((unsigned)g.ny);
    return pi;
}

namespace {

constexpr int kGridStride = 152 * 8;   // CTAs of the grid-stride launches (8 per SM of a GB300)

bool vec4_ok(const Geom& g, std::initializer_list<const void*> ptrs) {
    if (g.nx % 4) return false;
    for (const void* q : ptrs)
        if (q && ((uintptr_t)q & 15u)) return false;
    return true;
}

// Wide pixel tiles on large levels, narrow ones (more CTAs, more frame groups) on small levels.
bool narrow_tiles(const Geom& g, bool v4) { return g.N < 4LL * 152 * (v4 ? 64 : 32); }

}  // namespace

template <int MODE>
static cudaError_t dir_launch(const Geom& g, const FrameSet& fs, const Coef& cf, const float* dT, float* v, float* r,
                              const float* grad, float* x, float* mean_s, float* sum_v, double* partials,
                              DevScalars* S, PcgArgs a, cudaStream_t s) {
    const PixIndex pi = make_pix_index(g);
    const bool v4 = vec4_ok(g, {dT, v, r, grad, x});
    const bool narrow = narrow_tiles(g, v4);
    const int seg = v4 ? (narrow ? 16 : 64) : (narrow ? 8 : 32);
    const unsigned blocks = (unsigned)((g.N + seg - 1) / seg);
#define STML_DIR(D_, V_, T_) \
    dir_kernel<D_, V_, MODE, T_><<<blocks, kThreads, 0, s>>>(g, pi, fs, cf, dT, v, r, grad, x, mean_s, sum_v, partials, S, a)
    if (g.d == 2) {
        if (v4) { if (narrow) STML_DIR(2, 4, 4); else STML_DIR(2, 4, 16); }
        else { if (narrow) STML_DIR(2, 1, 8); else STML_DIR(2, 1, 32); }
    } else {
        if (v4) { if (narrow) STML_DIR(3, 4, 4); else STML_DIR(3, 4, 16); }
        else { if (narrow) STML_DIR(3, 1, 8); else STML_DIR(3, 1, 32); }
    }
#undef STML_DIR
    count_launches(1);
    return cudaGetLastError();
}

size_t gn_partials(const Geom& g, int nK) {
    const size_t dir = (size_t)((g.N + 7) / 8) * 2;
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
    if ((size_t)((g.N + 7) / 8) * 2 > partials_cap) return cudaErrorInvalidValue;
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

namespace {

template <int D, int VEC, int TPR>
cudaError_t coop_go(const Geom& g, const FrameSet& fs, const Coef& cf, const float* grad, const float* dT, float* x,
                    float* r, float* p, float* q, float* mean_s, float* sum_v, double* partials, size_t partials_cap,
                    DevScalars* S, PcgArgs a, cudaStream_t s) {
    const void* kern = (const void*)pcg_coop_kernel<D, VEC, TPR>;
    int dev = 0, sms = 1, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    PixIndex pi = make_pix_index(g);
    long long cpf = (g.N + (long long)kThreads * VEC - 1) / ((long long)kThreads * VEC);
    long long aitems = cpf * fs.nK, uitems = cpf * fs.nK * D;
    unsigned tiles = (unsigned)((g.N + TPR * VEC - 1) / (TPR * VEC));
    const long long want = uitems > (long long)tiles ? uitems : (long long)tiles;
    // one CTA per SM at most: the solve is small and grid barriers get dearer with more CTAs
    const long long cap = (long long)sms;
    unsigned blocks = (unsigned)(want < cap ? want : cap);
    if (blocks < 1) blocks = 1;
    if ((size_t)blocks * 4 > partials_cap) return cudaErrorInvalidValue;
    FastDiv chunks = FastDiv::make((unsigned)cpf);
    Geom gg = g;
    FrameSet ff = fs;
    Coef cc = cf;
    PcgArgs aa = a;
    void* args[] = {&gg, &pi, &chunks, &aitems, &uitems, &tiles, &ff, &cc, (void*)&grad, (void*)&dT, &x, &r, &p,
                    &q, &mean_s, &sum_v, &partials, &S, &aa};
    e = cudaLaunchCooperativeKernel(kern, dim3(blocks), dim3(kThreads), args, 0, s);
    count_launches(1);
    return e;
}

}  // namespace

bool pcg_coop_preferred(const Geom& g, int nK) { return (long long)g.N * nK <= (1LL << 20); }

cudaError_t launch_pcg_coop(const Geom& g, const FrameSet& fs, const Coef& cf, const float* grad, const float* dT,
                            float* x, float* r, float* p, float* q, float* mean_s, float* sum_v, double* partials,
                            size_t partials_cap, DevScalars* S, PcgArgs a, cudaStream_t s) {
    const bool v4 = vec4_ok(g, {grad, dT, x, r, p, q, mean_s, sum_v});
    if (g.d == 2)
        return v4 ? coop_go<2, 4, 4>(g, fs, cf, grad, dT, x, r, p, q, mean_s, sum_v, partials, partials_cap, S, a, s)
                  : coop_go<2, 1, 8>(g, fs, cf, grad, dT, x, r, p, q, mean_s, sum_v, partials, partials_cap, S, a, s);
    return v4 ? coop_go<3, 4, 4>(g, fs, cf, grad, dT, x, r, p, q, mean_s, sum_v, partials, partials_cap, S, a, s)
              : coop_go<3, 1, 8>(g, fs, cf, grad, dT, x, r, p, q, mean_s, sum_v, partials, partials_cap, S, a, s);
}

}  // namespace stml
