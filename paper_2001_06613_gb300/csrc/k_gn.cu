// Gauss-Newton Hessian product and the PCG solve around it.
//
//   (Hv)_k = hd grad T_k (s_k - sbar) + alpha hd B^T B v_k + alpha_t hd (L_t v)_k
//            + 2 lambda hd / |K|^2 sum_j v_j,          s_k = grad T_k . v_k
//
// The Hessian product needs two per-pixel sums over all frames of K (sbar and
// sum_j v_j) before any (Hv)_k can be written, so it is two passes: the sums,
// then an element-wise stencil stream that reads v (stencil neighbours come
// from L1/L2), grad T and the sums, writes Hv and reduces <v, Hv>.
//
// Jacobi PCG.  Large levels stream three passes per iteration: the Hessian
// product of p (its frame sums come from the pass that wrote p), the update
// x += alpha p, r -= alpha q with rho = <r, M^-1 r>, and the pixel-tiled
// direction step p = M^-1 r + beta p, which visits all frames of a pixel and
// reduces the frame sums of the new p in the same pass.  Per iteration and
// pixel-frame: 12d + 28d + 16d bytes.  The cooperative solve of small levels
// is latency-bound and uses two phases (two grid barriers) per iteration:
// the pixel-tiled update also forms z = M^-1 r and its frame sums, and the
// Hessian-product phase forms p = z + beta p_old on the fly (sums of p = sums
// of z + beta sums of p_old), with p and its sums double-buffered.
//
// Two ways to run a solve: three stream kernels per iteration whose CG
// coefficients stay in device memory (large levels), or one cooperative
// kernel that runs the whole solve with two grid-wide barriers per iteration
// (small levels, where launch latency would dominate).  Both use the same
// per-item code below.  The Jacobi preconditioner is computed from grad T
// where it is needed (`jacobi_inv`, one rounding sequence everywhere).
#include <cooperative_groups.h>

#include <type_traits>

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
    template <typename T>
    __device__ __forceinline__ void load_t(const T* p) { ld4f(p, a); }   // stored type -> float
};
template <>
struct V<1> {
    float a[1];
    __device__ __forceinline__ void load(const float* p) { a[0] = __ldg(p); }
    __device__ __forceinline__ void load_rw(const float* p) { a[0] = *p; }
    __device__ __forceinline__ void store(float* p) const { *p = a[0]; }
    __device__ __forceinline__ void zero() { a[0] = 0.f; }
    template <typename T>
    __device__ __forceinline__ void load_t(const T* p) { a[0] = ldf(p); }
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
enum TileMode { TILE_SUMS = 0, TILE_DIR = 1, TILE_INIT = 2, TILE_UPDATE = 3 };

// Pixel-tiled pass over one tile (SEG pixels, all frames; CTA = SEG/VEC
// threads per row x FG frame groups) that ends with the per-pixel frame sums
// mean_s = sum_k grad T_k . w_k / |K| and sum_v[c] = sum_k w_{k,c} of a field w.
//   TILE_SUMS:   w = v (given).
//   TILE_DIR:    w = p = M^-1 r + beta p, in place in v.
//   TILE_INIT:   r = -g, w = z = M^-1 r (written to v), x = 0;
//                rz += <r, z>, rr += |r|^2.
//   TILE_UPDATE: x += al p, r -= al q, w = z = M^-1 r (written to v);
//                rz += <r, z>, rr += |r|^2.
// The frame groups are combined in group order.  Every thread of the CTA
// must call it (it synchronises).
template <int D, int VEC, int MODE, int TPR, typename TD>
__device__ __forceinline__ void tile_pass(const Geom& g, const PixIndex& pi, const FrameSet& fs, const Coef& cf,
                                          const TD* __restrict__ dT, float* __restrict__ v,
                                          float* __restrict__ r, const float* __restrict__ grad,
                                          float* __restrict__ x, const float* __restrict__ p,
                                          const float* __restrict__ q, float al, float beta,
                                          float* __restrict__ mean_s,
                                          float* __restrict__ sum_v, unsigned tile, float* sh, float& rz,
                                          float& rr) {
    constexpr int SEG = TPR * VEC, FG = kThreads / TPR, NR = 1 + D;
    const int lane = threadIdx.x % TPR, fg = threadIdx.x / TPR;
    const unsigned px = tile * SEG + lane * VEC;
    const bool valid = px < (unsigned)g.N;
    const size_t N = (size_t)g.N;
    int nnb[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) nnb[e] = 0;
    if (MODE != TILE_SUMS && valid) {
        int xx, yy, zz;
        pix_pos(pi, px, xx, yy, zz);
#pragma unroll
        for (int e = 0; e < VEC; ++e) nnb[e] = neighbour_count(g, xx + e, yy, zz);
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
            const float tdiag = MODE != TILE_SUMS ? tdiag_of(fs, j) : 0.f;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const size_t e0 = ((size_t)j * D + c) * N + px;
                V<VEC> dt, wv;
                dt.load_t(dT + e0);
                if constexpr (MODE == TILE_SUMS) {
                    wv.load(v + e0);
                } else if constexpr (MODE == TILE_DIR) {
                    V<VEC> rv;
                    rv.load(r + e0);
                    wv.load_rw(v + e0);
#pragma unroll
                    for (int e = 0; e < VEC; ++e)
                        wv.a[e] = fmaf(beta, wv.a[e], jacobi_inv(dt.a[e], nnb[e], tdiag, cf) * rv.a[e]);
                    wv.store(v + e0);
                } else {
                    V<VEC> rv;
                    if constexpr (MODE == TILE_INIT) {
                        V<VEC> gv, zero;
                        gv.load(grad + e0);
                        zero.zero();
#pragma unroll
                        for (int e = 0; e < VEC; ++e) rv.a[e] = -gv.a[e];
                        zero.store(x + e0);
                    } else {
                        V<VEC> pv, qv, xv;
                        pv.load(p + e0);
                        qv.load(q + e0);
                        xv.load_rw(x + e0);
                        rv.load_rw(r + e0);
#pragma unroll
                        for (int e = 0; e < VEC; ++e) {
                            xv.a[e] = fmaf(al, pv.a[e], xv.a[e]);
                            rv.a[e] = fmaf(-al, qv.a[e], rv.a[e]);
                        }
                        xv.store(x + e0);
                    }
#pragma unroll
                    for (int e = 0; e < VEC; ++e) {
                        wv.a[e] = jacobi_inv(dt.a[e], nnb[e], tdiag, cf) * rv.a[e];
                        rz = fmaf(rv.a[e], wv.a[e], rz);
                        rr = fmaf(rv.a[e], rv.a[e], rr);
                    }
                    rv.store(r + e0);
                    wv.store(v + e0);
                }
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    as[e] = fmaf(dt.a[e], wv.a[e], as[e]);
                    av[c][e] += wv.a[e];
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
        const int qq = i / SEG, k = i - qq * SEG;
        const unsigned pp = tile * SEG + k;
        if (pp >= (unsigned)g.N) continue;
        float s = 0.f;
#pragma unroll
        for (int w = 0; w < FG; ++w) s += sh[(w * NR + qq) * SEG + k];
        if (qq == 0)
            mean_s[pp] = s * invK;
        else
            sum_v[(size_t)(qq - 1) * N + pp] = s;
    }
    __syncthreads();
}

// The field the Hessian product is applied to, and its per-pixel frame sums.
// Plain product: w = v.  PCG (FUSED): w = p = z + beta p_old (p_old absent on
// the first iteration, beta = 0), written to pout by the item that computes
// it; its sums are the sums of z plus beta times those of p_old, and the
// items of frame 0 store them for the next iteration.
struct DirSrc {
    const float* z;       // v, or z of the PCG
    const float* pold;    // p_old, or nullptr
    float beta;
    float* pout;          // the new p (PCG), or nullptr
    const float* ms_z;    // mean_s and sum_v of v (or of z)
    const float* sv_z;
    const float* ms_p;    // ... of p_old (PCG with p_old)
    const float* sv_p;
    float* ms_out;        // ... of the new p (PCG)
    float* sv_out;
};

// Hessian product on one item: frame j, pixels [ch * kThreads * VEC, +kThreads * VEC).
// Every thread of the warp must call it (warp shuffles).  acc += <w, Hw>.
template <int D, int VEC, bool FUSED, typename TD>
__device__ __forceinline__ void apply_item(const Geom& g, const PixIndex& pi, const FrameSet& fs, const Coef& cf,
                                           const TD* __restrict__ dT, const DirSrc& src,
                                           float* __restrict__ Hv, int j, unsigned ch, float& acc) {
    const size_t N = (size_t)g.N;
    const int lane = threadIdx.x & 31;
    const unsigned p = (ch * kThreads + threadIdx.x) * VEC;
    const bool valid = p < (unsigned)g.N;
    const bool with_p = FUSED && src.pold != nullptr;
    const float w_next = (cf.alphat_hd != 0.f && j + 1 < fs.nK) ? __ldg(fs.w_next + j) : 0.f;
    const float w_prev = (cf.alphat_hd != 0.f && j > 0) ? __ldg(fs.w_next + j - 1) : 0.f;
    // w at an offset (a run of VEC values / one value)
    auto ldw = [&](size_t off, V<VEC>& o) {
        o.load(src.z + off);
        if (with_p) {
            V<VEC> t;
            t.load(src.pold + off);
#pragma unroll
            for (int e = 0; e < VEC; ++e) o.a[e] = fmaf(src.beta, t.a[e], o.a[e]);
        }
    };
    auto ldw1 = [&](size_t off) {
        const float w = __ldg(src.z + off);
        return with_p ? fmaf(src.beta, __ldg(src.pold + off), w) : w;
    };
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
            ldw(e0, vc[c]);
            dt[c].load_t(dT + e0);
            if (FUSED) vc[c].store(src.pout + e0);
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
        ms.load(src.ms_z + p);
        if (with_p) {
            V<VEC> t;
            t.load(src.ms_p + p);
#pragma unroll
            for (int e = 0; e < VEC; ++e) ms.a[e] = fmaf(src.beta, t.a[e], ms.a[e]);
        }
        if (FUSED && j == 0) ms.store(src.ms_out + p);
#pragma unroll
        for (int e = 0; e < VEC; ++e) ds[e] = cf.hd * (s[e] - ms.a[e]);
#pragma unroll
        for (int c = 0; c < D; ++c) {
            V<VEC> t;
            t.load(src.sv_z + (size_t)c * N + p);
            if (with_p) {
                V<VEC> u;
                u.load(src.sv_p + (size_t)c * N + p);
#pragma unroll
                for (int e = 0; e < VEC; ++e) t.a[e] = fmaf(src.beta, u.a[e], t.a[e]);
            }
            if (FUSED && j == 0) t.store(src.sv_out + (size_t)c * N + p);
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
        if (x > 0) left = (lane > 0) ? up_l : ldw1(e0 - 1);
        if (x + VEC < g.nx) right = (lane < 31) ? dn_r : ldw1(e0 + VEC);
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
            ldw(e0 - g.nx, nb);
#pragma unroll
            for (int e = 0; e < VEC; ++e) lap[e] += vc[c].a[e] - nb.a[e];
        }
        if (y < g.ny - 1) {
            ldw(e0 + g.nx, nb);
#pragma unroll
            for (int e = 0; e < VEC; ++e) lap[e] += vc[c].a[e] - nb.a[e];
        }
        if constexpr (D == 3) {
            const size_t sz = (size_t)g.nx * g.ny;
            if (z > 0) {
                ldw(e0 - sz, nb);
#pragma unroll
                for (int e = 0; e < VEC; ++e) lap[e] += vc[c].a[e] - nb.a[e];
            }
            if (z < g.nz - 1) {
                ldw(e0 + sz, nb);
#pragma unroll
                for (int e = 0; e < VEC; ++e) lap[e] += vc[c].a[e] - nb.a[e];
            }
        }
        V<VEC> h;
#pragma unroll
        for (int e = 0; e < VEC; ++e)
            h.a[e] = fmaf(ds[e], dt[c].a[e], fmaf(cf.alpha_hd * cf.inv_h2, lap[e], cf.pen_h * sv[c][e]));
        if (w_next != 0.f) {
            ldw(e0 + (size_t)D * N, nb);
#pragma unroll
            for (int e = 0; e < VEC; ++e) h.a[e] = fmaf(cf.alphat_hd * w_next, vc[c].a[e] - nb.a[e], h.a[e]);
        }
        if (w_prev != 0.f) {
            ldw(e0 - (size_t)D * N, nb);
#pragma unroll
            for (int e = 0; e < VEC; ++e) h.a[e] = fmaf(cf.alphat_hd * w_prev, vc[c].a[e] - nb.a[e], h.a[e]);
        }
        h.store(Hv + e0);
#pragma unroll
        for (int e = 0; e < VEC; ++e) acc = fmaf(vc[c].a[e], h.a[e], acc);
    }
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
    s.beta = 0.f;
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
// Pixel-tiled pass (frame sums, PCG start, PCG direction); the PCG start ends
// with the CG decisions of its step in the last CTA.
template <int D, int VEC, int MODE, int TPR, typename TD>
__global__ void __launch_bounds__(kThreads)
tile_kernel(Geom g, PixIndex pi, FrameSet fs, Coef cf, const TD* __restrict__ dT, float* __restrict__ v,
            float* __restrict__ r, const float* __restrict__ grad, float* __restrict__ x,
            float* __restrict__ mean_s, float* __restrict__ sum_v, double* __restrict__ partials, DevScalars* S,
            PcgArgs a, const int* gate) {
    static_assert(MODE != TILE_UPDATE, "the update runs as a grid-stride stream");
    if (MODE == TILE_DIR && !S->cg_active) return;
    if (gate && !*gate) return;
    __shared__ float sh[(kThreads / TPR) * (1 + D) * TPR * VEC];
    const float beta = MODE == TILE_DIR ? S->beta : 0.f;
    float rz = 0.f, rr = 0.f;
    tile_pass<D, VEC, MODE, TPR, TD>(g, pi, fs, cf, dT, v, r, grad, x, nullptr, nullptr, 0.f, beta, mean_s, sum_v,
                                 blockIdx.x, sh, rz, rr);
    if constexpr (MODE == TILE_INIT) {
        float acc[2] = {rz, rr};
        double tot[2];
        if (grid_reduce<2>(acc, partials, &S->ticket[2], tot) && threadIdx.x == 0) {
            CgState st = cg_load(S);
            cg_after_init(st, (float)tot[0], (float)tot[1], a.max_cg);
            cg_store(S, st);
        }
    }
}

// PCG update on one item: plane (frame j, component c), one chunk of pixels.
// x += alpha p, r -= alpha q; rz += <r, M^-1 r>, rr += |r|^2.
template <int D, int VEC, typename TD>
__device__ __forceinline__ void update_item(const Geom& g, const PixIndex& pi, const FrameSet& fs, const Coef& cf,
                                            const TD* __restrict__ dT, float* __restrict__ x,
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
    dt.load_t(dT + e0);
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

template <int D, int VEC, typename TD>
__global__ void __launch_bounds__(kThreads)
update_kernel(Geom g, PixIndex pi, FastDiv chunks, long long items, FrameSet fs, Coef cf,
              const TD* __restrict__ dT, float* __restrict__ x, float* __restrict__ r,
              const float* __restrict__ p, const float* __restrict__ q, double* __restrict__ partials,
              DevScalars* S, PcgArgs a) {
    if (!S->cg_active) return;
    const float al = S->alpha;
    float acc[2] = {0.f, 0.f};
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const int plane = (int)chunks.div((unsigned)it);
        update_item<D, VEC, TD>(g, pi, fs, cf, dT, x, r, p, q, plane, (unsigned)it - (unsigned)plane * chunks.d, al,
                            acc[0], acc[1]);
    }
    double tot[2];
    if (grid_reduce<2>(acc, partials, &S->ticket[2], tot) && threadIdx.x == 0) {
        CgState st = cg_load(S);
        cg_after_update(st, (float)tot[0], (float)tot[1], a.tol_cg, a.max_cg);
        cg_store(S, st);
    }
}

// Hessian product stream (grid-stride over (frame, chunk) items) of
// v = src.z with its frame sums src.ms_z / src.sv_z.  With pcg != nullptr the
// launch is a PCG step: it does nothing once cg_active is 0 and the last CTA
// sets alpha = rho / <p, Hp> (or flags a breakdown).
// CTAs per SM the Hessian-product kernel is compiled for (a register cap):
// 3 for the 3-D float4 form, where 80 registers instead of 84 let a third
// CTA in; otherwise the count its register use gives anyway.
template <int D, int VEC>
constexpr int apply_min_ctas() { return VEC == 4 ? (D == 3 ? 3 : 4) : (D == 3 ? 5 : 6); }

template <int D, int VEC, typename TD>
__global__ void __launch_bounds__(kThreads, (apply_min_ctas<D, VEC>()))
apply_kernel(Geom g, PixIndex pi, FastDiv chunks, long long items, FrameSet fs, Coef cf,
             const TD* __restrict__ dT, DirSrc src, float* __restrict__ Hv, double* __restrict__ partials,
             unsigned int* ticket, double* out, DevScalars* pcg) {
    if (pcg && !pcg->cg_active) return;
    float acc[1] = {0.f};
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const int j = (int)chunks.div((unsigned)it);
        apply_item<D, VEC, false, TD>(g, pi, fs, cf, dT, src, Hv, j, (unsigned)it - (unsigned)j * chunks.d, acc[0]);
    }
    if (grid_reduce<1>(acc, partials, ticket, out) && threadIdx.x == 0 && pcg) {
        CgState st = cg_load(pcg);
        cg_after_apply(st, (float)out[0]);
        cg_store(pcg, st);
    }
}

// ----------------------------------------------------------------- cooperative solve
// The whole PCG solve in one cooperative launch: the start, then per
// iteration the fused direction + Hessian product and the update, separated
// by two grid-wide barriers.  Every CTA evaluates the same CG decisions from
// the same fixed-order totals, so all CTAs leave the loop together.
template <int D, int VEC, int TPR, typename TD>
__global__ void __launch_bounds__(kThreads)
pcg_coop_kernel(Geom g, PixIndex pi, FastDiv chunks, long long aitems, unsigned tiles, FrameSet fs, Coef cf,
                const float* __restrict__ grad, const TD* __restrict__ dT, PcgBufs b,
                double* __restrict__ partials, DevScalars* S, PcgArgs a, const int* gate) {
    if (gate && !*gate) return;   // every CTA leaves before the first barrier
    cg::grid_group grid = cg::this_grid();
    __shared__ float sh[(kThreads / TPR) * (1 + D) * TPR * VEC];
    // two partial-sum buffers: A for <p, Hp>, B for the start and the
    // update; a buffer is rewritten only after a barrier that follows every
    // CTA's read of it
    float2* partA = reinterpret_cast<float2*>(partials);
    float2* partB = partA + 2 * (size_t)gridDim.x;
    CgState st{0, 0, 0, 0, 0, 0, 0, 0, 0};
    {   // r = -g, z = M^-1 r, x = 0, frame sums of z
        float rz = 0.f, rr = 0.f;
        for (unsigned t = blockIdx.x; t < tiles; t += gridDim.x)
            tile_pass<D, VEC, TILE_INIT, TPR, TD>(g, pi, fs, cf, dT, b.z, b.r, grad, b.x, nullptr, nullptr, 0.f, 0.f,
                                              b.ms_z, b.sv_z, t, sh, rz, rr);
        const float v2[2] = {rz, rr};
        cta_partials<2>(v2, partB, blockIdx.x);
        grid.sync();
        dfloat tot[2];
        cta_total<2>(partB, gridDim.x, tot);
        cg_after_init(st, df_val(tot[0]), df_val(tot[1]), a.max_cg);
    }
    for (int k = 0; st.active; ++k) {
        const int cur = k & 1, old = cur ^ 1;
        const DirSrc src{b.z, k > 0 ? b.p[old] : nullptr, st.beta, b.p[cur], b.ms_z, b.sv_z,
                         b.ms_p[old], b.sv_p[old], b.ms_p[cur], b.sv_p[cur]};
        float pq = 0.f;
        for (long long it = blockIdx.x; it < aitems; it += gridDim.x) {
            const int j = (int)chunks.div((unsigned)it);
            apply_item<D, VEC, true, TD>(g, pi, fs, cf, dT, src, b.q, j, (unsigned)it - (unsigned)j * chunks.d, pq);
        }
        {
            const float v1[1] = {pq};
            cta_partials<1>(v1, partA, blockIdx.x);
        }
        grid.sync();   // p, q and the <p, Hp> partials are complete
        {
            dfloat tot[1];
            cta_total<1>(partA, gridDim.x, tot);
            cg_after_apply(st, df_val(tot[0]));
        }
        if (!st.active) break;
        float rz = 0.f, rr = 0.f;
        for (unsigned t = blockIdx.x; t < tiles; t += gridDim.x)
            tile_pass<D, VEC, TILE_UPDATE, TPR, TD>(g, pi, fs, cf, dT, b.z, b.r, nullptr, b.x, b.p[cur], b.q, st.alpha,
                                                0.f, b.ms_z, b.sv_z, t, sh, rz, rr);
        {
            const float v2[2] = {rz, rr};
            cta_partials<2>(v2, partB, blockIdx.x);
        }
        grid.sync();   // x, r, z, the sums of z and the update partials are complete
        {
            dfloat tot[2];
            cta_total<2>(partB, gridDim.x, tot);
            cg_after_update(st, df_val(tot[0]), df_val(tot[1]), a.tol_cg, a.max_cg);
        }
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

constexpr int kGridStride = 152 * 8;   // most CTAs of a grid-stride launch (8 of 256 threads per SM of a GB300)

bool vec4_ok(const Geom& g, std::initializer_list<const void*> ptrs) {
    if (g.nx % 4) return false;
    for (const void* q : ptrs)
        if (q && ((uintptr_t)q & 15u)) return false;
    return true;
}

// Wide pixel tiles on large levels, narrow ones (more CTAs, more frame groups) on small levels.
bool narrow_tiles(const Geom& g, bool v4) { return g.N < 4LL * 152 * (v4 ? 64 : 32); }

template <int MODE>
cudaError_t tile_launch(const Geom& g, const FrameSet& fs, const Coef& cf, const Stored& dT, float* v, float* r,
                        const float* grad, float* x, float* mean_s, float* sum_v, double* partials, DevScalars* S,
                        PcgArgs a, cudaStream_t s, const int* gate = nullptr) {
    const PixIndex pi = make_pix_index(g);
    const bool v4 = vec4_ok(g, {dT.p, v, r, grad, x});
    const bool narrow = narrow_tiles(g, v4);
    const int seg = v4 ? (narrow ? 16 : 64) : (narrow ? 8 : 32);
    const unsigned blocks = (unsigned)((g.N + seg - 1) / seg);
#define STML_TILE(D_, V_, T_)                                                                                      \
    tile_kernel<D_, V_, MODE, T_, TD><<<blocks, kThreads, 0, s>>>(g, pi, fs, cf, Td, v, r, grad, x, mean_s, sum_v, \
                                                                  partials, S, a, gate)
    with_store_type(dT.type, [&](auto tag) {
        using TD = decltype(tag);
        const TD* Td = static_cast<const TD*>(dT.p);
        if constexpr (MODE == TILE_SUMS && !std::is_same<TD, float>::value) return 0;   // float grad T only
        if (g.d == 2) {
            if (v4) { if (narrow) STML_TILE(2, 4, 4); else STML_TILE(2, 4, 16); }
            else { if (narrow) STML_TILE(2, 1, 8); else STML_TILE(2, 1, 32); }
        } else {
            if (v4) { if (narrow) STML_TILE(3, 4, 4); else STML_TILE(3, 4, 16); }
            else { if (narrow) STML_TILE(3, 1, 8); else STML_TILE(3, 1, 32); }
        }
        return 0;
    });
#undef STML_TILE
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t apply_launch(const Geom& g, const FrameSet& fs, const Coef& cf, const Stored& dT, const DirSrc& src,
                         float* Hv, double* partials, size_t partials_cap, unsigned int* ticket, double* out,
                         DevScalars* pcg, cudaStream_t s) {
    const PixIndex pi = make_pix_index(g);
    const bool v4 = vec4_ok(g, {dT.p, src.z, Hv, src.ms_z, src.sv_z});
    const int vec = v4 ? 4 : 1;
    const long long cpf = (g.N + (long long)kThreads * vec - 1) / ((long long)kThreads * vec);
    const long long items = cpf * fs.nK;
    const FastDiv chunks = FastDiv::make((unsigned)cpf);
    return with_store_type(dT.type, [&](auto tag) -> cudaError_t {
        using TD = decltype(tag);
        const TD* Td = static_cast<const TD*>(dT.p);
        auto k = g.d == 2 ? (v4 ? apply_kernel<2, 4, TD> : apply_kernel<2, 1, TD>)
                          : (v4 ? apply_kernel<3, 4, TD> : apply_kernel<3, 1, TD>);
        const unsigned grid = resident_grid((const void*)k, items, kGridStride);
        if ((size_t)grid > partials_cap) return cudaErrorInvalidValue;
        k<<<grid, kThreads, 0, s>>>(g, pi, chunks, items, fs, cf, Td, src, Hv, partials, ticket, out, pcg);
        count_launches(1);
        return cudaGetLastError();
    });
}

}  // namespace

size_t gn_partials(const Geom& g, int nK) {
    const size_t tile = (size_t)((g.N + 7) / 8) * 2;
    const size_t gs = (size_t)kGridStride * 2;
    (void)nK;
    return tile > gs ? tile : gs;
}

cudaError_t launch_hess_sums(const Geom& g, const FrameSet& fs, const float* dT, const float* v, float* mean_s,
                             float* sum_v, cudaStream_t s) {
    Coef cf{};
    return tile_launch<TILE_SUMS>(g, fs, cf, Stored{dT, ST_F32}, const_cast<float*>(v), nullptr, nullptr, nullptr, mean_s, sum_v,
                                  nullptr, nullptr, PcgArgs{0.f, 0}, s);
}

cudaError_t launch_hess_apply(const Geom& g, const FrameSet& fs, const Coef& cf, const float* dT, const float* v,
                              const float* mean_s, const float* sum_v, float* Hv, double* partials,
                              size_t partials_cap, unsigned int* ticket, double* out, DevScalars* pcg,
                              cudaStream_t s) {
    const DirSrc src{v, nullptr, 0.f, nullptr, mean_s, sum_v, nullptr, nullptr, nullptr, nullptr};
    return apply_launch(g, fs, cf, Stored{dT, ST_F32}, src, Hv, partials, partials_cap, ticket, out, pcg, s);
}

cudaError_t launch_pcg_init(const Geom& g, const FrameSet& fs, const Coef& cf, const float* grad, const Stored& dT,
                            const PcgBufs& b, double* partials, size_t partials_cap, DevScalars* S, PcgArgs a,
                            cudaStream_t s, const int* gate) {
    if ((size_t)((g.N + 7) / 8) * 2 > partials_cap) return cudaErrorInvalidValue;
    return tile_launch<TILE_INIT>(g, fs, cf, dT, b.p[0], b.r, grad, b.x, b.ms_z, b.sv_z, partials, S, a, s, gate);
}

cudaError_t launch_pcg_apply(const Geom& g, const FrameSet& fs, const Coef& cf, const Stored& dT, const PcgBufs& b,
                             double* partials, size_t partials_cap, DevScalars* S, cudaStream_t s) {
    const DirSrc src{b.p[0], nullptr, 0.f, nullptr, b.ms_z, b.sv_z, nullptr, nullptr, nullptr, nullptr};
    return apply_launch(g, fs, cf, dT, src, b.q, partials, partials_cap, &S->ticket[1], S->dots + 4, S, s);
}

cudaError_t launch_pcg_update(const Geom& g, const FrameSet& fs, const Coef& cf, const Stored& dT, const PcgBufs& b,
                              double* partials, size_t partials_cap, DevScalars* S, PcgArgs a, cudaStream_t s) {
    const PixIndex pi = make_pix_index(g);
    const bool v4 = vec4_ok(g, {dT.p, b.x, b.r, b.p[0], b.q});
    const int vec = v4 ? 4 : 1;
    const long long cpf = (g.N + (long long)kThreads * vec - 1) / ((long long)kThreads * vec);
    const long long items = cpf * fs.nK * g.d;
    const FastDiv chunks = FastDiv::make((unsigned)cpf);
    return with_store_type(dT.type, [&](auto tag) -> cudaError_t {
        using TD = decltype(tag);
        const TD* Td = static_cast<const TD*>(dT.p);
        auto k = g.d == 2 ? (v4 ? update_kernel<2, 4, TD> : update_kernel<2, 1, TD>)
                          : (v4 ? update_kernel<3, 4, TD> : update_kernel<3, 1, TD>);
        const unsigned grid = resident_grid((const void*)k, items, kGridStride);
        if ((size_t)grid * 2 > partials_cap) return cudaErrorInvalidValue;
        k<<<grid, kThreads, 0, s>>>(g, pi, chunks, items, fs, cf, Td, b.x, b.r, b.p[0], b.q, partials, S, a);
        count_launches(1);
        return cudaGetLastError();
    });
}

cudaError_t launch_pcg_direction(const Geom& g, const FrameSet& fs, const Coef& cf, const Stored& dT,
                                 const PcgBufs& b, DevScalars* S, cudaStream_t s) {
    return tile_launch<TILE_DIR>(g, fs, cf, dT, b.p[0], b.r, nullptr, nullptr, b.ms_z, b.sv_z, nullptr, S,
                                 PcgArgs{0.f, 0}, s);
}

namespace {

template <int D, int VEC, int TPR, typename TD>
cudaError_t coop_go(const Geom& g, const FrameSet& fs, const Coef& cf, const float* grad, const TD* dT,
                    const PcgBufs& b, double* partials, size_t partials_cap, DevScalars* S, PcgArgs a,
                    cudaStream_t s, const int* gate) {
    const void* kern = (const void*)pcg_coop_kernel<D, VEC, TPR, TD>;
    int dev = 0, sms = 1, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    PixIndex pi = make_pix_index(g);
    long long cpf = (g.N + (long long)kThreads * VEC - 1) / ((long long)kThreads * VEC);
    long long aitems = cpf * fs.nK;
    unsigned tiles = (unsigned)((g.N + TPR * VEC - 1) / (TPR * VEC));
    const long long want = aitems > (long long)tiles ? aitems : (long long)tiles;
    // at most two CTAs per SM (and what fits): more warps for the memory
    // stream, while the grid barriers stay cheap
    const long long cap = (long long)sms * (per_sm < 2 ? per_sm : 2);
    unsigned blocks = (unsigned)(want < cap ? want : cap);
    if (blocks < 1) blocks = 1;
    if ((size_t)blocks * 4 > partials_cap) return cudaErrorInvalidValue;
    FastDiv chunks = FastDiv::make((unsigned)cpf);
    Geom gg = g;
    FrameSet ff = fs;
    Coef cc = cf;
    PcgBufs bb = b;
    PcgArgs aa = a;
    void* args[] = {&gg, &pi, &chunks, &aitems, &tiles, &ff, &cc, (void*)&grad, (void*)&dT, &bb, &partials, &S, &aa,
                    (void*)&gate};
    e = cudaLaunchCooperativeKernel(kern, dim3(blocks), dim3(kThreads), args, 0, s);
    count_launches(1);
    return e;
}

}  // namespace

// Cooperative solves win up to about 2^21 pixel-frames (measured with the
// autotuner on the paper-scale sequence).
bool pcg_coop_preferred(const Geom& g, int nK) { return (long long)g.N * nK <= (1LL << 21); }

cudaError_t launch_pcg_coop(const Geom& g, const FrameSet& fs, const Coef& cf, const float* grad, const Stored& dT,
                            const PcgBufs& b, double* partials, size_t partials_cap, DevScalars* S, PcgArgs a,
                            cudaStream_t s, const int* gate) {
    const bool v4 = vec4_ok(g, {grad, dT.p, b.x, b.r, b.z, b.q, b.p[0], b.p[1], b.ms_z, b.sv_z, b.ms_p[0],
                                b.sv_p[0], b.ms_p[1], b.sv_p[1]});
    return with_store_type(dT.type, [&](auto tag) {
        using TD = decltype(tag);
        const TD* Td = static_cast<const TD*>(dT.p);
        if (g.d == 2)
            return v4 ? coop_go<2, 4, 4>(g, fs, cf, grad, Td, b, partials, partials_cap, S, a, s, gate)
                      : coop_go<2, 1, 8>(g, fs, cf, grad, Td, b, partials, partials_cap, S, a, s, gate);
        return v4 ? coop_go<3, 4, 4>(g, fs, cf, grad, Td, b, partials, partials_cap, S, a, s, gate)
                  : coop_go<3, 1, 8>(g, fs, cf, grad, Td, b, partials, partials_cap, S, a, s, gate);
    });
}

}  // namespace stml
