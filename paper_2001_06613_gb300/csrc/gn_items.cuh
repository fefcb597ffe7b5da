// Per-item bodies of the Gauss-Newton Hessian product and of the Jacobi-PCG
// passes, shared by the stream kernels and the cooperative solve (k_gn.cu)
// and by the persistent batched solver (k_batch.cu):
//
//   (Hv)_k = hd grad T_k (s_k - sbar) + alpha hd B^T B v_k + alpha_t hd (L_t v)_k
//            + 2 lambda hd / |K|^2 sum_j v_j,          s_k = grad T_k . v_k
//
// tile_pass visits all frames of a pixel tile (frame sums, PCG start, update
// and direction steps); apply_item streams one (frame, chunk) item of the
// Hessian product; CgState and cg_after_* take the CG decisions from the
// reduced totals.  Internal to the library.
#pragma once

#include "kernels.h"

namespace stml {
namespace {

__device__ __forceinline__ float4 ld4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
// Streaming (evict-first) loads and stores for arrays a pass touches once and
// no pass reads again before several others have streamed through L2.
__device__ __forceinline__ float4 ld4cs(const float* p) { return __ldcs(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ void ldcs4f(const float* p, float (&o)[4]) {
    const float4 q = ld4cs(p);
    o[0] = q.x; o[1] = q.y; o[2] = q.z; o[3] = q.w;
}
__device__ __forceinline__ void ldcs4f(const __half* p, float (&o)[4]) {
    const uint2 q = __ldcs(reinterpret_cast<const uint2*>(p));
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&q.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&q.y));
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
__device__ __forceinline__ void ldcs4f(const __nv_bfloat16* p, float (&o)[4]) {
    const uint2 q = __ldcs(reinterpret_cast<const uint2*>(p));
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q.y));
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
__device__ __forceinline__ float ldcs1(const float* p) { return __ldcs(p); }
__device__ __forceinline__ float ldcs1(const __half* p) { return __half2float(__ldcs(p)); }
__device__ __forceinline__ float ldcs1(const __nv_bfloat16* p) { return __bfloat162float(__ldcs(p)); }
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
    __device__ __forceinline__ void load_cs(const float* p) { ldcs4f(p, a); }
    template <typename T>
    __device__ __forceinline__ void load_t_cs(const T* p) { ldcs4f(p, a); }
    __device__ __forceinline__ void store_cs(float* p) const {
        __stcs(reinterpret_cast<float4*>(p), make_float4(a[0], a[1], a[2], a[3]));
    }
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
    __device__ __forceinline__ void load_cs(const float* p) { a[0] = __ldcs(p); }
    template <typename T>
    __device__ __forceinline__ void load_t_cs(const T* p) { a[0] = ldcs1(p); }
    __device__ __forceinline__ void store_cs(float* p) const { __stcs(p, a[0]); }
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
                if constexpr (MODE == TILE_DIR)
                    dt.load_t_cs(dT + e0);
                else
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
            dt[c].load_t_cs(dT + e0);
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
}  // namespace stml
