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

#include "gn_items.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace stml {

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
    pdl_enter();
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
    dt.load_t_cs(dT + e0);   // grad T, q and x: next read after the other passes of the step
    pv.load(p + e0);         // p: read again by the direction step that follows
    qv.load_cs(q + e0);
    xv.load_cs(x + e0);
    rv.load_rw(r + e0);
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
        xv.a[e] = fmaf(al, pv.a[e], xv.a[e]);
        rv.a[e] = fmaf(-al, qv.a[e], rv.a[e]);
        const float zv = jacobi_inv(dt.a[e], neighbour_count(g, xx + e, yy, zz), tdiag, cf) * rv.a[e];
        rz = fmaf(rv.a[e], zv, rz);
        rr = fmaf(rv.a[e], rv.a[e], rr);
    }
    xv.store_cs(x + e0);
    rv.store(r + e0);        // r: read by the direction step that follows
}

// The PCG update.  It first completes the Hessian-product pass before it:
// every CTA sums that pass's CTA partials of <p, Hp> (fixed order, the same
// total everywhere) and takes the CG decision alpha = rho / <p, Hp>, so the
// Hessian-product pass ends without a serial last-CTA reduction.  On a
// breakdown (p^T H p <= 0) nothing is updated and CTA 0 records it.
template <int D, int VEC, typename TD>
__global__ void __launch_bounds__(kThreads)
update_kernel(Geom g, PixIndex pi, FastDiv chunks, long long items, FrameSet fs, Coef cf,
              const TD* __restrict__ dT, float* __restrict__ x, float* __restrict__ r,
              const float* __restrict__ p, const float* __restrict__ q, double* __restrict__ partials,
              const double* __restrict__ pq_partials, DevScalars* S, PcgArgs a) {
    pdl_enter();
    if (!S->cg_active) return;
    CgState st = cg_load(S);
    {
        dfloat tot[1];
        cta_total<1>(reinterpret_cast<const float2*>(pq_partials), (unsigned)S->pq_parts, tot);
        cg_after_apply(st, df_val(tot[0]));
    }
    if (!st.active) {
        if (blockIdx.x == 0 && threadIdx.x == 0) cg_store(S, st);
        return;
    }
    const float al = st.alpha;
    float acc[2] = {0.f, 0.f};
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const int plane = (int)chunks.div((unsigned)it);
        update_item<D, VEC, TD>(g, pi, fs, cf, dT, x, r, p, q, plane, (unsigned)it - (unsigned)plane * chunks.d, al,
                            acc[0], acc[1]);
    }
    double tot[2];
    if (grid_reduce<2>(acc, partials, &S->ticket[2], tot) && threadIdx.x == 0) {
        cg_after_update(st, (float)tot[0], (float)tot[1], a.tol_cg, a.max_cg);
        cg_store(S, st);
    }
}

// Hessian product stream (grid-stride over (frame, chunk) items) of
// v = src.z with its frame sums src.ms_z / src.sv_z.  Plain product: the
// last CTA writes <v, Hv> to out[0].  With pcg != nullptr the launch is a PCG
// step: it does nothing once cg_active is 0, and each CTA stores its partial
// of <p, Hp> (double-float) for the update pass, which completes the sum.
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
    pdl_enter();
    if (pcg && !pcg->cg_active) return;
    float acc[1] = {0.f};
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const int j = (int)chunks.div((unsigned)it);
        apply_item<D, VEC, false, TD>(g, pi, fs, cf, dT, src, Hv, j, (unsigned)it - (unsigned)j * chunks.d, acc[0]);
    }
    if (pcg) {
        cta_partials<1>(acc, reinterpret_cast<float2*>(partials), blockIdx.x);
        if (blockIdx.x == 0 && threadIdx.x == 0) pcg->pq_parts = (int)gridDim.x;
        return;
    }
    grid_reduce<1>(acc, partials, ticket, out);
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
// The PCG Hessian product's CTA partials of <p, Hp> (one double each) start
// here in the partials buffer, after the update pass's own (2 per CTA).
constexpr size_t kPqOffset = 2 * (size_t)kGridStride;

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
    e = launch_pdl(tile_kernel<D_, V_, MODE, T_, TD>, dim3(blocks), dim3(kThreads), 0, s, g, pi, fs, cf, Td, v, r,  \
                   grad, x, mean_s, sum_v, partials, S, a, gate)
    cudaError_t e = cudaSuccess;
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
    return e != cudaSuccess ? e : cudaGetLastError();
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
        const cudaError_t e =
            launch_pdl(k, dim3(grid), dim3(kThreads), 0, s, g, pi, chunks, items, fs, cf, Td, src, Hv, partials, ticket,
                       out, pcg);
        count_launches(1);
        return e != cudaSuccess ? e : cudaGetLastError();
    });
}

}  // namespace

size_t gn_partials(const Geom& g, int nK) {
    const size_t tile = (size_t)((g.N + 7) / 8) * 2;
    const size_t gs = (size_t)kGridStride * 3;   // the update's partials, then the PCG <p, Hp> partials
    (void)nK;
    return tile > gs ? tile : gs;
}

cudaError_t launch_hess_sums(const Geom& g, const FrameSet& fs, const float* dT, const float* v, float* mean_s,
                             float* sum_v, cudaStream_t s, const int* gate) {
    Coef cf{};
    return tile_launch<TILE_SUMS>(g, fs, cf, Stored{dT, ST_F32}, const_cast<float*>(v), nullptr, nullptr, nullptr, mean_s, sum_v,
                                  nullptr, nullptr, PcgArgs{0.f, 0}, s, gate);
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
    if (partials_cap < kPqOffset) return cudaErrorInvalidValue;
    return apply_launch(g, fs, cf, dT, src, b.q, partials + kPqOffset, partials_cap - kPqOffset, &S->ticket[1],
                        S->dots + 4, S, s);
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
        if ((size_t)grid * 2 > kPqOffset || partials_cap < kPqOffset + kGridStride) return cudaErrorInvalidValue;
        const cudaError_t e = launch_pdl(k, dim3(grid), dim3(kThreads), 0, s, g, pi, chunks, items, fs, cf, Td, b.x,
                                         b.r, b.p[0], b.q, partials, partials + kPqOffset, S, a);
        count_launches(1);
        return e != cudaSuccess ? e : cudaGetLastError();
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
