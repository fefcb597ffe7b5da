// Objective of eq. (1) with the regulariser S and penalty P (Sec. 2), its
// gradient and grad T at the warped positions, as two streaming passes.
//
// obj_kernel (pixel-tiled, all frames of a pixel in one CTA): for every frame
//   a_k = T_k(x + u_k(x)) (linear interpolation, zero outside), folded into a
//   per-pixel Welford mean / sum of squared deviations, so that
//   D = hd/2 sum_x sum_k (a_k - abar)^2 needs no second sweep; the diffusion
//   energy of u_k (forward differences), the temporal term, |u|^2 and the
//   frame sum of u.  It writes abar and ubar per pixel and reduces D, S, P.
// grad_kernel (element-wise over (frame, pixels)): a_k and grad T_k again,
//   r_k = a_k - abar, g_k = hd r_k grad T_k + alpha hd B^T B u_k
//   + alpha_t hd (L_t u)_k + 2 lambda hd ubar / |K|; writes g and grad T and
//   reduces |g|^2.
// Fields may be read as u + t du (an Armijo trial point); grad_kernel can also
// write that point out (the accepted Gauss-Newton step), so the objective
// pass of the trial supplies abar and ubar at the new iterate.
#include "kernels.h"

namespace stml {

namespace {

struct FView {
    const float* __restrict__ u;
    const float* __restrict__ d;
    float t;
    __device__ __forceinline__ float ld(size_t i) const { return d ? fmaf(t, __ldg(d + i), __ldg(u + i)) : __ldg(u + i); }
    __device__ __forceinline__ float4 ld4(size_t i) const {
        const float4 a = __ldg(reinterpret_cast<const float4*>(u + i));
        if (!d) return a;
        const float4 b = __ldg(reinterpret_cast<const float4*>(d + i));
        return make_float4(fmaf(t, b.x, a.x), fmaf(t, b.y, a.y), fmaf(t, b.z, a.z), fmaf(t, b.w, a.w));
    }
};

template <int VEC>
__device__ __forceinline__ void vload(const FView& V, size_t i, float (&o)[VEC]) {
    if constexpr (VEC == 4) {
        const float4 q = V.ld4(i);
        o[0] = q.x; o[1] = q.y; o[2] = q.z; o[3] = q.w;
    } else {
        o[0] = V.ld(i);
    }
}

template <int VEC>
__device__ __forceinline__ void vstore(float* p, size_t i, const float (&v)[VEC]) {
    if constexpr (VEC == 4)
        *reinterpret_cast<float4*>(p + i) = make_float4(v[0], v[1], v[2], v[3]);
    else
        p[i] = v[0];
}

__device__ __forceinline__ void pos_of(const PixIndex& pi, unsigned p, int& x, int& y, int& z) {
    const unsigned r = pi.nx.div(p);
    x = (int)(p - r * pi.nx.d);
    const unsigned zz = pi.ny.div(r);
    y = (int)(r - zz * pi.ny.d);
    z = (int)zz;
}

template <int D>
__device__ __forceinline__ void interp(const float* __restrict__ Tk, const Geom& g, int x, int y, int z,
                                       const float (&u)[D], float& a, float (&gr)[D]) {
    if constexpr (D == 2)
        interp2(Tk, g, x, y, u[0], u[1], a, gr[0], gr[1]);
    else
        interp3(Tk, g, x, y, z, u[0], u[1], u[2], a, gr[0], gr[1], gr[2]);
}

}  // namespace

// ----------------------------------------------------------------- objective
// Reduced values: 0 D, 1 S_x, 2 S_t, 3 P, 4 (unused), 5 |u|^2.
// With gdot != nullptr the pass also reduces <gdot, du> and |du|^2 (the
// directional derivative of the Gauss-Newton step) into out[6], out[7].
template <int D, int VEC, int TPR>
__global__ void __launch_bounds__(kThreads, 3)
obj_kernel(const float* __restrict__ T, Geom g, PixIndex pi, FrameSet fs, Coef cf, FView U,
           const float* __restrict__ gdot, float* __restrict__ abar, float* __restrict__ ubar,
           double* __restrict__ partials, unsigned int* ticket, double* out) {
    constexpr int SEG = TPR * VEC, FG = kThreads / TPR;
    __shared__ float sh_n[FG][SEG], sh_m[FG][SEG], sh_q[FG][SEG];
    __shared__ float sh_u[FG][D][SEG];
    const int lane = threadIdx.x % TPR, fg = threadIdx.x / TPR;
    const unsigned p = blockIdx.x * SEG + lane * VEC;
    const bool valid = p < (unsigned)g.N;
    const size_t N = (size_t)g.N;
    int x = 0, y = 0, z = 0;
    if (valid) pos_of(pi, p, x, y, z);
    float cnt = 0.f, mean[VEC], m2[VEC], su[D][VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
        mean[e] = 0.f;
        m2[e] = 0.f;
#pragma unroll
        for (int c = 0; c < D; ++c) su[c][e] = 0.f;
    }
    float sx = 0.f, st = 0.f, u2 = 0.f, gd = 0.f, dd = 0.f;
    if (valid) {
#pragma unroll 2
        for (int j = fg; j < fs.nK; j += FG) {
            const float* Tk = T + (size_t)__ldg(fs.frames + j) * N;
            if (gdot) {
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    const size_t base = ((size_t)j * D + c) * N + p;
                    float gv[VEC], dv[VEC];
                    const FView G{gdot, nullptr, 0.f}, Dv{U.d, nullptr, 0.f};
                    vload<VEC>(G, base, gv);
                    vload<VEC>(Dv, base, dv);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) {
                        gd = fmaf(gv[e], dv[e], gd);
                        dd = fmaf(dv[e], dv[e], dd);
                    }
                }
            }
            const float w_next = (cf.alphat_hd != 0.f && j + 1 < fs.nK) ? __ldg(fs.w_next + j) : 0.f;
            float uc[D][VEC];
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const size_t base = ((size_t)j * D + c) * N + p;
                vload<VEC>(U, base, uc[c]);
                // forward differences to +x (inside the thread's run, then the next run), +y, +z
                float fw = 0.f;
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    if (x + e < g.nx - 1) {
                        const float nb = e + 1 < VEC ? uc[c][e + 1] : U.ld(base + VEC);
                        fw = fmaf(nb - uc[c][e], nb - uc[c][e], fw);
                    }
                }
                if (y < g.ny - 1) {
                    float nb[VEC];
                    vload<VEC>(U, base + g.nx, nb);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) fw = fmaf(nb[e] - uc[c][e], nb[e] - uc[c][e], fw);
                }
                if constexpr (D == 3) {
                    if (z < g.nz - 1) {
                        float nb[VEC];
                        vload<VEC>(U, base + (size_t)g.nx * g.ny, nb);
#pragma unroll
                        for (int e = 0; e < VEC; ++e) fw = fmaf(nb[e] - uc[c][e], nb[e] - uc[c][e], fw);
                    }
                }
                sx = fmaf(0.5f * cf.alpha_hd * cf.inv_h2, fw, sx);
                if (w_next != 0.f) {
                    float nb[VEC];
                    vload<VEC>(U, base + (size_t)D * N, nb);
#pragma unroll
                    for (int e = 0; e < VEC; ++e)
                        st = fmaf(0.5f * cf.alphat_hd * w_next * (nb[e] - uc[c][e]), nb[e] - uc[c][e], st);
                }
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    su[c][e] += uc[c][e];
                    u2 = fmaf(uc[c][e], uc[c][e], u2);
                }
            }
            cnt += 1.f;
            const float rc = 1.0f / cnt;
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                float a;
                if constexpr (D == 2) {
                    a = interp2_val(Tk, g, x + e, y, uc[0][e], uc[1][e]);
                } else {
                    float uu[D], gr[D];
#pragma unroll
                    for (int c = 0; c < D; ++c) uu[c] = uc[c][e];
                    interp<D>(Tk, g, x + e, y, z, uu, a, gr);
                }
                const float dlt = a - mean[e];
                mean[e] = fmaf(dlt, rc, mean[e]);
                m2[e] = fmaf(dlt, a - mean[e], m2[e]);
            }
        }
    }
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
        const int k = lane * VEC + e;
        sh_n[fg][k] = cnt;
        sh_m[fg][k] = mean[e];
        sh_q[fg][k] = m2[e];
#pragma unroll
        for (int c = 0; c < D; ++c) sh_u[fg][c][k] = su[c][e];
    }
    __syncthreads();
    // combine the frame groups of every pixel (Chan's update, group order)
    float dsum = 0.f, pen = 0.f;
    if (threadIdx.x < SEG) {
        const int k = threadIdx.x;
        const unsigned pp = blockIdx.x * SEG + k;
        if (pp < (unsigned)g.N) {
            float n = 0.f, m = 0.f, q = 0.f;
            for (int w = 0; w < FG; ++w) {
                const float nb = sh_n[w][k];
                if (nb == 0.f) continue;
                const float tot = n + nb;
                const float dl = sh_m[w][k] - m;
                m = fmaf(dl, nb / tot, m);
                q = q + sh_q[w][k] + dl * dl * (n * nb / tot);
                n = tot;
            }
            abar[pp] = m;
            dsum = cf.half_hd * q;
            const float invK = 1.0f / (float)fs.nK;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                float s = 0.f;
                for (int w = 0; w < FG; ++w) s += sh_u[w][c][k];
                const float ub = s * invK;
                ubar[(size_t)c * N + pp] = ub;
                pen = fmaf(cf.lam_hd * ub, ub, pen);
            }
        }
    }
    float acc[8] = {dsum, sx, st, pen, 0.f, u2, gd, dd};
    if (grid_reduce<8>(acc, partials, ticket, out) && threadIdx.x == 0) {
        const double Dv = out[0], Sx = out[1], St = out[2], Pv = out[3];
        out[0] = Dv + Sx + St + Pv;
        out[1] = Dv;
        out[2] = Sx + St;
        out[3] = Pv;
    }
}

// ----------------------------------------------------------------- gradient
// Grid-stride over items (frame j, chunk of kThreads * VEC pixels).  Reduced:
// out[4] = |g|^2 (added to the objective pass's totals), out[5] = |u|^2.
template <int D, int VEC>
__global__ void __launch_bounds__(kThreads)
grad_kernel(const float* __restrict__ T, Geom g, PixIndex pi, FastDiv chunks, long long items, FrameSet fs,
            Coef cf, FView U, const float* __restrict__ abar, const float* __restrict__ ubar,
            float* __restrict__ grad, float* __restrict__ dTout, float* __restrict__ unew,
            double* __restrict__ partials, unsigned int* ticket, double* out) {
    const size_t N = (size_t)g.N;
    const int lane = threadIdx.x & 31;
    float g2 = 0.f, u2 = 0.f;
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const unsigned j = chunks.div((unsigned)it);
        const unsigned ch = (unsigned)it - j * chunks.d;
        const unsigned p = (ch * kThreads + threadIdx.x) * VEC;
        const bool valid = p < (unsigned)g.N;
        int x = 0, y = 0, z = 0;
        if (valid) pos_of(pi, p, x, y, z);
        const float* Tk = T + (size_t)__ldg(fs.frames + j) * N;
        const float w_next = (cf.alphat_hd != 0.f && j + 1 < (unsigned)fs.nK) ? __ldg(fs.w_next + j) : 0.f;
        const float w_prev = (cf.alphat_hd != 0.f && j > 0) ? __ldg(fs.w_next + j - 1) : 0.f;
        float uc[D][VEC];
#pragma unroll
        for (int c = 0; c < D; ++c) {
            if (valid)
                vload<VEC>(U, ((size_t)j * D + c) * N + p, uc[c]);
            else
#pragma unroll
                for (int e = 0; e < VEC; ++e) uc[c][e] = 0.f;
        }
        float r[VEC], dt[D][VEC];
        if (valid) {
            float ab[VEC];
            if constexpr (VEC == 4) {
                const float4 q = __ldg(reinterpret_cast<const float4*>(abar + p));
                ab[0] = q.x; ab[1] = q.y; ab[2] = q.z; ab[3] = q.w;
            } else {
                ab[0] = __ldg(abar + p);
            }
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                float uu[D], a, gr[D];
#pragma unroll
                for (int c = 0; c < D; ++c) uu[c] = uc[c][e];
                interp<D>(Tk, g, x + e, y, z, uu, a, gr);
                r[e] = a - ab[e];
#pragma unroll
                for (int c = 0; c < D; ++c) dt[c][e] = gr[c];
            }
        }
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const size_t base = ((size_t)j * D + c) * N + p;
            const float up_l = __shfl_up_sync(0xffffffffu, uc[c][VEC - 1], 1);
            const float dn_r = __shfl_down_sync(0xffffffffu, uc[c][0], 1);
            if (!valid) continue;
            float left = 0.f, right = 0.f;
            if (x > 0) left = lane > 0 ? up_l : U.ld(base - 1);
            if (x + VEC < g.nx) right = lane < 31 ? dn_r : U.ld(base + VEC);
            float lap[VEC];
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                const float le = e == 0 ? left : uc[c][e - 1];
                const float re = e == VEC - 1 ? right : uc[c][e + 1];
                float lp = 0.f;
                if (x + e > 0) lp += uc[c][e] - le;
                if (x + e < g.nx - 1) lp += uc[c][e] - re;
                lap[e] = lp;
            }
            float nb[VEC];
            if (y > 0) {
                vload<VEC>(U, base - g.nx, nb);
#pragma unroll
                for (int e = 0; e < VEC; ++e) lap[e] += uc[c][e] - nb[e];
            }
            if (y < g.ny - 1) {
                vload<VEC>(U, base + g.nx, nb);
#pragma unroll
                for (int e = 0; e < VEC; ++e) lap[e] += uc[c][e] - nb[e];
            }
            if constexpr (D == 3) {
                const size_t sz = (size_t)g.nx * g.ny;
                if (z > 0) {
                    vload<VEC>(U, base - sz, nb);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) lap[e] += uc[c][e] - nb[e];
                }
                if (z < g.nz - 1) {
                    vload<VEC>(U, base + sz, nb);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) lap[e] += uc[c][e] - nb[e];
                }
            }
            float tg[VEC];
#pragma unroll
            for (int e = 0; e < VEC; ++e) tg[e] = 0.f;
            if (w_next != 0.f) {
                vload<VEC>(U, base + (size_t)D * N, nb);
#pragma unroll
                for (int e = 0; e < VEC; ++e) tg[e] += w_next * (uc[c][e] - nb[e]);
            }
            if (w_prev != 0.f) {
                vload<VEC>(U, base - (size_t)D * N, nb);
#pragma unroll
                for (int e = 0; e < VEC; ++e) tg[e] += w_prev * (uc[c][e] - nb[e]);
            }
            float ub[VEC];
            if constexpr (VEC == 4) {
                const float4 q = __ldg(reinterpret_cast<const float4*>(ubar + (size_t)c * N + p));
                ub[0] = q.x; ub[1] = q.y; ub[2] = q.z; ub[3] = q.w;
            } else {
                ub[0] = __ldg(ubar + (size_t)c * N + p);
            }
            float gv[VEC];
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                gv[e] = fmaf(cf.hd * r[e], dt[c][e],
                             fmaf(cf.alpha_hd * cf.inv_h2, lap[e], fmaf(cf.alphat_hd, tg[e], cf.pen_g * ub[e])));
                g2 = fmaf(gv[e], gv[e], g2);
                u2 = fmaf(uc[c][e], uc[c][e], u2);
            }
            vstore<VEC>(grad, base, gv);
            vstore<VEC>(dTout, base, dt[c]);
            if (unew) vstore<VEC>(unew, base, uc[c]);
        }
    }
    float acc[2] = {g2, u2};
    double tot[2];
    if (grid_reduce<2>(acc, partials, ticket, tot) && threadIdx.x == 0) {
        out[4] = tot[0];
        out[5] = tot[1];
    }
}

// ----------------------------------------------------------------- launchers
namespace {

constexpr int kGridStride = 152 * 8;   // CTAs of the grid-stride launches (8 per SM of a GB300)

bool v4ok(const Geom& g, std::initializer_list<const void*> ptrs) {
    if (g.nx % 4) return false;
    for (const void* q : ptrs)
        if (q && ((uintptr_t)q & 15u)) return false;
    return true;
}

}  // namespace

size_t eval_partials(const Geom& g, int nK) {
    const size_t obj = (size_t)((g.N + 7) / 8) * 8;
    return obj > (size_t)kGridStride * 2 ? obj : (size_t)kGridStride * 2;
    (void)nK;
}

template <int D, int VEC, int TPR>
static void obj_go(unsigned blocks, cudaStream_t s, const float* T, const Geom& g, const PixIndex& pi,
                   const FrameSet& fs, const Coef& cf, const FView& U, const float* gdot, float* abar, float* ubar,
                   double* partials, unsigned int* ticket, double* out) {
    obj_kernel<D, VEC, TPR><<<blocks, kThreads, 0, s>>>(T, g, pi, fs, cf, U, gdot, abar, ubar, partials, ticket, out);
}

cudaError_t launch_objective(const float* T, const Geom& g, const FrameSet& fs, const Coef& cf, const float* u,
                             const float* du, float t, const float* gdot, float* abar, float* ubar, double* partials,
                             size_t partials_cap, unsigned int* ticket, double* out, cudaStream_t s) {
    const PixIndex pi{FastDiv::make((unsigned)g.nx), FastDiv::make((unsigned)g.ny)};
    const bool v4 = v4ok(g, {u, du, gdot, abar, ubar});
    // wide pixel tiles on large levels, narrow ones (more CTAs, more frame groups) on small levels
    const bool narrow = g.N < 4LL * 152 * (v4 ? 64 : 32);
    const int seg = v4 ? (narrow ? 16 : 64) : (narrow ? 8 : 32);
    const unsigned blocks = (unsigned)((g.N + seg - 1) / seg);
    if ((size_t)blocks * 8 > partials_cap) return cudaErrorInvalidValue;
    if (gdot && !du) return cudaErrorInvalidValue;
    const FView U{u, du, t};
#define STML_OBJ(D_, V_, T_) obj_go<D_, V_, T_>(blocks, s, T, g, pi, fs, cf, U, gdot, abar, ubar, partials, ticket, out)
    if (g.d == 2) {
        if (v4) { if (narrow) STML_OBJ(2, 4, 4); else STML_OBJ(2, 4, 16); }
        else { if (narrow) STML_OBJ(2, 1, 8); else STML_OBJ(2, 1, 32); }
    } else {
        if (v4) { if (narrow) STML_OBJ(3, 4, 4); else STML_OBJ(3, 4, 16); }
        else { if (narrow) STML_OBJ(3, 1, 8); else STML_OBJ(3, 1, 32); }
    }
#undef STML_OBJ
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_gradient(const float* T, const Geom& g, const FrameSet& fs, const Coef& cf, const float* u,
                            const float* du, float t, const float* abar, const float* ubar, float* grad, float* dT,
                            float* unew, double* partials, size_t partials_cap, unsigned int* ticket, double* out,
                            cudaStream_t s) {
    const PixIndex pi{FastDiv::make((unsigned)g.nx), FastDiv::make((unsigned)g.ny)};
    const bool v4 = v4ok(g, {u, du, abar, ubar, grad, dT, unew});
    const int vec = v4 ? 4 : 1;
    const long long cpf = (g.N + (long long)kThreads * vec - 1) / ((long long)kThreads * vec);
    const long long items = cpf * fs.nK;
    const unsigned blocks = (unsigned)(items < kGridStride ? items : kGridStride);
    if ((size_t)blocks * 2 > partials_cap) return cudaErrorInvalidValue;
    const FastDiv chunks = FastDiv::make((unsigned)cpf);
    const FView U{u, du, t};
    if (g.d == 2) {
        if (v4) grad_kernel<2, 4><<<blocks, kThreads, 0, s>>>(T, g, pi, chunks, items, fs, cf, U, abar, ubar, grad, dT, unew, partials, ticket, out);
        else grad_kernel<2, 1><<<blocks, kThreads, 0, s>>>(T, g, pi, chunks, items, fs, cf, U, abar, ubar, grad, dT, unew, partials, ticket, out);
    } else {
        if (v4) grad_kernel<3, 4><<<blocks, kThreads, 0, s>>>(T, g, pi, chunks, items, fs, cf, U, abar, ubar, grad, dT, unew, partials, ticket, out);
        else grad_kernel<3, 1><<<blocks, kThreads, 0, s>>>(T, g, pi, chunks, items, fs, cf, U, abar, ubar, grad, dT, unew, partials, ticket, out);
    }
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace stml
