// Persistent batched Gauss-Newton solver: the GIRs of many sequences (of
// uneven frame counts and sizes) at one (spatial level, temporal level) stage
// of their multilevel sweeps, in one cooperative launch.
//
// Every sequence carries a small state machine on the device (its next phase,
// the CG coefficients, the Armijo state and the Gauss-Newton bookkeeping).
// The kernel runs in steps; in a step every active sequence executes its
// current phase:
//
//   EVAL0   objective and gradient at the start (pixel tiles over all frames)
//   INIT    PCG start r = -g, z = M^-1 r, x = 0 and the frame sums of z
//   APPLY   p = z + beta p_old and q = H p (frame, chunk items)
//   UPDATE  x += alpha p, r -= alpha q, z = M^-1 r and its frame sums
//   TRIAL   objective at u + t d, t = 2^-k (Armijo test)
//   GRAD    gradient at the accepted point, which becomes the iterate
//
// The grid is cut, in every step, into contiguous CTA ranges, one per active
// sequence, sized in proportion to the bytes its phase moves: the device work
// queue is the list of (sequence, phase, tile) items the ranges stride over.
// Each CTA reduces its items' sums in double-float and stores them in its own
// slot; after a grid barrier the first CTA of each range sums its range's
// slots in a fixed order and takes the sequence's decisions (CG coefficients,
// stopping tests, Armijo, Gauss-Newton stop); after a second barrier every CTA
// reads the new states.  Results depend only on the launch shape, never on
// scheduling.  The decisions are those of the single-sequence path (the
// Gauss-Newton-PCG-Armijo reading of the GIR of Sec. 2): the same tests in the
// same order on the same kinds of totals.
//
// The grid barriers are the library's own and bounded: a CTA that waits for
// more than kBarrierNs sets bit 0 of *err and every CTA leaves; the host
// reports STML_ETIMEOUT.  (A cooperative launch makes all CTAs resident, so
// the bound only guards against a logic error.)
#include "../../include/stml.h"
#include "gn_items.cuh"
#include "kernels.h"

namespace stml {

namespace {

constexpr int kFG = kThreads / 32;                 // frame groups (warps) of an evaluation tile
constexpr unsigned long long kBarrierNs = 2000000000ull;   // 2 s
constexpr int kNV = 8;                             // values reduced per step: D, S, St, P, |w|^2, |g|^2, <g,d>, |d|^2

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier over all CTAs of a cooperative launch: an arrival count
// and a generation word (both zero at launch).  Returns false in every thread
// when the wait expired or another CTA reported an error.
__device__ bool batch_sync(BatchSync* bs, unsigned& gen, unsigned nblocks) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned want = gen + 1;
        __threadfence();
        if (atomicAdd(&bs->count, 1u) == nblocks - 1) {
            atomicExch(&bs->count, 0u);
            __threadfence();
            atomicExch(&bs->gen, want);
        } else {
            const unsigned long long t0 = global_ns();
            while (ld_acquire(&bs->gen) != want) {
                if (ld_acquire(&bs->err) != 0u) {
                    ok = 0;
                    break;
                }
                if (global_ns() - t0 > kBarrierNs) {
                    atomicOr(&bs->err, 1u);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        gen = want;
        s_ok = ok && ld_acquire(&bs->err) == 0u;
    }
    __syncthreads();
    return s_ok != 0;
}

// Bytes per pixel-frame a phase moves (for the CTA partition only).
__device__ __forceinline__ unsigned long long phase_cost(int ph) {
    switch (ph) {
        case BPH_EVAL0: return 60;
        case BPH_INIT: return 40;
        case BPH_APPLY: return 24;
        case BPH_UPDATE: return 56;
        case BPH_TRIAL: return 24;
        case BPH_GRAD: return 44;
        case BPH_LAND: return 24;
        default: return 0;
    }
}

// Objective and gradient of eq. (1) (distance, diffusion S, temporal term,
// penalty P) over one tile of 32 VEC consecutive pixels and all frames of K,
// at w = u + t d (d may be null).  A warp is a frame group (frames fg,
// fg + 8, ...), lanes hold VEC pixels each.
//   OBJ:  per-pixel frame means of a = T(x + w) and of w to abar / ubar;
//         sums D, S, St, P, |w|^2 (and <g, d>, |d|^2 with gdot).
//   GRAD: with abar / ubar of the same point: g, grad T (and w to wout);
//         sums |g|^2, |w|^2.
//   FULL: both, the means passed through shared memory.
enum EvalMode { EV_OBJ = 0, EV_GRAD = 1, EV_FULL = 2 };

// grad T in the image storage type (round to nearest even for 16-bit types).
template <typename TI, int VEC>
__device__ __forceinline__ void store_dT(void* dT, size_t i, const float (&v)[VEC]) {
    TI* p = static_cast<TI*>(dT) + i;
    if constexpr (VEC == 4)
        st4f(p, v);
    else
        stf(p, v[0]);
}

// Shared memory of an evaluation tile: per frame group and pixel the count,
// mean and squared deviations of a and the sums of w; the merged means.
template <int D, int VEC>
struct EvalSh {
    static constexpr int SEG = 32 * VEC;
    float mean[kFG][SEG], m2[kFG][SEG];
    float u[kFG][D][SEG];
    float n[kFG];
    float abar[SEG], ubar[D][SEG];
};

template <int D, int VEC, int MODE, typename TI>
__device__ __forceinline__ void eval_tile(const BatchSeq& b, const TI* __restrict__ T, unsigned tile,
                                          const float* __restrict__ u, const float* __restrict__ dvec, float t,
                                          const float* __restrict__ gdot, float* __restrict__ wout,
                                          EvalSh<D, VEC>& sh, float (&acc)[kNV]) {
    constexpr int SEG = 32 * VEC;
    auto& sh_mean = sh.mean;
    auto& sh_m2 = sh.m2;
    auto& sh_u = sh.u;
    auto& sh_n = sh.n;
    auto& sh_abar = sh.abar;
    auto& sh_ubar = sh.ubar;
    const Geom& g = b.g;
    const int lane = threadIdx.x & 31, fg = threadIdx.x >> 5;
    const size_t N = (size_t)g.N;
    const unsigned px = tile * SEG + (unsigned)lane * VEC;
    const bool valid = px < (unsigned)g.N;
    int x = 0, y = 0, z = 0;
    if (valid) pix_pos(b.pi, px, x, y, z);
    const int nK = b.fs.nK;
    const size_t sz = (size_t)g.nx * g.ny;
    auto ldw = [&](size_t i, float (&o)[VEC]) {
        V<VEC> a;
        a.load(u + i);
        if (dvec) {
            V<VEC> d;
            d.load(dvec + i);
#pragma unroll
            for (int e = 0; e < VEC; ++e) a.a[e] = fmaf(t, d.a[e], a.a[e]);
        }
#pragma unroll
        for (int e = 0; e < VEC; ++e) o[e] = a.a[e];
    };
    auto ldw1 = [&](size_t i) { return dvec ? fmaf(t, __ldg(dvec + i), __ldg(u + i)) : __ldg(u + i); };

    if constexpr (MODE != EV_GRAD) {
        float cnt = 0.f, sft[VEC], s1[VEC], s2[VEC], su[D][VEC];
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
            sft[e] = s1[e] = s2[e] = 0.f;
#pragma unroll
            for (int c = 0; c < D; ++c) su[c][e] = 0.f;
        }
        const float c_sx = 0.5f * b.cf.alpha_hd * b.cf.inv_h2;
        for (int j = fg; j < nK; j += kFG) {   // warp-uniform
            const TI* Tk = T + (size_t)__ldg(b.fs.frames + j) * N;
            float w[D][VEC];
#pragma unroll
            for (int c = 0; c < D; ++c) {
                if (valid) {
                    ldw(((size_t)j * D + c) * N + px, w[c]);
                } else {
#pragma unroll
                    for (int e = 0; e < VEC; ++e) w[c][e] = 0.f;
                }
            }
            if (gdot && valid) {
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    V<VEC> gv, dv;
                    gv.load(gdot + ((size_t)j * D + c) * N + px);
                    dv.load(dvec + ((size_t)j * D + c) * N + px);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) {
                        acc[6] = fmaf(gv.a[e], dv.a[e], acc[6]);
                        acc[7] = fmaf(dv.a[e], dv.a[e], acc[7]);
                    }
                }
            }
            float a[VEC];
            if constexpr (D == 2) {
                interp2_row<VEC>(Tk, g, x, y, w[0], w[1], a);   // every lane (invalid: pixel 0, zero field)
            } else {
#pragma unroll
                for (int e = 0; e < VEC; ++e) a[e] = interp3_val(Tk, g, x + e, y, z, w[0][e], w[1][e], w[2][e]);
            }
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const float right = __shfl_down_sync(0xffffffffu, w[c][0], 1);
                if (!valid) continue;
                const size_t base = ((size_t)j * D + c) * N + px;
                float fw = 0.f;
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    const float cc = w[c][e];
                    if (e + 1 < VEC) {
                        const float nb = w[c][e + 1 < VEC ? e + 1 : e];
                        fw = fmaf(nb - cc, nb - cc, fw);
                    } else if (x + VEC < g.nx) {
                        const float nb = lane < 31 ? right : ldw1(base + VEC);
                        fw = fmaf(nb - cc, nb - cc, fw);
                    }
                    su[c][e] += cc;
                    acc[4] = fmaf(cc, cc, acc[4]);
                }
                if (y + 1 < g.ny) {
                    float nb[VEC];
                    ldw(base + g.nx, nb);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) fw = fmaf(nb[e] - w[c][e], nb[e] - w[c][e], fw);
                }
                if constexpr (D == 3) {
                    if (z + 1 < g.nz) {
                        float nb[VEC];
                        ldw(base + sz, nb);
#pragma unroll
                        for (int e = 0; e < VEC; ++e) fw = fmaf(nb[e] - w[c][e], nb[e] - w[c][e], fw);
                    }
                }
                acc[1] = fmaf(c_sx, fw, acc[1]);
                if (b.cf.alphat_hd != 0.f && j + 1 < nK) {
                    const float cw = 0.5f * b.cf.alphat_hd * __ldg(b.fs.w_next + j);
                    float nt[VEC];
                    ldw(base + (size_t)D * N, nt);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) acc[2] = fmaf(cw * (nt[e] - w[c][e]), nt[e] - w[c][e], acc[2]);
                }
            }
            if (cnt == 0.f) {
#pragma unroll
                for (int e = 0; e < VEC; ++e) sft[e] = a[e];
            }
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                const float dl = a[e] - sft[e];
                s1[e] += dl;
                s2[e] = fmaf(dl, dl, s2[e]);
            }
            cnt += 1.f;
        }
        // frame-group statistics (count, mean, sum of squared deviations) per pixel
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
            const int k = lane * VEC + e;
            const float mean = cnt > 0.f ? sft[e] + s1[e] / cnt : 0.f;
            const float m2 = cnt > 0.f ? fmaxf(s2[e] - s1[e] * (s1[e] / cnt), 0.f) : 0.f;
            sh_mean[fg][k] = mean;
            sh_m2[fg][k] = m2;
#pragma unroll
            for (int c = 0; c < D; ++c) sh_u[fg][c][k] = su[c][e];
        }
        if (lane == 0) sh_n[fg] = cnt;
        __syncthreads();
        // merge the frame groups in group order (Chan's pairwise update)
        for (int k = threadIdx.x; k < SEG; k += blockDim.x) {
            const unsigned pp = tile * SEG + (unsigned)k;
            float n = 0.f, mean = 0.f, m2 = 0.f, us[D];
#pragma unroll
            for (int c = 0; c < D; ++c) us[c] = 0.f;
            for (int w = 0; w < kFG; ++w) {
                const float nb = sh_n[w];
                if (nb == 0.f) continue;
                const float mb = sh_mean[w][k], dlt = mb - mean, nn = n + nb;
                mean = fmaf(dlt, nb / nn, mean);
                m2 += sh_m2[w][k] + dlt * dlt * (n * nb / nn);
                n = nn;
#pragma unroll
                for (int c = 0; c < D; ++c) us[c] += sh_u[w][c][k];
            }
            float pn = 0.f;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                us[c] *= b.cf.inv_nK;
                pn = fmaf(us[c], us[c], pn);
            }
            sh_abar[k] = mean;
#pragma unroll
            for (int c = 0; c < D; ++c) sh_ubar[c][k] = us[c];
            if (pp < (unsigned)g.N) {
                acc[0] = fmaf(b.cf.half_hd, m2, acc[0]);
                acc[3] = fmaf(b.cf.lam_hd, pn, acc[3]);
                b.abar[pp] = mean;
#pragma unroll
                for (int c = 0; c < D; ++c) b.ubar[(size_t)c * N + pp] = us[c];
            }
        }
        __syncthreads();
    }
    if constexpr (MODE != EV_OBJ) {
        float ab[VEC], ub[D][VEC];
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
            const int k = lane * VEC + e;
            if (MODE == EV_FULL) {
                ab[e] = sh_abar[k];
#pragma unroll
                for (int c = 0; c < D; ++c) ub[c][e] = sh_ubar[c][k];
            } else {
                ab[e] = valid ? __ldcg(b.abar + px + e) : 0.f;
#pragma unroll
                for (int c = 0; c < D; ++c) ub[c][e] = valid ? __ldcg(b.ubar + (size_t)c * N + px + e) : 0.f;
            }
        }
        const float lap_c = b.cf.alpha_hd * b.cf.inv_h2;
        for (int j = fg; j < nK; j += kFG) {   // warp-uniform
            const TI* Tk = T + (size_t)__ldg(b.fs.frames + j) * N;
            const float w_next = (b.cf.alphat_hd != 0.f && j + 1 < nK) ? __ldg(b.fs.w_next + j) : 0.f;
            const float w_prev = (b.cf.alphat_hd != 0.f && j > 0) ? __ldg(b.fs.w_next + j - 1) : 0.f;
            float w[D][VEC];
#pragma unroll
            for (int c = 0; c < D; ++c) {
                if (valid) {
                    ldw(((size_t)j * D + c) * N + px, w[c]);
                } else {
#pragma unroll
                    for (int e = 0; e < VEC; ++e) w[c][e] = 0.f;
                }
            }
            float a[VEC], dt[D][VEC];
            if constexpr (D == 2) {
                interp2_row_grad<VEC>(Tk, g, x, y, w[0], w[1], a, dt[0], dt[1]);
            } else {
#pragma unroll
                for (int e = 0; e < VEC; ++e) interp3(Tk, g, x + e, y, z, w[0][e], w[1][e], w[2][e], a[e], dt[0][e],
                                                      dt[1][e], dt[2][e]);
            }
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const float up_l = __shfl_up_sync(0xffffffffu, w[c][VEC - 1], 1);
                const float dn_r = __shfl_down_sync(0xffffffffu, w[c][0], 1);
                if (!valid) continue;
                const size_t base = ((size_t)j * D + c) * N + px;
                float left = 0.f, right = 0.f;
                if (x > 0) left = lane > 0 ? up_l : ldw1(base - 1);
                if (x + VEC < g.nx) right = lane < 31 ? dn_r : ldw1(base + VEC);
                float lap[VEC];
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    const float le = e == 0 ? left : w[c][e > 0 ? e - 1 : 0];
                    const float re = e == VEC - 1 ? right : w[c][e + 1 < VEC ? e + 1 : e];
                    float lp = 0.f;
                    if (x + e > 0) lp += w[c][e] - le;
                    if (x + e < g.nx - 1) lp += w[c][e] - re;
                    lap[e] = lp;
                }
                float nb[VEC];
                if (y > 0) {
                    ldw(base - g.nx, nb);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) lap[e] += w[c][e] - nb[e];
                }
                if (y < g.ny - 1) {
                    ldw(base + g.nx, nb);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) lap[e] += w[c][e] - nb[e];
                }
                if constexpr (D == 3) {
                    if (z > 0) {
                        ldw(base - sz, nb);
#pragma unroll
                        for (int e = 0; e < VEC; ++e) lap[e] += w[c][e] - nb[e];
                    }
                    if (z < g.nz - 1) {
                        ldw(base + sz, nb);
#pragma unroll
                        for (int e = 0; e < VEC; ++e) lap[e] += w[c][e] - nb[e];
                    }
                }
                float tg[VEC];
#pragma unroll
                for (int e = 0; e < VEC; ++e) tg[e] = 0.f;
                if (w_next != 0.f) {
                    ldw(base + (size_t)D * N, nb);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) tg[e] += w_next * (w[c][e] - nb[e]);
                }
                if (w_prev != 0.f) {
                    ldw(base - (size_t)D * N, nb);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) tg[e] += w_prev * (w[c][e] - nb[e]);
                }
                float gv[VEC];
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    const float r = a[e] - ab[e];
                    gv[e] = fmaf(b.cf.hd * r, dt[c][e],
                                 fmaf(lap_c, lap[e], fmaf(b.cf.alphat_hd, tg[e], b.cf.pen_g * ub[c][e])));
                    acc[5] = fmaf(gv[e], gv[e], acc[5]);
                    if (MODE == EV_GRAD) acc[4] = fmaf(w[c][e], w[c][e], acc[4]);
                }
                V<VEC> o;
#pragma unroll
                for (int e = 0; e < VEC; ++e) o.a[e] = gv[e];
                o.store(b.grad + base);
                if (wout) {
#pragma unroll
                    for (int e = 0; e < VEC; ++e) o.a[e] = w[c][e];
                    o.store(wout + base);
                }
                store_dT<TI, VEC>(b.dT, base, dt[c]);
            }
        }
    }
}

// ------------------------------------------------------------- decisions
__device__ __forceinline__ double tot_val(const dfloat& v) { return (double)v.hi + (double)v.lo; }

// Gauss-Newton stopping tests at the current iterate (those of the
// single-sequence GIR, in the same order).
__device__ __forceinline__ bool gn_stop(BatchState& S, const BatchCtl& c) {
    if (!isfinite(S.J) || !isfinite(S.gnorm2)) {
        S.status = STML_ENONFINITE;
        return true;
    }
    const double gnorm = sqrt(S.gnorm2);
    if (S.it > 0) {
        const bool c1 = fabs(S.Jold - S.J) <= c.tol_J * (1.0 + fabs(S.J0));
        const bool c2 = S.step <= c.tol_Y * (1.0 + sqrt(S.unorm2));
        const bool c3 = gnorm <= c.tol_G * (1.0 + fabs(S.J0));
        if (c1 && c2 && c3) return true;
    }
    return gnorm <= c.g_abs * (1.0 + fabs(S.J0)) || S.it >= c.max_gn;
}

__device__ __forceinline__ CgState cg_of(const BatchState& S) {
    CgState c;
    c.rho = S.cg_rho;
    c.bnorm2 = S.cg_bnorm2;
    c.rnorm2 = S.cg_rnorm2;
    c.pq = S.cg_pq;
    c.alpha = S.cg_alpha;
    c.beta = S.cg_beta;
    c.iter = S.cg_iter;
    c.flag = S.cg_flag;
    c.active = S.cg_active;
    return c;
}

__device__ __forceinline__ void cg_put(BatchState& S, const CgState& c) {
    S.cg_rho = c.rho;
    S.cg_bnorm2 = c.bnorm2;
    S.cg_rnorm2 = c.rnorm2;
    S.cg_pq = c.pq;
    S.cg_alpha = c.alpha;
    S.cg_beta = c.beta;
    S.cg_iter = c.iter;
    S.cg_flag = c.flag;
    S.cg_active = c.active;
}

// The end of a PCG solve: its steps count, the line search starts at t = 1.
__device__ __forceinline__ void to_trials(BatchState& S) {
    S.cg_total += S.cg_iter;
    S.ls_k = 0;
    S.t = 1.0f;
    S.phase = BPH_TRIAL;
}

// The decisions of one sequence after a step, from its reduced totals (one thread).
__device__ void decide(BatchState& S, const dfloat (&tot)[kNV], const BatchCtl& c, const BatchSeq& b) {
    switch (S.phase) {
        case BPH_EVAL0: {
            S.D = tot_val(tot[0]);
            S.S = tot_val(tot[1]) + tot_val(tot[2]);
            S.P = tot_val(tot[3]);
            S.J = S.J0 = S.D + S.S + S.P;
            S.unorm2 = tot_val(tot[4]);
            S.gnorm2 = tot_val(tot[5]);
            if (b.target > 0.0 && S.J0 <= b.target) S.phase = BPH_DONE;   // at the target already
            else S.phase = gn_stop(S, c) ? BPH_DONE : BPH_INIT;
            break;
        }
        case BPH_INIT: {
            CgState cs{};
            cg_after_init(cs, tot[0].hi + tot[0].lo, tot[1].hi + tot[1].lo, c.max_cg);
            cg_put(S, cs);
            S.cg_k = 0;
            S.dir_p0 = 0;
            if (cs.active) S.phase = BPH_APPLY;
            else to_trials(S);
            break;
        }
        case BPH_APPLY: {
            CgState cs = cg_of(S);
            cg_after_apply(cs, tot[0].hi + tot[0].lo);
            cg_put(S, cs);
            if (cs.active) {
                S.phase = BPH_UPDATE;
            } else {   // breakdown: the iterate so far, or p_0 if it was the first step
                S.dir_p0 = cs.iter == 0 ? 1 : 0;
                to_trials(S);
            }
            break;
        }
        case BPH_UPDATE: {
            CgState cs = cg_of(S);
            cg_after_update(cs, tot[0].hi + tot[0].lo, tot[1].hi + tot[1].lo, c.tol_cg, c.max_cg);
            cg_put(S, cs);
            if (cs.active) {
                S.cg_k += 1;
                S.phase = BPH_APPLY;
            } else {
                to_trials(S);
            }
            break;
        }
        case BPH_TRIAL: {
            const double Dv = tot_val(tot[0]), Sx = tot_val(tot[1]), St = tot_val(tot[2]), Pv = tot_val(tot[3]);
            const double Jt = Dv + Sx + St + Pv;
            S.ls_total += 1;
            if (S.ls_k == 0) {
                S.gTd = tot_val(tot[6]);
                S.dnorm2 = tot_val(tot[7]);
                if (!(S.gTd < 0.0)) {
                    S.status = STML_EBREAKDOWN;
                    S.phase = BPH_DONE;
                    break;
                }
            }
            if (Jt <= S.J + c.armijo_c * (double)S.t * S.gTd) {
                S.Jt = Jt;
                S.Dt = Dv;
                S.St = Sx + St;
                S.Pt = Pv;
                S.phase = BPH_GRAD;
                if (b.target > 0.0 && Jt <= b.target) {
                    // the step crosses the target: regula falsi (Illinois) on its length
                    S.la = 0.0;
                    S.lfa = S.J - b.target;
                    S.lb = (double)S.t;
                    S.lfb = Jt - b.target;
                    S.side = 0;
                    S.land_it = 0;
                    S.best_t = S.lb;
                    S.best_f = fabs(S.lfb);
                    S.best_J = Jt;
                    S.best_D = Dv;
                    S.best_S = Sx + St;
                    S.best_P = Pv;
                    S.land_final = 1;
                    if (S.best_f > b.target_tol * b.target) {
                        S.t = (float)((S.la * S.lfb - S.lb * S.lfa) / (S.lfb - S.lfa));
                        S.phase = BPH_LAND;
                    }
                }
            } else if (S.ls_k + 1 < c.max_ls) {
                S.ls_k += 1;
                S.t = ldexpf(1.0f, -S.ls_k);
            } else {
                S.status = STML_ELINESEARCH;
                S.phase = BPH_DONE;
            }
            break;
        }
        case BPH_LAND: {
            const double Dv = tot_val(tot[0]), Sx = tot_val(tot[1]), St = tot_val(tot[2]), Pv = tot_val(tot[3]);
            const double Jt = Dv + Sx + St + Pv, ft = Jt - b.target, tv = (double)S.t;
            S.land_it += 1;   // (not an Armijo trial: not counted in ls_total)
            if (fabs(ft) < S.best_f) {
                S.best_f = fabs(ft);
                S.best_t = tv;
                S.best_J = Jt;
                S.best_D = Dv;
                S.best_S = Sx + St;
                S.best_P = Pv;
            }
            if (S.best_f <= b.target_tol * b.target || S.land_it >= 40) {
                S.Jt = S.best_J;
                S.Dt = S.best_D;
                S.St = S.best_S;
                S.Pt = S.best_P;
                // the gradient pass needs the per-pixel means of the landed point:
                // evaluate it once more unless it was the last point evaluated
                if ((float)S.best_t == S.t) {
                    S.phase = BPH_GRAD;
                } else {
                    S.t = (float)S.best_t;
                    S.best_f = -1.0;   // the next evaluation is the final one
                }
                break;
            }
            if (ft > 0.0) {
                S.la = tv;
                S.lfa = ft;
                if (S.side == 1) S.lfb *= 0.5;
                S.side = 1;
            } else {
                S.lb = tv;
                S.lfb = ft;
                if (S.side == -1) S.lfa *= 0.5;
                S.side = -1;
            }
            S.t = (float)((S.la * S.lfb - S.lb * S.lfa) / (S.lfb - S.lfa));
            break;
        }
        case BPH_GRAD: {
            S.cur ^= 1;
            S.step = (double)S.t * sqrt(S.dnorm2);
            S.Jold = S.J;
            S.J = S.Jt;
            S.D = S.Dt;
            S.S = S.St;
            S.P = S.Pt;
            S.it += 1;
            S.gnorm2 = tot_val(tot[5]);
            S.unorm2 = tot_val(tot[4]);
            if (S.land_final) S.phase = BPH_DONE;   // the target is reached
            else S.phase = gn_stop(S, c) ? BPH_DONE : BPH_INIT;
            break;
        }
        default:
            break;
    }
}

// ------------------------------------------------------------- the kernel
template <int D, int VEC, int TPR, typename TI>
__global__ void __launch_bounds__(kThreads)
batch_gir_kernel(const BatchSeq* __restrict__ seqs, int nseq, BatchState* st, BatchCtl ctl, float2* part,
                 BatchSync* bs, int max_steps) {
    __shared__ int s_seq, s_first, s_count, s_any;
    // the evaluation tiles and the PCG tiles run in different phases
    __shared__ union {
        EvalSh<D, VEC> ev;
        float tile[(kThreads / TPR) * (1 + D) * TPR * VEC];
    } sh;
    float* tile_sh = sh.tile;
    unsigned gen = 0;
    int step = 0;
    for (; step < max_steps; ++step) {
        // the CTA ranges of this step: one per active sequence, at least one
        // CTA each, the rest in proportion to the bytes of its phase
        if (threadIdx.x == 0) {
            const unsigned G = gridDim.x;
            unsigned long long W = 0;
            unsigned A = 0;
            for (int s = 0; s < nseq; ++s) {
                const int ph = __ldcg(&st[s].phase);
                if (ph == BPH_DONE) continue;
                ++A;
                W += phase_cost(ph) * (unsigned long long)seqs[s].g.N * (unsigned long long)seqs[s].fs.nK;
            }
            s_any = A > 0;
            s_seq = -1;
            s_first = 0;
            s_count = 0;
            if (A > 0 && A <= G) {
                const unsigned R = G - A;
                unsigned given = 0, first = 0;
                unsigned extra_left = R;
                // extra CTAs: floor of the proportional share; the remainder
                // goes to the first active sequences in order
                for (int s = 0; s < nseq; ++s) {
                    const int ph = __ldcg(&st[s].phase);
                    if (ph == BPH_DONE) continue;
                    const unsigned long long w =
                        phase_cost(ph) * (unsigned long long)seqs[s].g.N * (unsigned long long)seqs[s].fs.nK;
                    given += W ? (unsigned)((unsigned long long)R * w / W) : 0u;
                }
                extra_left = R - given;
                for (int s = 0; s < nseq; ++s) {
                    const int ph = __ldcg(&st[s].phase);
                    if (ph == BPH_DONE) continue;
                    const unsigned long long w =
                        phase_cost(ph) * (unsigned long long)seqs[s].g.N * (unsigned long long)seqs[s].fs.nK;
                    unsigned n = 1u + (W ? (unsigned)((unsigned long long)R * w / W) : 0u);
                    if (extra_left > 0) {
                        ++n;
                        --extra_left;
                    }
                    if (blockIdx.x >= first && blockIdx.x < first + n) {
                        s_seq = s;
                        s_first = (int)first;
                        s_count = (int)n;
                    }
                    first += n;
                }
            } else if (A > G) {
                atomicOr(&bs->err, 2u);   // more sequences than CTAs: refused by the host, never reached
                s_any = 0;
            }
        }
        __syncthreads();
        if (!s_any) break;
        float acc[kNV];
#pragma unroll
        for (int i = 0; i < kNV; ++i) acc[i] = 0.f;
        const int s = s_seq;
        if (s >= 0) {
            const BatchSeq& b = seqs[s];
            const TI* T = static_cast<const TI*>(b.T);
            const int ph = __ldcg(&st[s].phase);
            const int cur = __ldcg(&st[s].cur);
            const unsigned li = blockIdx.x - (unsigned)s_first, ns = (unsigned)s_count;
            const TI* dT = static_cast<const TI*>(b.dT);
            if (ph == BPH_EVAL0) {
                for (unsigned t = li; t < b.eval_tiles; t += ns)
                    eval_tile<D, VEC, EV_FULL, TI>(b, T, t, b.u[cur], nullptr, 0.f, nullptr, nullptr, sh.ev, acc);
            } else if (ph == BPH_INIT) {
                float rz = 0.f, rr = 0.f;
                for (unsigned t = li; t < b.pcg_tiles; t += ns)
                    tile_pass<D, VEC, TILE_INIT, TPR, TI>(b.g, b.pi, b.fs, b.cf, dT, b.z, b.r, b.grad, b.x, nullptr,
                                                         nullptr, 0.f, 0.f, b.ms_z, b.sv_z, t, tile_sh, rz, rr);
                acc[0] = rz;
                acc[1] = rr;
            } else if (ph == BPH_APPLY) {
                const int k = __ldcg(&st[s].cg_k);
                const float beta = __ldcg(&st[s].cg_beta);
                const int c0 = k & 1, c1 = c0 ^ 1;
                const DirSrc src{b.z, k > 0 ? b.p[c1] : nullptr, beta, b.p[c0], b.ms_z, b.sv_z,
                                 b.ms_p[c1], b.sv_p[c1], b.ms_p[c0], b.sv_p[c0]};
                float pq = 0.f;
                for (unsigned it = li; it < b.chunks; it += ns) {
                    const unsigned j = b.cpf.div(it);
                    apply_item<D, VEC, true, TI>(b.g, b.pi, b.fs, b.cf, dT, src, b.q, (int)j, it - j * b.cpf.d, pq);
                }
                acc[0] = pq;
            } else if (ph == BPH_UPDATE) {
                const int k = __ldcg(&st[s].cg_k);
                const float al = __ldcg(&st[s].cg_alpha);
                float rz = 0.f, rr = 0.f;
                for (unsigned t = li; t < b.pcg_tiles; t += ns)
                    tile_pass<D, VEC, TILE_UPDATE, TPR, TI>(b.g, b.pi, b.fs, b.cf, dT, b.z, b.r, nullptr, b.x,
                                                           b.p[k & 1], b.q, al, 0.f, b.ms_z, b.sv_z, t, tile_sh, rz,
                                                           rr);
                acc[0] = rz;
                acc[1] = rr;
            } else if (ph == BPH_TRIAL || ph == BPH_GRAD || ph == BPH_LAND) {
                const float tt = __ldcg(&st[s].t);
                const float* dir = __ldcg(&st[s].dir_p0) ? b.p[0] : b.x;
                if (ph != BPH_GRAD) {
                    const float* gd = (ph == BPH_TRIAL && __ldcg(&st[s].ls_k) == 0) ? b.grad : nullptr;
                    for (unsigned t = li; t < b.eval_tiles; t += ns)
                        eval_tile<D, VEC, EV_OBJ, TI>(b, T, t, b.u[cur], dir, tt, gd, nullptr, sh.ev, acc);
                } else {
                    for (unsigned t = li; t < b.eval_tiles; t += ns)
                        eval_tile<D, VEC, EV_GRAD, TI>(b, T, t, b.u[cur], dir, tt, nullptr, b.u[cur ^ 1], sh.ev,
                                                        acc);
                }
            }
        }
        cta_partials<kNV>(acc, part, blockIdx.x);
        if (!batch_sync(bs, gen, gridDim.x)) break;   // every item of the step is complete
        if (s >= 0 && (int)blockIdx.x == s_first) {
            dfloat tot[kNV];
            cta_total<kNV>(part + (size_t)s_first * kNV, (unsigned)s_count, tot);
            if (threadIdx.x == 0) {
                // the state was written by the previous step's leader, maybe on
                // another SM: read it from L2, word by word
                static_assert(sizeof(BatchState) % 4 == 0, "whole words");
                BatchState S;
                const unsigned* src = reinterpret_cast<const unsigned*>(st + s);
                unsigned* dst = reinterpret_cast<unsigned*>(&S);
                for (int w = 0; w < (int)(sizeof(BatchState) / 4); ++w) dst[w] = __ldcg(src + w);
                decide(S, tot, ctl, seqs[s]);
                st[s] = S;
                __threadfence();
            }
        }
        if (!batch_sync(bs, gen, gridDim.x)) break;   // every decision of the step is visible
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        bs->steps = (unsigned)step;
        if (step >= max_steps) atomicOr(&bs->err, 4u);   // the step budget ran out
    }
}

// One CTA enters a barrier that expects two: nothing else arrives, so the
// wait must give up after its bound and report it (*expired = 1).
__global__ void barrier_probe_kernel(BatchSync* bs, int* expired) {
    unsigned gen = 0;
    const bool ok = batch_sync(bs, gen, 2u);
    if (threadIdx.x == 0) *expired = (!ok && (ld_acquire(&bs->err) & 1u)) ? 1 : 0;
}

template <int D, int VEC, int TPR, typename TI>
const void* batch_kernel_ptr() {
    return reinterpret_cast<const void*>(batch_gir_kernel<D, VEC, TPR, TI>);
}

template <typename F>
auto with_batch_kernel(int d, int vec, int tpr, int img_type, F&& f) {
    return with_store_type(img_type, [&](auto tag) {
        using TI = decltype(tag);
        if (d == 2) {
            if (vec == 4) return tpr == 16 ? f(batch_kernel_ptr<2, 4, 16, TI>()) : f(batch_kernel_ptr<2, 4, 4, TI>());
            return tpr == 16 ? f(batch_kernel_ptr<2, 1, 16, TI>()) : f(batch_kernel_ptr<2, 1, 4, TI>());
        }
        if (vec == 4) return tpr == 16 ? f(batch_kernel_ptr<3, 4, 16, TI>()) : f(batch_kernel_ptr<3, 4, 4, TI>());
        return tpr == 16 ? f(batch_kernel_ptr<3, 1, 16, TI>()) : f(batch_kernel_ptr<3, 1, 4, TI>());
    });
}

}  // namespace

size_t batch_partials(int ctas) { return (size_t)ctas * kNV; }

cudaError_t launch_batch_barrier_probe(BatchSync* sync, int* expired, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(sync, 0, sizeof(BatchSync), s);
    if (e != cudaSuccess) return e;
    barrier_probe_kernel<<<1, 32, 0, s>>>(sync, expired);
    count_launches(1);
    return cudaGetLastError();
}

int batch_grid(int d, int vec, int img_type, const BatchShape& sh) {
    const int sms = device_sms();
    if (sms <= 0) return 0;
    return with_batch_kernel(d, vec, sh.tpr, img_type, [&](const void* k) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, 0) != cudaSuccess) return 0;
        const int n = per_sm < sh.ctas_per_sm ? per_sm : sh.ctas_per_sm;
        return n > 0 ? n * sms : 0;
    });
}

cudaError_t launch_batch_gir(const BatchSeq* seqs_dev, int nseq, BatchState* states, const BatchCtl& ctl, int d,
                             int vec, int img_type, const BatchShape& sh, float2* part, BatchSync* sync,
                             int max_steps, cudaStream_t s) {
    const int grid = batch_grid(d, vec, img_type, sh);
    if (grid <= 0 || nseq < 1 || nseq > grid) return cudaErrorInvalidConfiguration;
    return with_batch_kernel(d, vec, sh.tpr, img_type, [&](const void* k) {
        const BatchSeq* a0 = seqs_dev;
        int a1 = nseq;
        BatchState* a2 = states;
        BatchCtl a3 = ctl;
        float2* a4 = part;
        BatchSync* a5 = sync;
        int a6 = max_steps;
        void* args[] = {(void*)&a0, &a1, &a2, &a3, &a4, &a5, &a6};
        const cudaError_t e = cudaLaunchCooperativeKernel(k, dim3((unsigned)grid), dim3(kThreads), args, 0, s);
        count_launches(1);
        return e;
    });
}

}  // namespace stml
