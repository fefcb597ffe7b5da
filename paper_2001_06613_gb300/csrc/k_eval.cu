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
#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>

#include "kernels.h"

namespace cg = cooperative_groups;

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

template <int D, typename TI>
__device__ __forceinline__ void interp(const TI* __restrict__ Tk, const Geom& g, int x, int y, int z,
                                       const float (&u)[D], float& a, float (&gr)[D]) {
    if constexpr (D == 2)
        interp2(Tk, g, x, y, u[0], u[1], a, gr[0], gr[1]);
    else
        interp3(Tk, g, x, y, z, u[0], u[1], u[2], a, gr[0], gr[1], gr[2]);
}

}  // namespace

// ----------------------------------------------------------------- objective
// Reduced values: 0 D, 1 S_x, 2 S_t, 3 P, 4 (unused), 5 |u|^2; with GDOT also
// 6 <gdot, du> and 7 |du|^2 (the directional derivative of the Gauss-Newton
// step).  Fields are read as u + t du when TRIAL.
//
// A CTA covers a run of SEG = 32 VEC pixels of one image row with FG warps;
// lane l owns the VEC pixels p0 + VEC l ...  The frames are dealt to frame
// groups: warp w of split r (blockIdx.y) takes j = r FG + w, j + FG S, ...,
// with the field of its next frame loaded while the current one is used.
// Per pixel a warp keeps shifted sums of a_k - s (s = its first a_k), which
// give the mean and the sum of squared deviations at the end; the FG warps
// of a CTA are merged in shared memory by a pairwise tree (Chan's update),
// and the S splits of a run form one thread-block cluster whose rank 0
// merges the others' results through distributed shared memory, in rank
// order.
namespace {

// Resident CTAs per SM the objective kernel is compiled for (register cap).
constexpr int obj_min_blocks(int d, int vec) { return vec == 4 || (d == 3 && vec == 2) ? 2 : 3; }

template <int VEC>
__device__ __forceinline__ void ldv(const float* __restrict__ q, size_t i, float (&o)[VEC]) {
    if constexpr (VEC == 4) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(q + i));
        o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
    } else if constexpr (VEC == 2) {
        const float2 a = __ldg(reinterpret_cast<const float2*>(q + i));
        o[0] = a.x; o[1] = a.y;
    } else {
        o[0] = __ldg(q + i);
    }
}

// A hint to fetch the line holding p into L2 (no register is written, so
// nothing waits for it); p must lie inside an allocation.
__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// VEC consecutive floats from shared memory, aligned to 4 VEC bytes.
template <int VEC>
__device__ __forceinline__ void lds_vec(const float* p, float (&o)[VEC]) {
    if constexpr (VEC == 4) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        o[0] = q.x; o[1] = q.y; o[2] = q.z; o[3] = q.w;
    } else if constexpr (VEC == 2) {
        const float2 q = *reinterpret_cast<const float2*>(p);
        o[0] = q.x; o[1] = q.y;
    } else {
        o[0] = p[0];
    }
}

// The field of one frame at a thread's pixels: the pixels, the next row, the
// next plane (3-D) and, in lane 31, the first pixel of the next run.
template <int D, int VEC, bool TRIAL>
struct FrameU {
    float c[D][VEC], ny[D][VEC], nz[D == 3 ? D : 1][VEC], tail[D];

    __device__ __forceinline__ static void ld(const float* __restrict__ u, const float* __restrict__ du, float t,
                                              size_t i, float (&o)[VEC]) {
        ldv<VEC>(u, i, o);
        if constexpr (TRIAL) {
            float d[VEC];
            ldv<VEC>(du, i, d);
#pragma unroll
            for (int e = 0; e < VEC; ++e) o[e] = fmaf(t, d[e], o[e]);
        }
    }
    __device__ __forceinline__ void load(const float* __restrict__ u, const float* __restrict__ du, float t,
                                         size_t b, size_t N, int nx, size_t sz, bool valid, bool has_y,
                                         bool has_z, bool has_tail) {
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const size_t bk = b + (size_t)k * N;
#pragma unroll
            for (int e = 0; e < VEC; ++e) c[k][e] = ny[k][e] = 0.f;
            if (valid) ld(u, du, t, bk, c[k]);
            if (has_y) ld(u, du, t, bk + nx, ny[k]);
            if constexpr (D == 3) {
#pragma unroll
                for (int e = 0; e < VEC; ++e) nz[k][e] = 0.f;
                if (has_z) ld(u, du, t, bk + sz, nz[k]);
            }
            tail[k] = has_tail ? (TRIAL ? fmaf(t, __ldg(du + bk + VEC), __ldg(u + bk + VEC)) : __ldg(u + bk + VEC))
                               : 0.f;
        }
    }
};

// One stage of the 2-D objective pass's copy ring (floats, per warp): for u
// (and du in a trial) and each component, the run of 32 VEC pixels and the
// run one row below; then the first pixel of the next run (lane 31).
constexpr int kObjStages = 3;
template <int D, int VEC, bool TRIAL>
struct ObjStage {
    static constexpr int kSrc = TRIAL ? 2 : 1;
    static constexpr int kRow = 32 * VEC;
    static constexpr int kRows = kSrc * D * 2 * kRow;
    static constexpr int floats = kRows + ((kSrc * D + 3) / 4) * 4;
    static constexpr size_t ring_bytes = (size_t)(kThreads / 32) * kObjStages * floats * sizeof(float);
};

}  // namespace

template <int D, int VEC, bool TRIAL, bool GDOT, typename TI>
__global__ void __launch_bounds__(kThreads, obj_min_blocks(D, VEC))
obj_kernel(const TI* __restrict__ T, Geom g, PixIndex pi, FrameSet fs, Coef cf, const float* __restrict__ u,
           const float* __restrict__ du, float t, const float* __restrict__ gdot, float* __restrict__ abar,
           float* __restrict__ ubar, double* __restrict__ partials, unsigned int* ticket, double* out,
           LineSearchArgs ls) {
    pdl_enter();
    // a later Armijo trial has nothing to do once an earlier one decided
    if (ls.S && ls.k > 0 && (ls.S->ls_accepted || ls.S->ls_nodescent)) return;
    constexpr int FG = kThreads / 32, SEG = 32 * VEC;
    __shared__ float sh_m[FG][SEG], sh_q[FG][SEG];
    __shared__ float sh_u[FG][D][SEG];
    __shared__ float sh_n[FG];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int S = (int)gridDim.y, TG = FG * S;
    const unsigned p0 = blockIdx.x * SEG, p = p0 + (unsigned)lane * VEC;
    const size_t N = (size_t)g.N;
    const size_t sz = (size_t)g.nx * g.ny;
    const bool valid = p < (unsigned)g.N;
    int x = 0, y = 0, z = 0;
    if (valid) pos_of(pi, p, x, y, z);
    // rows hold a multiple of VEC pixels, so only the last pixel of a thread
    // can have its x + 1 neighbour outside the row
    const bool has_y = valid && y + 1 < g.ny, has_z = valid && D == 3 && z + 1 < g.nz;
    const bool has_xl = valid && x + VEC < g.nx;
    const bool has_tail = lane == 31 && has_xl;

    float cnt = 0.f, sft[VEC], s1[VEC], s2[VEC], su[D][VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
        sft[e] = s1[e] = s2[e] = 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) su[k][e] = 0.f;
    }
    float sx = 0.f, st = 0.f, u2 = 0.f, gd = 0.f, dd = 0.f;
    const float c_sx = 0.5f * cf.alpha_hd * cf.inv_h2;
    const int j0 = (int)blockIdx.y * FG + w;
    if constexpr (GDOT) {
        if (valid) {
            for (int j = j0; j < fs.nK; j += TG) {
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    const size_t b = ((size_t)j * D + k) * N + p;
                    float gv[VEC], dv[VEC];
                    ldv<VEC>(gdot, b, gv);
                    ldv<VEC>(du, b, dv);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) {
                        gd = fmaf(gv[e], dv[e], gd);
                        dd = fmaf(dv[e], dv[e], dd);
                    }
                }
            }
        }
    }
    // the work on frame j (field `cur`, image number fr): warped image,
    // forward-difference energy, temporal term, sums
    auto consume = [&](const FrameU<D, VEC, TRIAL>& cur, int j, int fr) {
        // every gather is unconditional (clamped addresses; invalid lanes
        // sample pixel 0 with a zero field)
        const TI* Tk = T + (size_t)fr * N;
        float a[VEC];
        if constexpr (D == 2) {
            interp2_row<VEC>(Tk, g, x, y, cur.c[0], cur.c[1], a);
        } else {
#pragma unroll
            for (int e = 0; e < VEC; ++e)
                a[e] = interp3_val(Tk, g, x + e, y, z, cur.c[0][e], cur.c[1][e], cur.c[2][e]);
        }
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const float right = __shfl_down_sync(0xffffffffu, cur.c[k][0], 1);
            const float xl = lane < 31 ? right : cur.tail[k];
            float fw = 0.f;
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                const float cc = cur.c[k][e];
                if (e + 1 < VEC || has_xl) {
                    const float nb = e + 1 < VEC ? cur.c[k][(e + 1) % VEC] : xl;
                    fw = fmaf(nb - cc, nb - cc, fw);
                }
                if (has_y) fw = fmaf(cur.ny[k][e] - cc, cur.ny[k][e] - cc, fw);
                if constexpr (D == 3)
                    if (has_z) fw = fmaf(cur.nz[k][e] - cc, cur.nz[k][e] - cc, fw);
                su[k][e] += cc;
                u2 = fmaf(cc, cc, u2);
            }
            sx = fmaf(c_sx, valid ? fw : 0.f, sx);
            if (cf.alphat_hd != 0.f && j + 1 < fs.nK && valid) {
                const float cw = 0.5f * cf.alphat_hd * __ldg(fs.w_next + j);
                float nt[VEC];
                FrameU<D, VEC, TRIAL>::ld(u, du, t, ((size_t)(j + 1) * D + k) * N + p, nt);
#pragma unroll
                for (int e = 0; e < VEC; ++e) st = fmaf(cw * (nt[e] - cur.c[k][e]), nt[e] - cur.c[k][e], st);
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
    };
    if constexpr (D == 2) {
        // Each lane copies its own pieces of the fields of its next frames
        // into this warp's ring of kObjStages stages with cp.async (one commit
        // group per frame) and reads back only what it copied, so many loads
        // are in flight without holding registers and no barrier is needed.
        using STG = ObjStage<D, VEC, TRIAL>;
        extern __shared__ float4 obj_ring4[];
        float* ring = reinterpret_cast<float*>(obj_ring4) + (size_t)w * kObjStages * STG::floats;
        auto issue = [&](int jj, int stage) {
            float* b = ring + stage * STG::floats;
#pragma unroll
            for (int src = 0; src < STG::kSrc; ++src) {
                const float* arr = src ? du : u;
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    const float* gk = arr + ((size_t)jj * D + k) * N + p;
                    float* rk = b + ((src * D + k) * 2) * STG::kRow + lane * VEC;
                    if (valid) cp_async<4 * VEC>(rk, gk);
                    if (has_y) cp_async<4 * VEC>(rk + STG::kRow, gk + g.nx);
                    if (has_tail) cp_async<4>(b + STG::kRows + src * D + k, gk + VEC);
                }
            }
        };
        auto read = [&](int stage, FrameU<D, VEC, TRIAL>& cur) {
            const float* b = ring + stage * STG::floats;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const float* r0 = b + (k * 2) * STG::kRow + lane * VEC;
                const float* r1 = b + ((STG::kSrc - 1) * D + k) * 2 * STG::kRow + lane * VEC;   // du rows
                // one vector load per row piece (a lane's VEC floats are
                // contiguous and aligned): scalar loads at a lane stride of
                // VEC words would conflict on the banks; slots a lane did not
                // copy are read but not used
                float c0[VEC], n0[VEC], c1[VEC], n1[VEC];
                lds_vec<VEC>(r0, c0);
                lds_vec<VEC>(r0 + STG::kRow, n0);
                if constexpr (TRIAL) {
                    lds_vec<VEC>(r1, c1);
                    lds_vec<VEC>(r1 + STG::kRow, n1);
                }
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    float cv = valid ? c0[e] : 0.f, nv = has_y ? n0[e] : 0.f;
                    if constexpr (TRIAL) {
                        if (valid) cv = fmaf(t, c1[e], cv);
                        if (has_y) nv = fmaf(t, n1[e], nv);
                    }
                    cur.c[k][e] = cv;
                    cur.ny[k][e] = nv;
                }
                float tl = has_tail ? b[STG::kRows + k] : 0.f;
                if constexpr (TRIAL)
                    if (has_tail) tl = fmaf(t, b[STG::kRows + (STG::kSrc - 1) * D + k], tl);
                cur.tail[k] = tl;
            }
        };
#pragma unroll
        for (int s0 = 0; s0 < kObjStages - 1; ++s0) {
            const int jj = j0 + s0 * TG;
            if (jj < fs.nK) issue(jj, s0);
            cp_async_commit();
        }
        int stage = 0;
        for (int j = j0; j < fs.nK; j += TG) {
            const int jf = j + (kObjStages - 1) * TG;
            if (jf < fs.nK) {
                issue(jf, (stage + kObjStages - 1) % kObjStages);
                // the image rows its gathers start from (warped positions
                // stay within a few pixels), into L2 two frames ahead
                const TI* Tf = T + (size_t)__ldg(fs.frames + jf) * N + (valid ? p : 0u);
                prefetch_l2(Tf);
                if (has_y) prefetch_l2(Tf + g.nx);
            }
            cp_async_commit();
            const int fr = __ldg(fs.frames + j);
            cp_async_wait<kObjStages - 1>();
            FrameU<D, VEC, TRIAL> cur;
            read(stage, cur);
            consume(cur, j, fr);
            stage = stage + 1 == kObjStages ? 0 : stage + 1;
        }
        cp_async_wait<0>();
    } else if (j0 < fs.nK) {
        // 3-D: the field of the next frame is loaded into registers while the
        // current one is used
        FrameU<D, VEC, TRIAL> cur;
        cur.load(u, du, t, (size_t)j0 * D * N + p, N, g.nx, sz, valid, has_y, has_z, has_tail);
        int fr = __ldg(fs.frames + j0);
        for (int j = j0; j < fs.nK; j += TG) {
            const int jn = j + TG < fs.nK ? j + TG : j;
            FrameU<D, VEC, TRIAL> nxt;
            nxt.load(u, du, t, (size_t)jn * D * N + p, N, g.nx, sz, valid, has_y, has_z, has_tail);
            const int fr_next = __ldg(fs.frames + jn);
            consume(cur, j, fr);
            cur = nxt;
            fr = fr_next;
        }
    }
    // this warp's mean and sum of squared deviations per pixel
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
        const int k = lane * VEC + e;
        const float mb = cnt > 0.f ? s1[e] / cnt : 0.f;
        sh_m[w][k] = sft[e] + mb;
        sh_q[w][k] = fmaxf(fmaf(-s1[e], mb, s2[e]), 0.f);
#pragma unroll
        for (int c = 0; c < D; ++c) sh_u[w][c][k] = su[c][e];
    }
    if (lane == 0) sh_n[w] = cnt;
    // pairwise tree over the warps of this CTA: slot w absorbs slot w + s
#pragma unroll
    for (int s = FG / 2; s > 0; s >>= 1) {
        __syncthreads();
        if (w < s) {
            const float na = sh_n[w], nb = sh_n[w + s];
            if (nb > 0.f) {
                const float n = na + nb, wb = nb / n, wab = na * nb / n;
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    const int k = lane * VEC + e;
                    const float dl = sh_m[w + s][k] - sh_m[w][k];
                    sh_m[w][k] = na > 0.f ? fmaf(dl, wb, sh_m[w][k]) : sh_m[w + s][k];
                    sh_q[w][k] = sh_q[w][k] + sh_q[w + s][k] + dl * dl * wab;
#pragma unroll
                    for (int c = 0; c < D; ++c) sh_u[w][c][k] += sh_u[w + s][c][k];
                }
            }
            __syncwarp();
            if (lane == 0) sh_n[w] = na + nb;
        }
    }
    __syncthreads();
    bool finisher = true;
    if (S > 1) {
        // merge the splits of this run: rank 0 reads ranks 1..S-1 in order
        cg::cluster_group cl = cg::this_cluster();
        cl.sync();
        finisher = cl.block_rank() == 0;
        if (finisher && threadIdx.x < SEG) {
            const int k = threadIdx.x;
            float n = sh_n[0], m = sh_m[0][k], q = sh_q[0][k], us[D];
#pragma unroll
            for (int c = 0; c < D; ++c) us[c] = sh_u[0][c][k];
            for (int rr = 1; rr < S; ++rr) {
                const float nb = *cl.map_shared_rank(&sh_n[0], rr);
                if (nb > 0.f) {
                    const float mb = *cl.map_shared_rank(&sh_m[0][k], rr);
                    const float qb = *cl.map_shared_rank(&sh_q[0][k], rr);
                    const float tot = n + nb, dl = mb - m;
                    m = n > 0.f ? fmaf(dl, nb / tot, m) : mb;
                    q = q + qb + dl * dl * (n * nb / tot);
                    n = tot;
#pragma unroll
                    for (int c = 0; c < D; ++c) us[c] += *cl.map_shared_rank(&sh_u[0][c][k], rr);
                }
            }
            sh_m[0][k] = m;
            sh_q[0][k] = q;
#pragma unroll
            for (int c = 0; c < D; ++c) sh_u[0][c][k] = us[c];
        }
        cl.sync();   // the other ranks' shared memory stays alive until rank 0 has read it
    }
    float dsum = 0.f, pen = 0.f;
    if (finisher && threadIdx.x < SEG) {
        const int k = threadIdx.x;
        const unsigned pp = p0 + k;
        if (pp < (unsigned)g.N) {
            abar[pp] = sh_m[0][k];
            dsum = cf.half_hd * sh_q[0][k];
            const float invK = 1.0f / (float)fs.nK;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const float ub = sh_u[0][c][k] * invK;
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
        if (ls.S) {   // Armijo decision of trial k
            DevScalars* L = ls.S;
            if (ls.k == 0) {
                L->ls_gTd = out[6];
                L->ls_dnorm2 = out[7];
                L->ls_accepted = 0;
                L->ls_nodescent = !(out[6] < 0.0);
            }
            L->ls_trials = ls.k + 1;
            if (!L->ls_nodescent && out[0] <= ls.J + ls.c * (double)t * L->ls_gTd) {
                L->ls_accepted = 1;
                L->ls_t = t;
            }
        }
    }
}

// ----------------------------------------------------------------- gradient
// Grid-stride over items (frame j, chunk of kThreads * VEC pixels).  Reduced:
// out[4] = |g|^2 (added to the objective pass's totals), out[5] = |u|^2.
template <int D, int VEC, typename TI, typename TD>
__global__ void __launch_bounds__(kThreads)
grad_kernel(const TI* __restrict__ T, Geom g, PixIndex pi, FastDiv chunks, long long items, FrameSet fs,
            Coef cf, FView U, const float* __restrict__ abar, const float* __restrict__ ubar,
            float* __restrict__ grad, TD* __restrict__ dTout, float* __restrict__ unew,
            double* __restrict__ partials, unsigned int* ticket, double* out, const DevScalars* gate) {
    pdl_enter();
    if (gate) {   // the accepted step of a line search decided on the device
        if (!gate->ls_accepted) return;
        U.t = gate->ls_t;
    }
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
        const TI* Tk = T + (size_t)__ldg(fs.frames + j) * N;
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
        if constexpr (D == 2) {
            // every lane takes part (invalid lanes sample pixel 0 with a zero field)
            float a[VEC];
            interp2_row_grad<VEC>(Tk, g, x, y, uc[0], uc[1], a, dt[0], dt[1]);
            if (valid) {
                float ab[VEC];
                if constexpr (VEC == 4) {
                    const float4 q = __ldg(reinterpret_cast<const float4*>(abar + p));
                    ab[0] = q.x; ab[1] = q.y; ab[2] = q.z; ab[3] = q.w;
                } else {
                    ab[0] = __ldg(abar + p);
                }
#pragma unroll
                for (int e = 0; e < VEC; ++e) r[e] = a[e] - ab[e];
            }
        } else if (valid) {
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
            if constexpr (VEC == 4)
                st4f(dTout + base, dt[c]);
            else
                stf(dTout + base, dt[c][0]);
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

constexpr int kGridStride = 152 * 8;   // most CTAs of a grid-stride launch (8 of 256 threads per SM of a GB300)

bool v4ok(const Geom& g, std::initializer_list<const void*> ptrs) {
    if (g.nx % 4) return false;
    for (const void* q : ptrs)
        if (q && ((uintptr_t)q & 15u)) return false;
    return true;
}

}  // namespace

// Launch shape of the objective pass: pixels per lane and frame splits.
struct ObjShape {
    int vec, splits;
    unsigned runs;
};

// Built-in launch shape (measured with the autotuner on 32^2 .. 256^2 levels
// of 51 .. 200 frames): about 256 CTAs, from the widest pixel runs that reach
// it with at most 4 frame splits; Armijo trials (field and step staged, twice
// the ring) at most 2 pixels per lane in 2-D.
ObjShape obj_shape(const Geom& g, int nK, int vec_max, bool trial) {
    constexpr int FG = kThreads / 32, kTarget = 256, kMaxSplit = 4;
    if (g.d == 2 && trial) vec_max = std::min(vec_max, 2);
    const int max_split = std::max(1, std::min(kMaxSplit, (nK + FG - 1) / FG));
    ObjShape sh{1, 1, 0};
    for (int v : {4, 2, 1}) {
        if (v > vec_max || g.nx % v || (g.d == 3 && v == 4)) continue;
        sh.vec = v;
        sh.runs = (unsigned)((g.N + 32LL * v - 1) / (32LL * v));
        if ((long long)sh.runs * max_split >= kTarget) break;
    }
    sh.splits = (int)std::min<long long>(max_split, ((long long)kTarget + sh.runs - 1) / sh.runs);
    return sh;
}

int obj_shape_candidates(const Geom& g, int nK, ObjShapeChoice* out, int cap) {
    constexpr int FG = kThreads / 32;
    const int max_split = std::max(1, std::min(8, (nK + FG - 1) / FG));
    int n = 0;
    for (int v : {4, 2, 1}) {
        if (g.nx % v || (g.d == 3 && v == 4)) continue;
        for (int sp : {1, 2, 4, 8})
            if (sp <= max_split && n < cap) out[n++] = ObjShapeChoice{v, sp};
    }
    return n;
}

size_t eval_partials(const Geom& g, int nK) {
    const ObjShape sh = obj_shape(g, nK < 1 ? 1 : nK, 1, false);   // the most runs any launch uses
    const size_t obj = (size_t)sh.runs * 8 * 8;                     // every split count up to 8
    return obj > (size_t)kGridStride * 2 ? obj : (size_t)kGridStride * 2;
}

template <int D, int VEC, bool TRIAL, bool GDOT, typename TI>
static cudaError_t obj_go(const ObjShape& sh, cudaStream_t s, const TI* T, const Geom& g, const PixIndex& pi,
                          const FrameSet& fs, const Coef& cf, const float* u, const float* du, float t,
                          const float* gdot, float* abar, float* ubar, double* partials, unsigned int* ticket,
                          double* out, const LineSearchArgs& ls) {
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(sh.runs, (unsigned)sh.splits, 1);
    lc.blockDim = dim3(kThreads, 1, 1);
    lc.stream = s;
    if constexpr (D == 2) {   // the copy ring of the staged 2-D pass
        const size_t ring = ObjStage<D, VEC, TRIAL>::ring_bytes;
        const cudaError_t e =
            set_max_dynamic_smem(reinterpret_cast<const void*>(obj_kernel<D, VEC, TRIAL, GDOT, TI>), (int)ring);
        if (e != cudaSuccess) return e;
        lc.dynamicSmemBytes = ring;
    }
    cudaLaunchAttribute at[2];
    unsigned na = 0;
    if (sh.splits > 1) {
        at[na].id = cudaLaunchAttributeClusterDimension;
        at[na].val.clusterDim.x = 1;
        at[na].val.clusterDim.y = (unsigned)sh.splits;
        at[na].val.clusterDim.z = 1;
        ++na;
    }
    na += pdl_attr(s, at + na);
    lc.attrs = at;
    lc.numAttrs = na;
    return cudaLaunchKernelEx(&lc, obj_kernel<D, VEC, TRIAL, GDOT, TI>, T, g, pi, fs, cf, u, du, t, gdot, abar, ubar,
                              partials, ticket, out, ls);
}

template <int D, int VEC, typename TI>
static cudaError_t obj_mode(const ObjShape& sh, cudaStream_t s, const TI* T, const Geom& g, const PixIndex& pi,
                            const FrameSet& fs, const Coef& cf, const float* u, const float* du, float t,
                            const float* gdot, float* abar, float* ubar, double* partials, unsigned int* ticket,
                            double* out, const LineSearchArgs& ls) {
    if (!du) return obj_go<D, VEC, false, false>(sh, s, T, g, pi, fs, cf, u, du, t, gdot, abar, ubar, partials, ticket, out, ls);
    if (!gdot) return obj_go<D, VEC, true, false>(sh, s, T, g, pi, fs, cf, u, du, t, gdot, abar, ubar, partials, ticket, out, ls);
    return obj_go<D, VEC, true, true>(sh, s, T, g, pi, fs, cf, u, du, t, gdot, abar, ubar, partials, ticket, out, ls);
}

cudaError_t launch_objective(const Stored& T, const Geom& g, const FrameSet& fs, const Coef& cf, const float* u,
                             const float* du, float t, const float* gdot, float* abar, float* ubar, double* partials,
                             size_t partials_cap, unsigned int* ticket, double* out, cudaStream_t s,
                             const LineSearchArgs* lsp, const ObjShapeChoice* force) {
    const PixIndex pi{FastDiv::make((unsigned)g.nx), FastDiv::make((unsigned)g.ny)};
    const LineSearchArgs ls = lsp ? *lsp : LineSearchArgs{nullptr, 0, 0.0, 0.0};
    if (ls.S && ls.k == 0 && !gdot) return cudaErrorInvalidValue;
    // pixels per lane: 4 (2 in 3-D) when rows and every array allow vector access
    int vec_max = g.d == 3 ? 2 : 4;
    for (const void* q : {(const void*)u, (const void*)du, (const void*)gdot})
        if (q && ((uintptr_t)q & 15u)) vec_max = (uintptr_t)q & 7u ? 1 : std::min(vec_max, 2);
    ObjShape sh = obj_shape(g, fs.nK, vec_max, du != nullptr);
    if (force) {   // a tuned shape: valid for these arrays and this level, else refused
        if (force->vec > vec_max || g.nx % force->vec || force->splits < 1 || force->splits > 8 ||
            (g.d == 3 && force->vec == 4))
            return cudaErrorInvalidValue;
        sh.vec = force->vec;
        sh.splits = force->splits;
        sh.runs = (unsigned)((g.N + 32LL * sh.vec - 1) / (32LL * sh.vec));
    }
    if ((size_t)sh.runs * sh.splits * 8 > partials_cap) return cudaErrorInvalidValue;
    if (gdot && !du) return cudaErrorInvalidValue;
    cudaError_t e = with_store_type(T.type, [&](auto tag) {
        using TI = decltype(tag);
        const TI* Ti = static_cast<const TI*>(T.p);
        cudaError_t r;
#define STML_OBJ(D_, V_) r = obj_mode<D_, V_>(sh, s, Ti, g, pi, fs, cf, u, du, t, gdot, abar, ubar, partials, ticket, out, ls)
        if (g.d == 2) {
            if (sh.vec == 4) STML_OBJ(2, 4); else if (sh.vec == 2) STML_OBJ(2, 2); else STML_OBJ(2, 1);
        } else {
            if (sh.vec == 2) STML_OBJ(3, 2); else STML_OBJ(3, 1);
        }
#undef STML_OBJ
        return r;
    });
    count_launches(1);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_gradient(const Stored& T, const Geom& g, const FrameSet& fs, const Coef& cf, const float* u,
                            const float* du, float t, const float* abar, const float* ubar, float* grad, void* dT,
                            int dT_type, float* unew, double* partials, size_t partials_cap, unsigned int* ticket,
                            double* out, cudaStream_t s, const DevScalars* gate) {
    // grad T is stored as float or in the image's own 16-bit type
    if (dT_type != ST_F32 && dT_type != T.type) return cudaErrorInvalidValue;
    const PixIndex pi{FastDiv::make((unsigned)g.nx), FastDiv::make((unsigned)g.ny)};
    const bool v4 = v4ok(g, {u, du, abar, ubar, grad, dT, unew});
    const int vec = v4 ? 4 : 1;
    const long long cpf = (g.N + (long long)kThreads * vec - 1) / ((long long)kThreads * vec);
    const long long items = cpf * fs.nK;
    const FastDiv chunks = FastDiv::make((unsigned)cpf);
    const FView U{u, du, t};
    auto go = [&](auto ti_tag, auto td_tag) {
        using TI = decltype(ti_tag);
        using TD = decltype(td_tag);
        const TI* Ti = static_cast<const TI*>(T.p);
        TD* Td = static_cast<TD*>(dT);
#define STML_GRAD(D_, V_)                                                                                 \
    do {                                                                                                  \
        auto k = grad_kernel<D_, V_, TI, TD>;                                                             \
        const unsigned blocks = resident_grid((const void*)k, items, kGridStride);                        \
        if ((size_t)blocks * 2 > partials_cap) return cudaErrorInvalidValue;                              \
        const cudaError_t le = launch_pdl(k, dim3(blocks), dim3(kThreads), 0, s, Ti, g, pi, chunks, items, fs, cf, U, \
                                          abar, ubar, grad, Td, unew, partials, ticket, out, gate);       \
        if (le != cudaSuccess) return le;                                                                 \
    } while (0)
        if (g.d == 2) {
            if (v4) STML_GRAD(2, 4); else STML_GRAD(2, 1);
        } else {
            if (v4) STML_GRAD(3, 4); else STML_GRAD(3, 1);
        }
#undef STML_GRAD
        return cudaGetLastError();
    };
    cudaError_t e = with_store_type(T.type, [&](auto ti_tag) {
        using TI = decltype(ti_tag);
        return dT_type == ST_F32 ? go(ti_tag, float{}) : go(ti_tag, TI{});
    });
    count_launches(1);
    return e;
}

}  // namespace stml
