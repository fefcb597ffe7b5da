// Displacements on a grid coarser than the images.  The unknowns w_k of a
// level live on its image grid coarsened by F = 2^s per axis; the field that
// warps the images is u_k = P_s w_k, P_s the cell-centred multilinear
// interpolation from the coarse grid with clamp-to-edge (per axis, fine cell
// j sits at coarse index coordinate xi = (j + 1/2)/F - 1/2 and takes
// (1 - f) w[clamp(floor xi)] + f w[clamp(floor xi + 1)], f = xi - floor xi).
// The distance of eq. (1) is evaluated on the image grid at u; S and P of
// Sec. 2 on the coarse grid, where the unknowns are.
//
//   ugrid_prolong_kernel   u = P_s (w + t dw), one image-grid value per thread
//   ugrid_gather_kernel    P_s^T f (the gradient's adjoint), or the Jacobi
//                          inverse from (P_s o P_s)^T of the image-grid
//                          distance diagonal: one coarse value per thread,
//                          a fixed-order gather over the 2F (per axis) fine
//                          cells it is blended into; no atomics
//   ugrid_reg_kernel       S, P and their gradient (or Hessian product) on
//                          the coarse grid, added to the gathered data term
//   ugrid_vec_kernel       the PCG vector steps and dot products
// All element-wise, bound by HBM or L2 bandwidth; reductions are the
// library's deterministic two-stage sums.
#include "kernels.h"

namespace stml {

namespace {

struct AxisTap {
    int c0, c1;
    float w0, w1;
};

// Interpolation taps of fine cell j along one axis (mc coarse cells).  xi
// and f are exact in float32: F is a power of two.
__device__ __forceinline__ AxisTap axis_tap(int j, int mc, float inv_F) {
    const float xi = ((float)j + 0.5f) * inv_F - 0.5f;
    const float fl = floorf(xi);
    const int i0 = (int)fl;
    const float f = xi - fl;
    return {clampi(i0, mc - 1), clampi(i0 + 1, mc - 1), 1.0f - f, f};
}

// Entry (j, i) of the one-axis interpolation matrix.
__device__ __forceinline__ float axis_entry(int j, int i, int mc, float inv_F) {
    const AxisTap t = axis_tap(j, mc, inv_F);
    return (t.c0 == i ? t.w0 : 0.f) + (t.c1 == i ? t.w1 : 0.f);
}

__device__ __forceinline__ void coords(long long p, int nx, int ny, int& x, int& y, int& z) {
    x = (int)(p % nx);
    const long long r = p / nx;
    y = (int)(r % ny);
    z = (int)(r / ny);
}

__global__ void __launch_bounds__(kThreads)
ugrid_prolong_kernel(const float* __restrict__ w, const float* __restrict__ dw, float t, float* __restrict__ u,
                     long long planes, UGrid ug, const int* gate) {
    pdl_enter();
    if (gate && !*gate) return;
    const long long total = planes * ug.N;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
        const long long pl = e / ug.N;
        int x, y, z;
        coords(e - pl * ug.N, ug.nx, ug.ny, x, y, z);
        const AxisTap tx = axis_tap(x, ug.cx, ug.inv_F), ty = axis_tap(y, ug.cy, ug.inv_F);
        const AxisTap tz = ug.d == 3 ? axis_tap(z, ug.cz, ug.inv_F) : AxisTap{0, 0, 1.0f, 0.0f};
        const size_t base = (size_t)pl * ug.Nc;
        auto at = [&](int cz, int cy, int cx) {
            const size_t i = base + ((size_t)cz * ug.cy + cy) * ug.cx + cx;
            return dw ? fmaf(t, __ldg(dw + i), __ldg(w + i)) : __ldg(w + i);
        };
        float acc = 0.f;
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const float wz = a ? tz.w1 : tz.w0;
            if (wz == 0.f) continue;   // the second z tap of a 2-D grid
            const int cz = a ? tz.c1 : tz.c0;
            float col = 0.f;
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const int cy = b ? ty.c1 : ty.c0;
                const float row = fmaf(tx.w1, at(cz, cy, tx.c1), tx.w0 * at(cz, cy, tx.c0));
                col = fmaf(b ? ty.w1 : ty.w0, row, col);
            }
            acc = fmaf(wz, col, acc);
        }
        u[e] = acc;
    }
}

// MODE 0: out = P_s^T f.  MODE 1: out = 1 / diag with diag the Jacobi
// diagonal of the coarse-grid Gauss-Newton Hessian,
//   (P_s o P_s)^T (hd (1 - 1/|K|) (d_c T)^2) + alpha hd_w nnb / h_w^2
//   + alpha_t hd_w (w_prev + w_next) + 2 lambda hd_w / |K|^2,
// with f = grad T on the image grid and cw the coefficients of the coarse grid.
template <int MODE>
__global__ void __launch_bounds__(kThreads)
ugrid_gather_kernel(const float* __restrict__ f, float* __restrict__ out, long long planes, UGrid ug, FrameSet fs,
                    Coef cf, Coef cw, const int* gate) {
    pdl_enter();
    if (gate && !*gate) return;
    const long long total = planes * ug.Nc;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const int hF = ug.F / 2, F3 = 3 * ug.F / 2;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
        const long long pl = e / ug.Nc;
        int ix, iy, iz;
        coords(e - pl * ug.Nc, ug.cx, ug.cy, ix, iy, iz);
        const int x0 = max(0, ix * ug.F - hF), x1 = min(ug.nx, ix * ug.F + F3);
        const int y0 = max(0, iy * ug.F - hF), y1 = min(ug.ny, iy * ug.F + F3);
        const int z0 = ug.d == 3 ? max(0, iz * ug.F - hF) : 0, z1 = ug.d == 3 ? min(ug.nz, iz * ug.F + F3) : 1;
        const float* fp = f + (size_t)pl * ug.N;
        float acc = 0.f;
        for (int jz = z0; jz < z1; ++jz) {
            float ez = ug.d == 3 ? axis_entry(jz, iz, ug.cz, ug.inv_F) : 1.0f;
            if (ez == 0.f) continue;
            if (MODE == 1) ez *= ez;
            float accy = 0.f;
            for (int jy = y0; jy < y1; ++jy) {
                float ey = axis_entry(jy, iy, ug.cy, ug.inv_F);
                if (ey == 0.f) continue;
                if (MODE == 1) ey *= ey;
                const float* row = fp + ((size_t)jz * ug.ny + jy) * ug.nx;
                float accx = 0.f;
                for (int jx = x0; jx < x1; ++jx) {
                    float ex = axis_entry(jx, ix, ug.cx, ug.inv_F);
                    float v = __ldg(row + jx);
                    if (MODE == 1) {
                        ex *= ex;
                        v = cf.diag_D * v * v;
                    }
                    accx = fmaf(ex, v, accx);
                }
                accy = fmaf(ey, accx, accy);
            }
            acc = fmaf(ez, accy, acc);
        }
        if (MODE == 1) {
            const int j = (int)(pl / ug.d);
            Geom gw{ug.cx, ug.cy, ug.cz, ug.d, ug.Nc, 0.f, 0.f, 0.f};
            const int nnb = neighbour_count(gw, ix, iy, iz);
            const float tdiag = (j + 1 < fs.nK ? __ldg(fs.w_next + j) : 0.f) + (j > 0 ? __ldg(fs.w_next + j - 1) : 0.f);
            float dg = acc + cw.alpha_hd * cw.inv_h2 * (float)nnb;
            dg = fmaf(cw.alphat_hd, tdiag, dg) + cw.pen_h;
            acc = dg > 0.f ? 1.0f / dg : 1.0f;
        }
        out[e] = acc;
    }
}

// S and P on the coarse grid gw at the field w + t dw (dw may be null; gin
// may be the same array as gout, each element is read before it is written), one
// thread per (coarse pixel, component) over all frames of K.
// MODE 0 (objective): reduces out[0] = sum of squared forward differences
// (times h_w^2), out[1] = the temporal sum, out[2] = sum over pixels and
// components of (sum_j w_j)^2, out[3] = |g|^2, out[4] = |w|^2; with gout it
// writes g = gin + alpha hd_w B^T B w + alpha_t hd_w L_t w + 2 lambda hd_w wbar / |K|.
// MODE 1 (Hessian product of the regulariser and penalty): gout = gin +
// alpha hd_w B^T B w + alpha_t hd_w L_t w + 2 lambda hd_w / |K|^2 sum_j w_j,
// out[0] = <w, gout>.
template <int MODE>
__global__ void __launch_bounds__(kThreads)
ugrid_reg_kernel(Geom gw, FrameSet fs, Coef cw, const float* __restrict__ w, const float* __restrict__ dw, float t,
                 const float* gin, float* gout, double* __restrict__ partials, unsigned int* ticket, double* out,
                 UgCg* cg) {
    pdl_enter();
    if (cg && !cg->active) return;
    const long long Nc = gw.N;
    const long long items = Nc * gw.d;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long sz = (long long)gw.nx * gw.ny;
    double a_sx = 0.0, a_st = 0.0, a_pen = 0.0, a_g2 = 0.0, a_w2 = 0.0, a_pq = 0.0;
    for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < items; it += stride) {
        const int c = (int)(it / Nc);
        const long long q = it - (long long)c * Nc;
        int x, y, z;
        coords(q, gw.nx, gw.ny, x, y, z);
        auto fld = [&](int j, long long p) {
            const size_t i = ((size_t)j * gw.d + c) * (size_t)Nc + (size_t)p;
            return dw ? fmaf(t, __ldg(dw + i), __ldg(w + i)) : __ldg(w + i);
        };
        float wsum = 0.f;
        for (int j = 0; j < fs.nK; ++j) wsum += fld(j, q);
        if (MODE == 0) a_pen += (double)wsum * (double)wsum;
        const float pen = MODE == 0 ? cw.pen_g * wsum * cw.inv_nK : cw.pen_h * wsum;
        float prev = 0.f, cur = fld(0, q);
        for (int j = 0; j < fs.nK; ++j) {
            const float next = j + 1 < fs.nK ? fld(j + 1, q) : 0.f;
            float lap = 0.f, fwd = 0.f;
            if (x > 0) lap += cur - fld(j, q - 1);
            if (x < gw.nx - 1) { const float nb = fld(j, q + 1); lap += cur - nb; fwd += (nb - cur) * (nb - cur); }
            if (y > 0) lap += cur - fld(j, q - gw.nx);
            if (y < gw.ny - 1) { const float nb = fld(j, q + gw.nx); lap += cur - nb; fwd += (nb - cur) * (nb - cur); }
            if (gw.d == 3) {
                if (z > 0) lap += cur - fld(j, q - sz);
                if (z < gw.nz - 1) { const float nb = fld(j, q + sz); lap += cur - nb; fwd += (nb - cur) * (nb - cur); }
            }
            float tl = 0.f;
            if (cw.alphat_hd != 0.f) {
                const float wp = j > 0 ? __ldg(fs.w_next + j - 1) : 0.f;
                const float wn = j + 1 < fs.nK ? __ldg(fs.w_next + j) : 0.f;
                if (j > 0) tl += wp * (cur - prev);
                if (j + 1 < fs.nK) {
                    tl += wn * (cur - next);
                    if (MODE == 0) a_st += (double)(wn * (next - cur) * (next - cur));
                }
            }
            if (MODE == 0) {
                a_sx += (double)fwd;
                a_w2 += (double)cur * (double)cur;
            }
            if (gout) {
                const size_t i = ((size_t)j * gw.d + c) * (size_t)Nc + (size_t)q;
                float gv = fmaf(cw.alpha_hd * cw.inv_h2, lap, fmaf(cw.alphat_hd, tl, pen));
                if (gin) gv += gin[i];   // gin may be gout: read before the store
                gout[i] = gv;
                if (MODE == 0) a_g2 += (double)gv * (double)gv;
                if (MODE == 1) a_pq += (double)cur * (double)gv;
            }
            prev = cur;
            cur = next;
        }
    }
    if (MODE == 0) {
        float acc[5] = {(float)a_sx, (float)a_st, (float)a_pen, (float)a_g2, (float)a_w2};
        grid_reduce<5>(acc, partials, ticket, out);
    } else {
        float acc[1] = {(float)a_pq};
        if (grid_reduce<1>(acc, partials, ticket, out) && threadIdx.x == 0 && cg) {
            const double pq = out[0];   // the PCG decision of this step: alpha or breakdown
            cg->pq = pq;
            if (!(pq > 0.0)) {
                cg->flag = CG_BREAKDOWN;
                cg->active = 0;
                if (cg->mirror) *cg->mirror = 0;
            } else {
                cg->alpha = cg->rho / pq;
            }
        }
    }
}

// PCG vector steps on the coarse grid (n values), a the step coefficient:
//   VEC_INIT: r = -g, z = Minv r, p = z, x = 0;    out = {<r, z>, |r|^2}
//   VEC_STEP: x += a p, r -= a q, z = Minv r;     out = {|r|^2, <r, z>}
//   VEC_DIR:  p = z + a p
//   VEC_DOT:  out = {<x, p>}
//   VEC_AXPY: z = x + a p
// (x and p may be the same array in VEC_DOT.)
template <int MODE>
__global__ void __launch_bounds__(kThreads)
ugrid_vec_kernel(long long n, float a, const float* Minv, float* x, float* r, float* z, float* p, const float* q,
                 const float* g, double* __restrict__ partials, unsigned int* ticket, double* out, UgCg* cg,
                 double thr, int max_cg) {
    pdl_enter();
    if (cg && (MODE == VEC_STEP || MODE == VEC_DIR)) {
        if (!cg->active) return;
        a = (float)(MODE == VEC_STEP ? cg->alpha : cg->beta);
    }
    const long long stride = (long long)gridDim.x * blockDim.x;
    double s0 = 0.0, s1 = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        if (MODE == VEC_INIT) {
            const float rv = -g[i], zv = Minv[i] * rv;
            r[i] = rv;
            z[i] = zv;
            p[i] = zv;
            x[i] = 0.f;
            s0 += (double)rv * (double)zv;
            s1 += (double)rv * (double)rv;
        } else if (MODE == VEC_STEP) {
            x[i] = fmaf(a, p[i], x[i]);
            const float rv = fmaf(-a, q[i], r[i]), zv = Minv[i] * rv;
            r[i] = rv;
            z[i] = zv;
            s0 += (double)rv * (double)rv;
            s1 += (double)rv * (double)zv;
        } else if (MODE == VEC_DIR) {
            p[i] = fmaf(a, p[i], z[i]);
        } else if (MODE == VEC_DOT) {
            s0 += (double)x[i] * (double)p[i];
        } else {
            z[i] = fmaf(a, p[i], x[i]);
        }
    }
    if (MODE == VEC_INIT || MODE == VEC_STEP) {
        float acc[2] = {(float)s0, (float)s1};
        if (grid_reduce<2>(acc, partials, ticket, out) && threadIdx.x == 0 && cg) {
            if (MODE == VEC_INIT) {   // start: rho = <r, z>; stop at ||r|| <= thr
                cg->rho = out[0];
                cg->thr = thr;
                cg->iter = 0;
                cg->max_cg = max_cg;
                cg->pq = 0.0;
                cg->rnorm2 = out[1];
                cg->flag = !(out[1] > 0.0) ? CG_ZERO : max_cg <= 0 ? CG_MAXIT : CG_RUNNING;
                cg->active = cg->flag == CG_RUNNING;
            } else {                  // after x += alpha p, r -= alpha q: stop, or beta = <r, z> / rho
                cg->iter += 1;
                cg->rnorm2 = out[0];
                if (sqrt(out[0]) <= cg->thr) {
                    cg->flag = CG_CONVERGED;
                    cg->active = 0;
                } else if (cg->iter >= cg->max_cg) {
                    cg->flag = CG_MAXIT;
                    cg->active = 0;
                } else {
                    cg->beta = out[1] / cg->rho;
                    cg->rho = out[1];
                }
            }
            if (cg->mirror) *cg->mirror = cg->active;
        }
    } else if (MODE == VEC_DOT) {
        float acc[1] = {(float)s0};
        grid_reduce<1>(acc, partials, ticket, out);
    }
}

}  // namespace

UGrid make_ugrid(const Geom& fine, int s) {
    UGrid ug;
    ug.F = 1 << s;
    ug.inv_F = 1.0f / (float)ug.F;
    ug.d = fine.d;
    ug.nx = fine.nx;
    ug.ny = fine.ny;
    ug.nz = fine.nz;
    ug.cx = fine.nx / ug.F;
    ug.cy = fine.ny / ug.F;
    ug.cz = fine.d == 3 ? fine.nz / ug.F : 1;
    ug.N = fine.N;
    ug.Nc = (long long)ug.cx * ug.cy * ug.cz;
    return ug;
}

cudaError_t launch_ugrid_prolong(const float* w, const float* dw, float t, float* u, long long planes,
                                 const UGrid& ug, cudaStream_t s, const int* gate) {
    const long long total = planes * ug.N;
    if (total <= 0) return cudaSuccess;
    const unsigned grid = resident_grid((const void*)ugrid_prolong_kernel, (total + kThreads - 1) / kThreads, 152 * 8);
    count_launches(1);
    return launch_pdl(ugrid_prolong_kernel, dim3(grid), dim3(kThreads), 0, s, w, dw, t, u, planes, ug, gate);
}

cudaError_t launch_ugrid_adjoint(const float* f, float* out, long long planes, const UGrid& ug, cudaStream_t s,
                                 const int* gate) {
    const long long total = planes * ug.Nc;
    if (total <= 0) return cudaSuccess;
    const unsigned grid = resident_grid((const void*)ugrid_gather_kernel<0>, (total + kThreads - 1) / kThreads, 152 * 8);
    count_launches(1);
    return launch_pdl(ugrid_gather_kernel<0>, dim3(grid), dim3(kThreads), 0, s, f, out, planes, ug, FrameSet{},
                      Coef{}, Coef{}, gate);
}

cudaError_t launch_ugrid_jacobi(const float* dT, float* Minv, const UGrid& ug, const FrameSet& fs, const Coef& cf,
                                const Coef& cw, cudaStream_t s) {
    const long long planes = (long long)fs.nK * ug.d;
    const long long total = planes * ug.Nc;
    if (total <= 0) return cudaSuccess;
    const unsigned grid = resident_grid((const void*)ugrid_gather_kernel<1>, (total + kThreads - 1) / kThreads, 152 * 8);
    count_launches(1);
    return launch_pdl(ugrid_gather_kernel<1>, dim3(grid), dim3(kThreads), 0, s, dT, Minv, planes, ug, fs, cf, cw,
                      (const int*)nullptr);
}

cudaError_t launch_ugrid_reg(int mode, const Geom& gw, const FrameSet& fs, const Coef& cw, const float* w,
                             const float* dw, float t, const float* gin, float* gout, double* partials,
                             size_t partials_cap, unsigned int* ticket, double* out, cudaStream_t s, UgCg* cg) {
    const long long items = gw.N * gw.d;
    auto k = mode == 0 ? ugrid_reg_kernel<0> : ugrid_reg_kernel<1>;
    const unsigned grid = resident_grid((const void*)k, (items + kThreads - 1) / kThreads, 152 * 8);
    if ((size_t)grid * 5 > partials_cap) return cudaErrorInvalidValue;
    count_launches(1);
    return launch_pdl(k, dim3(grid), dim3(kThreads), 0, s, gw, fs, cw, w, dw, t, gin, gout, partials, ticket, out,
                      mode == 1 ? cg : nullptr);
}

cudaError_t launch_ugrid_vec(int mode, long long n, float a, const float* Minv, float* x, float* r, float* z,
                             float* p, const float* q, const float* g, double* partials, size_t partials_cap,
                             unsigned int* ticket, double* out, cudaStream_t s, UgCg* cg, double thr, int max_cg) {
    if (n <= 0) return cudaErrorInvalidValue;
    const void* kp = nullptr;
    switch (mode) {
        case VEC_INIT: kp = (const void*)ugrid_vec_kernel<VEC_INIT>; break;
        case VEC_STEP: kp = (const void*)ugrid_vec_kernel<VEC_STEP>; break;
        case VEC_DIR: kp = (const void*)ugrid_vec_kernel<VEC_DIR>; break;
        case VEC_DOT: kp = (const void*)ugrid_vec_kernel<VEC_DOT>; break;
        case VEC_AXPY: kp = (const void*)ugrid_vec_kernel<VEC_AXPY>; break;
        default: return cudaErrorInvalidValue;
    }
    const unsigned grid = resident_grid(kp, (n + kThreads - 1) / kThreads, 152 * 8);
    if ((size_t)grid * 2 > partials_cap) return cudaErrorInvalidValue;
    count_launches(1);
#define STML_VEC(M_) \
    return launch_pdl(ugrid_vec_kernel<M_>, dim3(grid), dim3(kThreads), 0, s, n, a, Minv, x, r, z, p, q, g, partials, \
                      ticket, out, cg, thr, max_cg)
    switch (mode) {
        case VEC_INIT: STML_VEC(VEC_INIT);
        case VEC_STEP: STML_VEC(VEC_STEP);
        case VEC_DIR: STML_VEC(VEC_DIR);
        case VEC_DOT: STML_VEC(VEC_DOT);
        default: STML_VEC(VEC_AXPY);
    }
#undef STML_VEC
}

}  // namespace stml
