// Shared device helpers of the STML library: level geometry, interpolation,
// stencils and the deterministic two-stage FP64 reduction.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace stml {

// Storage types of the image pyramid and of grad T (the arithmetic is FP32).
enum StoreType { ST_F32 = 0, ST_F16 = 1, ST_BF16 = 2 };

inline size_t store_bytes(int st) { return st == ST_F32 ? 4 : 2; }

// Entry of a kernel that may be launched as a programmatic dependent launch
// (the launch starts its CTAs while the previous kernel of the stream is
// still finishing).  griddepcontrol.wait blocks until every grid this launch
// depends on has completed and its memory is visible, so it comes before
// any global load or store and before any early return (a kernel that left
// without waiting could complete before its predecessor, and the kernel
// after it would then no longer be ordered after that predecessor).  Then
// launch_dependents lets the next kernel of the stream start its own CTAs,
// which wait in turn.  Both are no-ops in a launch without the attribute.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// One value of a stored array, as float (read-only path), and its store
// (round to nearest even).
__device__ __forceinline__ float ldf(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ldf(const __half* p) { return __half2float(__ldg(p)); }
__device__ __forceinline__ float ldf(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
__device__ __forceinline__ void stf(float* p, float v) { *p = v; }
__device__ __forceinline__ void stf(__half* p, float v) { *p = __float2half_rn(v); }
__device__ __forceinline__ void stf(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

// Asynchronous global -> shared copies (cp.async): BYTES = 4, 8 or 16, both
// addresses aligned to BYTES.  A thread commits its copies as a group and
// waits until at most N of its groups are still in flight.
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Four consecutive stored values (address aligned to four elements), as float.
__device__ __forceinline__ void ld4f(const float* p, float (&o)[4]) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = q.x; o[1] = q.y; o[2] = q.z; o[3] = q.w;
}
__device__ __forceinline__ void ld4f(const __half* p, float (&o)[4]) {
    const uint2 q = __ldg(reinterpret_cast<const uint2*>(p));
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&q.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&q.y));
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
__device__ __forceinline__ void ld4f(const __nv_bfloat16* p, float (&o)[4]) {
    const uint2 q = __ldg(reinterpret_cast<const uint2*>(p));
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q.y));
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
__device__ __forceinline__ void st4f(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4f(__half* p, const float (&v)[4]) {
    const __half2 a = __floats2half2_rn(v[0], v[1]), b = __floats2half2_rn(v[2], v[3]);
    uint2 q;
    q.x = *reinterpret_cast<const unsigned*>(&a);
    q.y = *reinterpret_cast<const unsigned*>(&b);
    *reinterpret_cast<uint2*>(p) = q;
}
__device__ __forceinline__ void st4f(__nv_bfloat16* p, const float (&v)[4]) {
    const __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]), b = __floats2bfloat162_rn(v[2], v[3]);
    uint2 q;
    q.x = *reinterpret_cast<const unsigned*>(&a);
    q.y = *reinterpret_cast<const unsigned*>(&b);
    *reinterpret_cast<uint2*>(p) = q;
}

constexpr int kThreads = 256;          // threads per CTA of the elementwise kernels
constexpr int kMaxRed = 8;             // values one reduction carries

// One spatial level.  Axes are (z, y, x) with x fastest; a 2-D level has nz = 1.
// Component c of a field moves along axis (3 - d) + c of (z, y, x).
struct Geom {
    int nx, ny, nz;
    int d;
    long long N;          // cells per frame
    float h, inv_h, hd;   // cell width, its inverse (a power of two), cell volume h^d
};

// Device-resident scalars of one context.  The reducing kernels write their
// totals here; the PCG kernels keep their coefficients here so that no value
// has to travel to the host inside the conjugate-gradient loop.
struct DevScalars {
    double red[kMaxRed];      // totals of the last evaluation (J, D, S, P, |g|^2, |u|^2, ...)
    double trial[kMaxRed];    // totals of the last objective-only evaluation
    double dots[kMaxRed];     // totals of the last dot-product kernel
    float rho, bnorm2, pq, alpha, beta, rnorm2;   // CG coefficients (device only)
    int cg_active, cg_iter, cg_flag;
    int pq_parts;              // CTA partials of <p, Hp> left by the last streaming Hessian product
    // Armijo line search decided on the device (trial k has t = 2^-k)
    double ls_gTd, ls_dnorm2;  // <g, d> and |d|^2 from trial 0
    float ls_t;                // the accepted step
    int ls_accepted;           // a trial met the Armijo test
    int ls_nodescent;          // trial 0 found <g, d> >= 0
    int ls_trials;             // trials that ran
    unsigned int err_flags;   // bit 0: a bounded device wait expired
    unsigned int err_pad;
    unsigned int ticket[8];   // arrival counters of the last-CTA reduction
};

enum CgFlag { CG_RUNNING = 0, CG_CONVERGED = 1, CG_MAXIT = 2, CG_BREAKDOWN = 3, CG_ZERO = 4 };

// Division by a fixed divisor d < 2^31 with a multiply-high (round-up method):
// q = (umulhi(n, m) + n) >> s, s = ceil(log2 d), m = floor(2^32 (2^s - d) / d) + 1.
struct FastDiv {
    unsigned d, m, s;
    static FastDiv make(unsigned dv) {
        FastDiv f;
        f.d = dv;
        unsigned sh = 0;
        while ((1ull << sh) < dv) ++sh;
        f.s = sh;
        f.m = (unsigned)((((1ull << sh) - dv) << 32) / dv + 1);
        return f;
    }
    __device__ __forceinline__ unsigned div(unsigned n) const {
        return (unsigned)(((unsigned long long)__umulhi(n, m) + n) >> s);
    }
};

// Divisors that turn a pixel index into (x, y, z).
struct PixIndex {
    FastDiv nx, ny;
};

// Per-GIR description of the frame subset K in device memory.
struct FrameSet {
    const int* frames;      // frame numbers of K (index into the image array)
    const float* w_next;    // 1/(k_{j+1} - k_j)^2, 0 for the last frame of K
    int nK;
};

// Constant coefficients of one objective evaluation.
struct Coef {
    float alpha_hd;     // alpha * hd
    float alphat_hd;    // alpha_t * hd
    float pen_g;        // 2 lambda hd / |K|   (penalty gradient factor on ubar)
    float pen_h;        // 2 lambda hd / |K|^2 (penalty Hessian factor on sum_j v_j)
    float lam_hd;       // lambda * hd
    float half_hd;      // hd / 2
    float hd;
    float inv_h2;       // 1 / h^2
    float inv_nK;       // 1 / |K|
    float diag_D;       // hd (1 - 1/|K|)
};

// ------------------------------------------------------------ coordinates
__device__ __forceinline__ void unflatten(const Geom& g, long long p, int& x, int& y, int& z) {
    x = (int)(p % g.nx);
    long long r = p / g.nx;
    y = (int)(r % g.ny);
    z = (int)(r / g.ny);
}

// Stride of axis a (0 = z, 1 = y, 2 = x) in a plane.
__device__ __forceinline__ long long axis_stride(const Geom& g, int a) {
    return a == 2 ? 1LL : (a == 1 ? (long long)g.nx : (long long)g.nx * g.ny);
}

// Number of neighbours inside the grid (all axes), i.e. h^2 * diag(B^T B).
__device__ __forceinline__ int neighbour_count(const Geom& g, int x, int y, int z) {
    int c = 0;
    c += (x > 0) + (x < g.nx - 1);
    c += (y > 0) + (y < g.ny - 1);
    if (g.d == 3) c += (z > 0) + (z < g.nz - 1);
    return c;
}

// (B^T B w)(p) * h^2 for one scalar plane w: sum over in-grid neighbours of
// (w(p) - w(neighbour)); homogeneous Neumann boundary.
__device__ __forceinline__ float neg_laplacian_h2(const float* __restrict__ w, const Geom& g,
                                                  long long p, int x, int y, int z) {
    const float c = w[p];
    float acc = 0.f;
    if (x > 0) acc += c - w[p - 1];
    if (x < g.nx - 1) acc += c - w[p + 1];
    if (y > 0) acc += c - w[p - g.nx];
    if (y < g.ny - 1) acc += c - w[p + g.nx];
    if (g.d == 3) {
        const long long s = (long long)g.nx * g.ny;
        if (z > 0) acc += c - w[p - s];
        if (z < g.nz - 1) acc += c - w[p + s];
    }
    return acc;
}

// Sum of squared forward differences (times h^2) from p to its +x, +y (, +z)
// neighbours, each interior edge counted once over the plane.
__device__ __forceinline__ float forward_diff2_h2(const float* __restrict__ w, const Geom& g,
                                                  long long p, int x, int y, int z) {
    const float c = w[p];
    float acc = 0.f;
    if (x < g.nx - 1) { float t = w[p + 1] - c; acc += t * t; }
    if (y < g.ny - 1) { float t = w[p + g.nx] - c; acc += t * t; }
    if (g.d == 3 && z < g.nz - 1) { float t = w[p + (long long)g.nx * g.ny] - c; acc += t * t; }
    return acc;
}

// ------------------------------------------------------------ interpolation
// Index coordinate of a displaced cell centre along one axis, split exactly:
// xi = i + u/h with u/h exact (h is a power of two), i0 = i + floor(u/h),
// f = u/h - floor(u/h) exact in float32.
__device__ __forceinline__ void split_coord(int i, float u, float inv_h, int& i0, float& f) {
    const float t = u * inv_h;
    const bool ok = fabsf(t) < 1.0e7f;   // false for NaN, Inf and absurd: far outside the grid
    const float fl = floorf(ok ? t : 0.f);
    f = ok ? t - fl : 0.f;
    i0 = ok ? i + (int)fl : -1000000000;
}

__device__ __forceinline__ int clampi(int v, int hi) { return min(max(v, 0), hi); }

// The four corners (ix, iy) .. (ix + 1, iy + 1) of a bilinear stencil, zero
// outside the grid.  Branch-free: every load reads a clamped (in-range)
// address and outside corners are zeroed afterwards, so the loads of several
// stencils can all be in flight together.
template <typename TI>
__device__ __forceinline__ void corners2(const TI* __restrict__ T, int nx, int ny, int ix, int iy, float& t00,
                                         float& t01, float& t10, float& t11) {
    const bool x0 = (unsigned)ix < (unsigned)nx, x1 = (unsigned)(ix + 1) < (unsigned)nx;
    const bool y0 = (unsigned)iy < (unsigned)ny, y1 = (unsigned)(iy + 1) < (unsigned)ny;
    const int cx0 = clampi(ix, nx - 1), cx1 = clampi(ix + 1, nx - 1);
    const TI* r0 = T + (long long)clampi(iy, ny - 1) * nx;
    const TI* r1 = T + (long long)clampi(iy + 1, ny - 1) * nx;
    const float v00 = ldf(r0 + cx0), v01 = ldf(r0 + cx1), v10 = ldf(r1 + cx0), v11 = ldf(r1 + cx1);
    t00 = (x0 && y0) ? v00 : 0.f;
    t01 = (x1 && y0) ? v01 : 0.f;
    t10 = (x0 && y1) ? v10 : 0.f;
    t11 = (x1 && y1) ? v11 : 0.f;
}

// Bilinear value and gradient (zero extension) of the level image T at the
// cell centre (x, y) displaced by (uy, ux) physical units.
template <typename TI>
__device__ __forceinline__ void interp2(const TI* __restrict__ T, const Geom& g, int x, int y,
                                        float uy, float ux, float& val, float& gy, float& gx) {
    int iy, ix;
    float fy, fx;
    split_coord(y, uy, g.inv_h, iy, fy);
    split_coord(x, ux, g.inv_h, ix, fx);
    float t00, t01, t10, t11;
    corners2(T, g.nx, g.ny, ix, iy, t00, t01, t10, t11);
    const float a0 = t00 + fx * (t01 - t00);
    const float a1 = t10 + fx * (t11 - t10);
    val = a0 + fy * (a1 - a0);
    gx = g.inv_h * ((t01 - t00) + fy * ((t11 - t10) - (t01 - t00)));
    gy = g.inv_h * (a1 - a0);
}

// Bilinear value only (zero extension).
template <typename TI>
__device__ __forceinline__ float interp2_val(const TI* __restrict__ T, const Geom& g, int x, int y, float uy,
                                             float ux) {
    int iy, ix;
    float fy, fx;
    split_coord(y, uy, g.inv_h, iy, fy);
    split_coord(x, ux, g.inv_h, ix, fx);
    float t00, t01, t10, t11;
    corners2(T, g.nx, g.ny, ix, iy, t00, t01, t10, t11);
    const float a0 = t00 + fx * (t01 - t00);
    const float a1 = t10 + fx * (t11 - t10);
    return a0 + fy * (a1 - a0);
}

// Bilinear values (zero extension) at the cells (x + e, y), e < VEC, of one
// row, displaced by (uy[e], ux[e]).  When every stencil of the warp lies
// inside the image (the common case), the corners are read from one base
// address per value with no per-corner tests; otherwise each value takes the
// general path.  Both paths give identical results.  All lanes of the warp
// must call it.
template <int VEC, typename TI>
__device__ __forceinline__ void interp2_row(const TI* __restrict__ T, const Geom& g, int x, int y,
                                            const float (&uy)[VEC], const float (&ux)[VEC], float (&a)[VEC]) {
    int ix[VEC], iy[VEC];
    float fx[VEC], fy[VEC];
    bool inside = true;
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
        const float ty = uy[e] * g.inv_h, tx = ux[e] * g.inv_h;
        const float fly = floorf(ty), flx = floorf(tx);
        fy[e] = ty - fly;
        fx[e] = tx - flx;
        iy[e] = y + (int)fly;
        ix[e] = x + e + (int)flx;
        inside = inside && fabsf(ty) < 1.0e7f && fabsf(tx) < 1.0e7f && (unsigned)ix[e] < (unsigned)(g.nx - 1) &&
                 (unsigned)iy[e] < (unsigned)(g.ny - 1);
    }
    if (__all_sync(0xffffffffu, inside)) {
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
            const TI* b = T + (iy[e] * g.nx + ix[e]);
            const float t00 = ldf(b), t01 = ldf(b + 1), t10 = ldf(b + g.nx), t11 = ldf(b + g.nx + 1);
            const float a0 = t00 + fx[e] * (t01 - t00);
            const float a1 = t10 + fx[e] * (t11 - t10);
            a[e] = a0 + fy[e] * (a1 - a0);
        }
    } else {
#pragma unroll
        for (int e = 0; e < VEC; ++e) a[e] = interp2_val(T, g, x + e, y, uy[e], ux[e]);
    }
}

// interp2_row with the image gradient (d/dy, d/dx) at the same points, as
// interp2 computes it.
template <int VEC, typename TI>
__device__ __forceinline__ void interp2_row_grad(const TI* __restrict__ T, const Geom& g, int x, int y,
                                                 const float (&uy)[VEC], const float (&ux)[VEC], float (&a)[VEC],
                                                 float (&gy)[VEC], float (&gx)[VEC]) {
    int ix[VEC], iy[VEC];
    float fx[VEC], fy[VEC];
    bool inside = true;
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
        const float ty = uy[e] * g.inv_h, tx = ux[e] * g.inv_h;
        const float fly = floorf(ty), flx = floorf(tx);
        fy[e] = ty - fly;
        fx[e] = tx - flx;
        iy[e] = y + (int)fly;
        ix[e] = x + e + (int)flx;
        inside = inside && fabsf(ty) < 1.0e7f && fabsf(tx) < 1.0e7f && (unsigned)ix[e] < (unsigned)(g.nx - 1) &&
                 (unsigned)iy[e] < (unsigned)(g.ny - 1);
    }
    if (__all_sync(0xffffffffu, inside)) {
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
            const TI* b = T + (iy[e] * g.nx + ix[e]);
            const float t00 = ldf(b), t01 = ldf(b + 1), t10 = ldf(b + g.nx), t11 = ldf(b + g.nx + 1);
            const float a0 = t00 + fx[e] * (t01 - t00);
            const float a1 = t10 + fx[e] * (t11 - t10);
            a[e] = a0 + fy[e] * (a1 - a0);
            gx[e] = g.inv_h * ((t01 - t00) + fy[e] * ((t11 - t10) - (t01 - t00)));
            gy[e] = g.inv_h * (a1 - a0);
        }
    } else {
#pragma unroll
        for (int e = 0; e < VEC; ++e) interp2(T, g, x + e, y, uy[e], ux[e], a[e], gy[e], gx[e]);
    }
}

// The eight corners c[dz][dy][dx] of a trilinear stencil, zero outside;
// branch-free like corners2.
template <typename TI>
__device__ __forceinline__ void corners3(const TI* __restrict__ T, const Geom& g, int ix, int iy, int iz,
                                         float (&c)[2][2][2]) {
    const long long sy = g.nx, sz = (long long)g.nx * g.ny;
    int cx[2], cy[2], cz[2];
    bool bx[2], by[2], bz[2];
#pragma unroll
    for (int o = 0; o < 2; ++o) {
        bx[o] = (unsigned)(ix + o) < (unsigned)g.nx;
        by[o] = (unsigned)(iy + o) < (unsigned)g.ny;
        bz[o] = (unsigned)(iz + o) < (unsigned)g.nz;
        cx[o] = clampi(ix + o, g.nx - 1);
        cy[o] = clampi(iy + o, g.ny - 1);
        cz[o] = clampi(iz + o, g.nz - 1);
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const TI* r = T + cz[a] * sz + cy[q] * sy;
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const float v = ldf(r + cx[e]);
                c[a][q][e] = (bz[a] && by[q] && bx[e]) ? v : 0.f;
            }
        }
}

// Trilinear value only (zero extension), displacement (uz, uy, ux).
template <typename TI>
__device__ __forceinline__ float interp3_val(const TI* __restrict__ T, const Geom& g, int x, int y, int z,
                                             float uz, float uy, float ux) {
    int iz, iy, ix;
    float fz, fy, fx;
    split_coord(z, uz, g.inv_h, iz, fz);
    split_coord(y, uy, g.inv_h, iy, fy);
    split_coord(x, ux, g.inv_h, ix, fx);
    float c[2][2][2];
    corners3(T, g, ix, iy, iz, c);
    float cy[2];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const float c0 = c[a][0][0] + fx * (c[a][0][1] - c[a][0][0]);
        const float c1 = c[a][1][0] + fx * (c[a][1][1] - c[a][1][0]);
        cy[a] = c0 + fy * (c1 - c0);
    }
    return cy[0] + fz * (cy[1] - cy[0]);
}

// Trilinear value and gradient (zero extension), displacement (uz, uy, ux).
template <typename TI>
__device__ __forceinline__ void interp3(const TI* __restrict__ T, const Geom& g, int x, int y, int z,
                                        float uz, float uy, float ux, float& val, float& gz,
                                        float& gy, float& gx) {
    int iz, iy, ix;
    float fz, fy, fx;
    split_coord(z, uz, g.inv_h, iz, fz);
    split_coord(y, uy, g.inv_h, iy, fy);
    split_coord(x, ux, g.inv_h, ix, fx);
    float c[2][2][2];
    corners3(T, g, ix, iy, iz, c);
    // blend along x
    float cx[2][2], dx[2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            dx[a][b] = c[a][b][1] - c[a][b][0];
            cx[a][b] = c[a][b][0] + fx * dx[a][b];
        }
    // along y
    float cy[2], dy[2], dxy[2];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        dy[a] = cx[a][1] - cx[a][0];
        cy[a] = cx[a][0] + fy * dy[a];
        dxy[a] = dx[a][0] + fy * (dx[a][1] - dx[a][0]);
    }
    val = cy[0] + fz * (cy[1] - cy[0]);
    gz = g.inv_h * (cy[1] - cy[0]);
    gy = g.inv_h * (dy[0] + fz * (dy[1] - dy[0]));
    gx = g.inv_h * (dxy[0] + fz * (dxy[1] - dxy[0]));
}

// ------------------------------------------------------------ reductions
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Double-float ("double-word") numbers hi + lo with |lo| <= ulp(hi) / 2 and
// their accurate addition from error-free transformations (TwoSum, Knuth;
// Fast2Sum, Dekker; the accurate double-word sum analysed by Joldes, Muller
// and Popescu, 2017): about 44 significant bits from FP32 instructions only.
// The reductions use it in place of FP64 arithmetic, whose instructions are
// far slower than FP32 ones on this GPU.
struct dfloat {
    float hi, lo;
};

__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
    const float s = a + b;
    const float ap = s - b;
    const float bp = s - ap;
    return {s, (a - ap) + (b - bp)};
}

__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b) {   // |a| >= |b| or a == 0
    const float s = a + b;
    return {s, b - (s - a)};
}

__device__ __forceinline__ dfloat df_add(dfloat x, dfloat y) {
    const dfloat s = df_two_sum(x.hi, y.hi);
    const dfloat t = df_two_sum(x.lo, y.lo);
    const dfloat v = df_fast_two_sum(s.hi, s.lo + t.hi);
    return df_fast_two_sum(v.hi, t.lo + v.lo);
}

__device__ __forceinline__ dfloat df_shfl_xor(dfloat v, int o) {
    return {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}

// Stage 1 of a grid reduction: the CTA total of each of NV float values
// (fixed butterfly inside a warp, then warp order in double-float), stored as
// (hi, lo) at part[block * NV + i].  Threads 0..NV-1 write; all threads of
// the CTA must call it.
template <int NV>
__device__ __forceinline__ void cta_partials(const float (&val)[NV], float2* __restrict__ part, unsigned block) {
    static_assert(NV <= 32, "at most 32 values");
    __shared__ float s_warp[kThreads / 32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        const float w = warp_sum(val[i]);
        if (lane == 0) s_warp[warp][i] = w;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        const int i = threadIdx.x;
        dfloat s = {s_warp[0][i], 0.f};
        for (int w = 1; w < nwarps; ++w) s = df_add(s, dfloat{s_warp[w][i], 0.f});
        part[(size_t)block * NV + i] = make_float2(s.hi, s.lo);
    }
}

// Stage 2: the sum over nblocks CTA totals in a fixed order (thread-strided
// double-float sums, a fixed butterfly, then warp order); every thread gets
// the totals.  All threads of the CTA must call it.
template <int NV>
__device__ __forceinline__ void cta_total(const float2* __restrict__ part, unsigned nblocks, dfloat (&tot)[NV]) {
    __shared__ dfloat s_w2[kThreads / 32][NV];
    __shared__ dfloat s_tot[NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        dfloat s = {0.f, 0.f};
        for (unsigned b = threadIdx.x; b < nblocks; b += blockDim.x) {
            const float2 q = __ldcg(part + (size_t)b * NV + i);
            s = df_add(s, dfloat{q.x, q.y});
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s = df_add(s, df_shfl_xor(s, o));
        if (lane == 0) s_w2[warp][i] = s;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        const int i = threadIdx.x;
        dfloat s = s_w2[0][i];
        for (int w = 1; w < nwarps; ++w) s = df_add(s, s_w2[w][i]);
        s_tot[i] = s;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NV; ++i) tot[i] = s_tot[i];
    __syncthreads();
}

// Two-stage deterministic reduction of NV values over the whole grid.
//
// Stage 1: every thread holds float partials over its few elements; a warp
// sums them in float with a fixed butterfly, the warp totals are summed in
// double-float in warp order and the CTA total goes to the partials buffer.
// Stage 2: the CTA that arrives last (an integer ticket, no float atomics)
// sums all CTA totals in double-float in a fixed order and writes out[0..NV)
// (as double, from thread 0).  The result depends only on the launch shape,
// never on scheduling.  Returns true in every thread of the last CTA (so it
// may finish the step).  `partials` holds one 8-byte slot per CTA and value.
template <int NV>
__device__ __forceinline__ bool grid_reduce(const float (&val)[NV], double* __restrict__ partials,
                                            unsigned int* ticket, double* out) {
    __shared__ bool s_last;
    float2* part = reinterpret_cast<float2*>(partials);
    const unsigned nblocks = gridDim.x * gridDim.y * gridDim.z;
    const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    cta_partials<NV>(val, part, bid);
    if (threadIdx.x < 32) {
        __threadfence();   // the CTA totals (written by lanes 0..NV-1) before the ticket
        if (threadIdx.x == 0) s_last = atomicAdd(ticket, 1u) == nblocks - 1;
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    dfloat tot[NV];
    cta_total<NV>(part, nblocks, tot);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) out[i] = (double)tot[i].hi + (double)tot[i].lo;
        *ticket = 0u;
    }
    __syncthreads();
    return true;
}

}  // namespace stml
