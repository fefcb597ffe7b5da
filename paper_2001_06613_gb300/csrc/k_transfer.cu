// Spatial transfer operators, temporal predictors, frame gather/scatter and
// the frame-correlation diagnostic.
//
// * restriction: 2^d block mean (Sec. 3; Sec. 4 smooths in space only);
// * prolongation P: cell-centred multilinear interpolation, clamp-to-edge,
//   and its transpose P^T as a gather with a fixed order (no atomics);
// * linear temporal predictor (Sec. 3) and the least-squares predictor of
//   eq. (2) solved by Thomas' algorithm (one factorisation for all series).
#include <atomic>
#include <map>
#include <mutex>
#include <utility>

#include "kernels.h"

namespace stml {

static std::atomic<long long> g_launches{0};
long long launches_total() { return g_launches.load(); }
void count_launches(int k) { g_launches.fetch_add(k); }

namespace {
std::mutex g_cache_mu;
// keyed by (device ordinal, kernel): occupancy and attributes are per device
std::map<std::pair<int, const void*>, unsigned> g_resident;
std::map<std::pair<int, const void*>, int> g_smem_attr;
std::map<int, int> g_sms;
}  // namespace

int device_sms() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lock(g_cache_mu);
    const auto it = g_sms.find(dev);
    if (it != g_sms.end()) return it->second;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 0;
    if (sms > 0) g_sms.emplace(dev, sms);
    return sms;
}

cudaError_t set_max_dynamic_smem(const void* kernel, int bytes) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_cache_mu);
    const auto key = std::make_pair(dev, kernel);
    const auto it = g_smem_attr.find(key);
    if (it != g_smem_attr.end() && it->second >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) g_smem_attr[key] = bytes;
    return e;
}

unsigned resident_grid(const void* kernel, long long items, unsigned cap) {
    unsigned n = 0;
    const int sms = device_sms();
    int dev = 0;
    const bool have_dev = cudaGetDevice(&dev) == cudaSuccess;
    {
        std::lock_guard<std::mutex> lock(g_cache_mu);
        const auto key = std::make_pair(have_dev ? dev : -1, kernel);
        auto it = g_resident.find(key);
        if (it != g_resident.end()) {
            n = it->second;
        } else {
            int per_sm = 0;
            if (have_dev && sms > 0 &&
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0) == cudaSuccess &&
                per_sm > 0) {
                n = (unsigned)(sms * per_sm);
                g_resident.emplace(key, n);
            } else {
                n = cap;   // the query failed: the caller's cap (the launch reports any real error)
            }
        }
    }
    if (n > cap) n = cap;
    if ((long long)n > items) n = (unsigned)(items > 0 ? items : 1);
    return n;
}

Geom make_geom(const int shape3[3], int d, float h) {
    Geom g;
    g.nz = shape3[0];
    g.ny = shape3[1];
    g.nx = shape3[2];
    g.d = d;
    g.N = (long long)g.nx * g.ny * g.nz;
    g.h = h;
    g.inv_h = 1.0f / h;
    g.hd = d == 3 ? h * h * h : h * h;
    return g;
}

static inline unsigned grid1d(long long n, int threads, long long cap = 1 << 20) {
    return blocks_for(n, threads, cap);
}

// ---------------------------------------------------------------- restriction
// 2^d block mean in float of stored values; the result is stored in the same
// type (rounded to nearest even for 16-bit storage).
template <typename TI>
__global__ void restrict_kernel(const TI* __restrict__ fine, TI* __restrict__ coarse,
                                long long total, Geom gc) {
    const int fx = 2 * gc.nx, fy = 2 * gc.ny;
    const long long Nf = gc.N * (gc.d == 3 ? 8 : 4);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long plane = e / gc.N;
        const long long pc = e - plane * gc.N;
        int x, y, z;
        unflatten(gc, pc, x, y, z);
        const TI* F = fine + plane * Nf;
        float s;
        if (gc.d == 2) {
            const long long b = (long long)(2 * y) * fx + 2 * x;
            s = (ldf(F + b) + ldf(F + b + 1)) + (ldf(F + b + fx) + ldf(F + b + fx + 1));
            s *= 0.25f;
        } else {
            const long long b = ((long long)(2 * z) * fy + 2 * y) * fx + 2 * x;
            const long long sz = (long long)fx * fy;
            s = ((ldf(F + b) + ldf(F + b + 1)) + (ldf(F + b + fx) + ldf(F + b + fx + 1))) +
                ((ldf(F + b + sz) + ldf(F + b + sz + 1)) + (ldf(F + b + sz + fx) + ldf(F + b + sz + fx + 1)));
            s *= 0.125f;
        }
        stf(coarse + e, s);
    }
}

cudaError_t launch_restrict(const void* fine, void* coarse, int type, int planes, const Geom& gc,
                            cudaStream_t s) {
    const long long total = (long long)planes * gc.N;
    if (total == 0) return cudaSuccess;
    with_store_type(type, [&](auto tag) {
        using TI = decltype(tag);
        restrict_kernel<TI><<<grid1d(total, kThreads), kThreads, 0, s>>>(static_cast<const TI*>(fine),
                                                                          static_cast<TI*>(coarse), total, gc);
        return 0;
    });
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- storage conversion
template <typename TI>
__global__ void to_store_kernel(const float* __restrict__ src, TI* __restrict__ dst, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        stf(dst + i, src[i]);
}

template <typename TI>
__global__ void from_store_kernel(const TI* __restrict__ src, float* __restrict__ dst, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = ldf(src + i);
}

cudaError_t launch_to_store(const float* src, void* dst, int type, long long n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    with_store_type(type, [&](auto tag) {
        using TI = decltype(tag);
        to_store_kernel<TI><<<grid1d(n, kThreads), kThreads, 0, s>>>(src, static_cast<TI*>(dst), n);
        return 0;
    });
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_from_store(const void* src, int type, float* dst, long long n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    with_store_type(type, [&](auto tag) {
        using TI = decltype(tag);
        from_store_kernel<TI><<<grid1d(n, kThreads), kThreads, 0, s>>>(static_cast<const TI*>(src), dst, n);
        return 0;
    });
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- prolongation
// Fine index j on an axis of m coarse cells: centre at coarse coordinate
// j/2 - 1/4, blended from coarse cells lo and hi (clamped) with weights wl, wh.
__device__ __forceinline__ void prolong_taps(int j, int m, int& lo, int& hi, float& wl, float& wh) {
    const int i = j >> 1;
    if ((j & 1) == 0) {
        lo = i - 1 < 0 ? 0 : i - 1;
        hi = i;
        wl = 0.25f;
        wh = 0.75f;
    } else {
        lo = i;
        hi = i + 1 > m - 1 ? m - 1 : i + 1;
        wl = 0.75f;
        wh = 0.25f;
    }
}

__global__ void prolong_kernel(const float* __restrict__ coarse, float* __restrict__ fine,
                               long long total, Geom gc) {
    const int fx = 2 * gc.nx, fy = 2 * gc.ny, fz = gc.d == 3 ? 2 * gc.nz : 1;
    const long long Nf = (long long)fx * fy * fz;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long plane = e / Nf;
        long long pf = e - plane * Nf;
        const int x = (int)(pf % fx);
        const int y = (int)((pf / fx) % fy);
        const int z = (int)(pf / ((long long)fx * fy));
        const float* C = coarse + plane * gc.N;
        int xl, xh, yl, yh;
        float wxl, wxh, wyl, wyh;
        prolong_taps(x, gc.nx, xl, xh, wxl, wxh);
        prolong_taps(y, gc.ny, yl, yh, wyl, wyh);
        float v;
        if (gc.d == 2) {
            const float r0 = wxl * C[(long long)yl * gc.nx + xl] + wxh * C[(long long)yl * gc.nx + xh];
            const float r1 = wxl * C[(long long)yh * gc.nx + xl] + wxh * C[(long long)yh * gc.nx + xh];
            v = wyl * r0 + wyh * r1;
        } else {
            int zl, zh;
            float wzl, wzh;
            prolong_taps(z, gc.nz, zl, zh, wzl, wzh);
            auto row = [&](int zz, int yy) {
                const float* R = C + ((long long)zz * gc.ny + yy) * gc.nx;
                return wxl * R[xl] + wxh * R[xh];
            };
            const float s0 = wyl * row(zl, yl) + wyh * row(zl, yh);
            const float s1 = wyl * row(zh, yl) + wyh * row(zh, yh);
            v = wzl * s0 + wzh * s1;
        }
        fine[e] = v;
    }
}

cudaError_t launch_prolong(const float* coarse, float* fine, int planes, const Geom& gc,
                           cudaStream_t s) {
    const long long total = (long long)planes * gc.N * (gc.d == 3 ? 8 : 4);
    if (total == 0) return cudaSuccess;
    prolong_kernel<<<grid1d(total, kThreads), kThreads, 0, s>>>(coarse, fine, total, gc);
    count_launches(1);
    return cudaGetLastError();
}

// Weight with which fine index j contributes to coarse index i (one axis).
__device__ __forceinline__ float prolong_weight(int j, int i, int m) {
    int lo, hi;
    float wl, wh;
    prolong_taps(j, m, lo, hi, wl, wh);
    return (lo == i ? wl : 0.f) + (hi == i ? wh : 0.f);
}

// P^T: coarse cell i gathers fine cells 2i-1 .. 2i+2 (those inside the grid)
// along every axis, in increasing order.
__global__ void prolong_adjoint_kernel(const float* __restrict__ fine, float* __restrict__ coarse,
                                       long long total, Geom gc) {
    const int fx = 2 * gc.nx, fy = 2 * gc.ny, fz = gc.d == 3 ? 2 * gc.nz : 1;
    const long long Nf = (long long)fx * fy * fz;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long plane = e / gc.N;
        const long long pc = e - plane * gc.N;
        int x, y, z;
        unflatten(gc, pc, x, y, z);
        const float* F = fine + plane * Nf;
        const int z0 = gc.d == 3 ? max(0, 2 * z - 1) : 0, z1 = gc.d == 3 ? min(fz - 1, 2 * z + 2) : 0;
        const int y0 = max(0, 2 * y - 1), y1 = min(fy - 1, 2 * y + 2);
        const int x0 = max(0, 2 * x - 1), x1 = min(fx - 1, 2 * x + 2);
        float acc = 0.f;
        for (int jz = z0; jz <= z1; ++jz) {
            const float wz = gc.d == 3 ? prolong_weight(jz, z, gc.nz) : 1.f;
            if (wz == 0.f) continue;
            for (int jy = y0; jy <= y1; ++jy) {
                const float wy = prolong_weight(jy, y, gc.ny);
                if (wy == 0.f) continue;
                const float* R = F + ((long long)jz * fy + jy) * fx;
                float row = 0.f;
                for (int jx = x0; jx <= x1; ++jx) row += prolong_weight(jx, x, gc.nx) * R[jx];
                acc += wz * wy * row;
            }
        }
        coarse[e] = acc;
    }
}

cudaError_t launch_prolong_adjoint(const float* fine, float* coarse, int planes, const Geom& gc,
                                   cudaStream_t s) {
    const long long total = (long long)planes * gc.N;
    if (total == 0) return cudaSuccess;
    prolong_adjoint_kernel<<<grid1d(total, kThreads), kThreads, 0, s>>>(fine, coarse, total, gc);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- predictors
__global__ void predict_linear_kernel(const float* __restrict__ in, float* __restrict__ out,
                                      const LinTap* __restrict__ taps, size_t plane) {
    const LinTap tp = taps[blockIdx.y];
    const float* L = in + (size_t)tp.src_l * plane;
    const float* R = in + (size_t)tp.src_r * plane;
    float* O = out + (size_t)tp.dst * plane;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < plane;
         e += (size_t)gridDim.x * blockDim.x) {
        O[e] = tp.wr == 0.f ? L[e] : tp.wl * L[e] + tp.wr * R[e];
    }
}

cudaError_t launch_predict_linear(const float* in, float* out, const LinTap* taps, int nT,
                                  size_t plane_elems, cudaStream_t s) {
    if (nT == 0 || plane_elems == 0) return cudaSuccess;
    dim3 grid(grid1d((long long)plane_elems, kThreads, 4096), nT);
    predict_linear_kernel<<<grid, kThreads, 0, s>>>(in, out, taps, plane_elems);
    count_launches(1);
    return cudaGetLastError();
}

// One thread per (pixel, component) series.  Forward elimination stores the
// modified right-hand side in zeta (it is overwritten by the back
// substitution), so no scratch beyond the output is used.
__global__ void predict_ls_kernel(const float* __restrict__ eta, const float* __restrict__ omega,
                                  float* __restrict__ zeta, const float* __restrict__ cp,
                                  const float* __restrict__ inv_den, const float* __restrict__ sub,
                                  const int* __restrict__ kidx, int n, size_t ncomp) {
    for (size_t col = blockIdx.x * (size_t)blockDim.x + threadIdx.x; col < ncomp;
         col += (size_t)gridDim.x * blockDim.x) {
        float dp = 0.f;
        for (int t = 0; t < n; ++t) {
            const int ki = __ldg(kidx + t);
            const float rhs = ki >= 0 ? eta[(size_t)ki * ncomp + col] - omega[(size_t)t * ncomp + col] : 0.f;
            dp = (rhs - __ldg(sub + t) * dp) * __ldg(inv_den + t);
            zeta[(size_t)t * ncomp + col] = dp;
        }
        float x = dp;
        zeta[(size_t)(n - 1) * ncomp + col] = omega[(size_t)(n - 1) * ncomp + col] + x;
        for (int t = n - 2; t >= 0; --t) {
            x = zeta[(size_t)t * ncomp + col] - __ldg(cp + t) * x;
            zeta[(size_t)t * ncomp + col] = omega[(size_t)t * ncomp + col] + x;
        }
    }
}

cudaError_t launch_predict_ls(const float* eta, const float* omega, float* zeta, const float* cp,
                              const float* inv_den, const float* sub, const int* kidx, int n,
                              size_t ncomp, cudaStream_t s) {
    if (ncomp == 0 || n == 0) return cudaSuccess;
    predict_ls_kernel<<<grid1d((long long)ncomp, kThreads), kThreads, 0, s>>>(
        eta, omega, zeta, cp, inv_den, sub, kidx, n, ncomp);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- gather / scatter
__global__ void gather_planes_kernel(const float4* __restrict__ src, float4* __restrict__ dst,
                                     const int* __restrict__ idx, size_t plane4) {
    const int j = blockIdx.y;
    const float4* S = src + (size_t)idx[j] * plane4;
    float4* D = dst + (size_t)j * plane4;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < plane4;
         e += (size_t)gridDim.x * blockDim.x)
        D[e] = S[e];
}

__global__ void scatter_planes_kernel(const float4* __restrict__ src, float4* __restrict__ dst,
                                      const int* __restrict__ idx, size_t plane4) {
    const int j = blockIdx.y;
    const float4* S = src + (size_t)j * plane4;
    float4* D = dst + (size_t)idx[j] * plane4;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < plane4;
         e += (size_t)gridDim.x * blockDim.x)
        D[e] = S[e];
}

__global__ void gather_planes_scalar(const float* __restrict__ src, float* __restrict__ dst,
                                     const int* __restrict__ idx, size_t plane, int scatter) {
    const int j = blockIdx.y;
    const float* S = src + (size_t)(scatter ? j : idx[j]) * plane;
    float* D = dst + (size_t)(scatter ? idx[j] : j) * plane;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < plane;
         e += (size_t)gridDim.x * blockDim.x)
        D[e] = S[e];
}

static cudaError_t planes_copy(const float* src, float* dst, const int* idx, int nK, size_t plane,
                               cudaStream_t s, int scatter) {
    if (nK == 0 || plane == 0) return cudaSuccess;
    const bool vec = (plane % 4 == 0) && ((uintptr_t)src % 16 == 0) && ((uintptr_t)dst % 16 == 0);
    if (vec) {
        dim3 grid(grid1d((long long)(plane / 4), kThreads, 2048), nK);
        if (scatter)
            scatter_planes_kernel<<<grid, kThreads, 0, s>>>((const float4*)src, (float4*)dst, idx, plane / 4);
        else
            gather_planes_kernel<<<grid, kThreads, 0, s>>>((const float4*)src, (float4*)dst, idx, plane / 4);
    } else {
        dim3 grid(grid1d((long long)plane, kThreads, 2048), nK);
        gather_planes_scalar<<<grid, kThreads, 0, s>>>(src, dst, idx, plane, scatter);
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_gather_planes(const float* src, float* dst, const int* idx, int nK,
                                 size_t plane_elems, cudaStream_t s) {
    return planes_copy(src, dst, idx, nK, plane_elems, s, 0);
}

cudaError_t launch_scatter_planes(const float* src, float* dst, const int* idx, int nK,
                                  size_t plane_elems, cudaStream_t s) {
    return planes_copy(src, dst, idx, nK, plane_elems, s, 1);
}

// ---------------------------------------------------------------- correlation
// One CTA per consecutive pair (k, k+1); sums in double, fixed order.
template <typename TI>
__global__ void corr_kernel(const TI* __restrict__ img, long long N, double* __restrict__ rho) {
    const int k = blockIdx.x;
    const TI* A = img + (size_t)k * N;
    const TI* B = A + N;
    double s[5] = {0, 0, 0, 0, 0};
    for (long long i = threadIdx.x; i < N; i += blockDim.x) {
        const double a = ldf(A + i), b = ldf(B + i);
        s[0] += a;
        s[1] += b;
        s[2] += a * a;
        s[3] += b * b;
        s[4] += a * b;
    }
    __shared__ double sh[kThreads / 32][5];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        double v = warp_sum_d(s[i]);
        if (lane == 0) sh[warp][i] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[5] = {0, 0, 0, 0, 0};
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            for (int i = 0; i < 5; ++i) t[i] += sh[w][i];
        const double ma = t[0] / N, mb = t[1] / N;
        const double cab = t[4] - N * ma * mb;
        const double caa = t[2] - N * ma * ma;
        const double cbb = t[3] - N * mb * mb;
        rho[k] = cab / sqrt(caa * cbb);
    }
}

cudaError_t launch_corr_coeff(const void* img, int type, int n, long long N, double* rho_dev, cudaStream_t s) {
    if (n < 2) return cudaSuccess;
    with_store_type(type, [&](auto tag) {
        using TI = decltype(tag);
        corr_kernel<TI><<<n - 1, kThreads, 0, s>>>(static_cast<const TI*>(img), N, rho_dev);
        return 0;
    });
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace stml
