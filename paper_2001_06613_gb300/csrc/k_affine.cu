// Affine-linear transformations per frame (Sec. 4) for the L-BFGS solver of
// Sec. 2: the displacement of frame k is u_k(x) = W_k (x - c) / rho + b_k,
// x the cell centre in finest-level pixel units, c the domain centre and rho
// half of its largest extent; theta_k = (W_k row by row, b_k), d (d + 1)
// values.  The objective and its field gradient come from the registration's
// own objective and gradient passes on the field these kernels write; the
// projection below turns the field gradient into dJ/dtheta.
#include "kernels.h"

namespace stml {

namespace {

// (x - c) / rho of the cell with indices (iz, iy, ix): component i of xhat
// belongs to array axis i (z, y, x in 3-D; y, x in 2-D).
template <int D>
__device__ __forceinline__ void cell_xhat(const Geom& g, const AffineFrame& af, long long p, float (&xh)[D]) {
    const int ix = (int)(p % g.nx);
    const long long q = p / g.nx;
    const int iy = (int)(q % g.ny);
    const int iz = (int)(q / g.ny);
    const float xs[3] = {((float)iz + 0.5f) * g.h, ((float)iy + 0.5f) * g.h, ((float)ix + 0.5f) * g.h};
#pragma unroll
    for (int i = 0; i < D; ++i) xh[i] = (xs[3 - D + i] - af.c[i]) * af.inv_rho;
}

template <int D>
__global__ void affine_field_kernel(Geom g, AffineFrame af, const float* __restrict__ theta, int nK,
                                    float* __restrict__ u) {
    constexpr int P = D * (D + 1);
    const int k = blockIdx.y;
    if (k >= nK) return;
    float th[P];
#pragma unroll
    for (int j = 0; j < P; ++j) th[j] = theta[k * P + j];
    float* uk = u + (size_t)k * D * g.N;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < g.N;
         p += (long long)gridDim.x * blockDim.x) {
        float xh[D];
        cell_xhat<D>(g, af, p, xh);
#pragma unroll
        for (int c = 0; c < D; ++c) {
            float v = th[D * D + c];
#pragma unroll
            for (int i = 0; i < D; ++i) v = fmaf(th[c * D + i], xh[i], v);
            uk[(size_t)c * g.N + p] = v;
        }
    }
}

// Per-CTA sums of g_{k,c}(x) xhat_i(x) and g_{k,c}(x) (FP32 per thread over
// its few cells, FP64 across the CTA), written to part[k][block][P].
template <int D>
__global__ void __launch_bounds__(256) affine_project_kernel(Geom g, AffineFrame af, const float* __restrict__ gu,
                                                             int nK, double* __restrict__ part) {
    constexpr int P = D * (D + 1);
    __shared__ double red[8][P];
    const int k = blockIdx.y;
    float acc[P];
#pragma unroll
    for (int j = 0; j < P; ++j) acc[j] = 0.f;
    const float* gk = gu + (size_t)k * D * g.N;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < g.N;
         p += (long long)gridDim.x * blockDim.x) {
        float xh[D];
        cell_xhat<D>(g, af, p, xh);
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const float gc = gk[(size_t)c * g.N + p];
#pragma unroll
            for (int i = 0; i < D; ++i) acc[c * D + i] = fmaf(gc, xh[i], acc[c * D + i]);
            acc[D * D + c] += gc;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < P; ++j) {
        double v = (double)acc[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][j] = v;
    }
    __syncthreads();
    if (threadIdx.x < P) {
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v += red[w][threadIdx.x];
        part[((size_t)k * gridDim.x + blockIdx.x) * P + threadIdx.x] = v;
    }
}

__global__ void affine_project_sum_kernel(const double* __restrict__ part, int blocks, int P,
                                          double* __restrict__ out) {
    const int k = blockIdx.x;
    for (int j = threadIdx.x; j < P; j += blockDim.x) {
        double v = 0.0;
        for (int b = 0; b < blocks; ++b) v += part[((size_t)k * blocks + b) * P + j];
        out[(size_t)k * P + j] = v;
    }
}

}  // namespace

int affine_project_blocks(const Geom& g) {
    long long b = (g.N + 256 * 8 - 1) / (256 * 8);
    if (b < 1) b = 1;
    if (b > 256) b = 256;
    return (int)b;
}

cudaError_t launch_affine_field(const Geom& g, const AffineFrame& af, const float* theta, int nK, float* u,
                                cudaStream_t s) {
    if (nK <= 0) return cudaErrorInvalidValue;
    long long bx = (g.N + 255) / 256;
    if (bx > 1024) bx = 1024;
    dim3 grid((unsigned)bx, (unsigned)nK);
    if (g.d == 2)
        affine_field_kernel<2><<<grid, 256, 0, s>>>(g, af, theta, nK, u);
    else
        affine_field_kernel<3><<<grid, 256, 0, s>>>(g, af, theta, nK, u);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_affine_project(const Geom& g, const AffineFrame& af, const float* gu, int nK, double* part,
                                  double* out, cudaStream_t s) {
    if (nK <= 0) return cudaErrorInvalidValue;
    const int blocks = affine_project_blocks(g);
    const int P = g.d * (g.d + 1);
    dim3 grid((unsigned)blocks, (unsigned)nK);
    if (g.d == 2)
        affine_project_kernel<2><<<grid, 256, 0, s>>>(g, af, gu, nK, part);
    else
        affine_project_kernel<3><<<grid, 256, 0, s>>>(g, af, gu, nK, part);
    affine_project_sum_kernel<<<nK, 32, 0, s>>>(part, blocks, P, out);
    count_launches(2);
    return cudaGetLastError();
}

}  // namespace stml

// ------------------------------------------- normalised-correlation distance
// D_NC = 1/2 sum_{i,j in K} (1 - rho_ij^2), rho_ij the correlation of the
// warped frames a_i = T_i o y_i over the grid (the reading of the SqN distance
// of Sec. 2): the warped frames and grad T (nc_warp), their Gram matrix about
// the frame means (nc_gram), and dD/du_i(x) = (sum_j Q_ij (a_j(x) - mu_j))
// grad T_i(x) for the K x K matrix Q the host forms from the Gram matrix.
namespace stml {
namespace {

template <int D, typename TI>
__global__ void __launch_bounds__(256) nc_warp_kernel(const TI* __restrict__ T, Geom g, FrameSet fs,
                                                      const float* __restrict__ u, float* __restrict__ a,
                                                      float* __restrict__ dT, double* __restrict__ part) {
    __shared__ double red[8][2];
    const int i = blockIdx.y;
    const int k = fs.frames[i];
    const TI* Tk = T + (size_t)k * g.N;
    const float* ui = u + (size_t)i * D * g.N;
    double s1 = 0.0, s2 = 0.0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < g.N;
         p += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(p % g.nx);
        const long long q = p / g.nx;
        const int y = (int)(q % g.ny);
        float v, gr[3] = {0.f, 0.f, 0.f};
        if constexpr (D == 2) {
            interp2(Tk, g, x, y, ui[p], ui[g.N + p], v, gr[0], gr[1]);
        } else {
            const int z = (int)(q / g.ny);
            interp3(Tk, g, x, y, z, ui[p], ui[g.N + p], ui[2 * g.N + p], v, gr[0], gr[1], gr[2]);
        }
        a[(size_t)i * g.N + p] = v;
#pragma unroll
        for (int c = 0; c < D; ++c) dT[((size_t)i * D + c) * g.N + p] = gr[c];
        s1 += v;
        s2 += (double)v * v;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) {
        red[warp][0] = s1;
        red[warp][1] = s2;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v += red[w][threadIdx.x];
        part[((size_t)i * gridDim.x + blockIdx.x) * 2 + threadIdx.x] = v;
    }
}

// mu_i = (sum over the CTA partials of frame i) / N, in a fixed order.
__global__ void nc_mean_kernel(const double* __restrict__ part, int blocks, long long N, float* __restrict__ mu) {
    const int i = blockIdx.x;
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int b = 0; b < blocks; ++b) v += part[((size_t)i * blocks + b) * 2];
        mu[i] = (float)(v / (double)N);
    }
}

// Partial Gram matrix of the centred frames over one slice of pixels:
// part[s][i][j] for a 16 x 16 tile of (i, j); FP32 over 64-pixel steps,
// FP64 across steps.
__global__ void __launch_bounds__(256) nc_gram_kernel(const float* __restrict__ a, const float* __restrict__ mu,
                                                      int nK, long long N, long long chunk,
                                                      double* __restrict__ part) {
    __shared__ float si[16][65], sj[16][65];
    const int ti = threadIdx.x >> 4, tj = threadIdx.x & 15;
    const int i0 = blockIdx.x * 16, j0 = blockIdx.y * 16;
    const long long pb = (long long)blockIdx.z * chunk;
    const long long pe = pb + chunk < N ? pb + chunk : N;
    double acc = 0.0;
    for (long long p0 = pb; p0 < pe; p0 += 64) {
        for (int t = threadIdx.x; t < 16 * 64; t += 256) {
            const int r = t >> 6, col = t & 63;
            const long long p = p0 + col;
            const bool okp = p < pe;
            const int fi = i0 + r, fj = j0 + r;
            si[r][col] = (okp && fi < nK) ? a[(size_t)fi * N + p] - mu[fi] : 0.f;
            sj[r][col] = (okp && fj < nK) ? a[(size_t)fj * N + p] - mu[fj] : 0.f;
        }
        __syncthreads();
        float s = 0.f;
#pragma unroll 16
        for (int col = 0; col < 64; ++col) s = fmaf(si[ti][col], sj[tj][col], s);
        acc += (double)s;
        __syncthreads();
    }
    const int i = i0 + ti, j = j0 + tj;
    if (i < nK && j < nK) part[((size_t)blockIdx.z * nK + i) * nK + j] = acc;
}

__global__ void nc_gram_sum_kernel(const double* __restrict__ part, int splits, int nK, double* __restrict__ G) {
    const long long n = (long long)nK * nK;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int s = 0; s < splits; ++s) v += part[(size_t)s * n + e];
        G[e] = v;
    }
}

// g_u[i][c](x) = (sum_j Q[i][j] (a_j(x) - mu_j)) dT[i][c](x) for a tile of 16
// frames i per CTA row, one pixel per thread.
template <int D>
__global__ void __launch_bounds__(256) nc_grad_kernel(const float* __restrict__ a, const float* __restrict__ mu,
                                                      const float* __restrict__ Q, const float* __restrict__ dT,
                                                      int nK, long long N, float* __restrict__ gu) {
    extern __shared__ float sq[];        // [16][nK]
    const int i0 = blockIdx.y * 16;
    for (int t = threadIdx.x; t < 16 * nK; t += blockDim.x) {
        const int r = t / nK, j = t - r * nK;
        sq[t] = (i0 + r < nK) ? Q[(size_t)(i0 + r) * nK + j] : 0.f;
    }
    __syncthreads();
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
        float v[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = 0.f;
        for (int j = 0; j < nK; ++j) {
            const float aj = a[(size_t)j * N + p] - mu[j];
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = fmaf(sq[r * nK + j], aj, v[r]);
        }
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const int i = i0 + r;
            if (i >= nK) break;
#pragma unroll
            for (int c = 0; c < D; ++c) gu[((size_t)i * D + c) * N + p] = v[r] * dT[((size_t)i * D + c) * N + p];
        }
    }
}

// Row i of rho = G_ij / (n_i n_j): srow[i] = sum_j rho_ij^2 (FP64, fixed
// order) and Q_ij = -(2 / n_i) (rho_ij / n_j - delta_ij srow_i / n_i).
__global__ void __launch_bounds__(128) nc_coeff_kernel(const double* __restrict__ G, int nK, double* __restrict__ srow,
                                                       float* __restrict__ Q) {
    __shared__ double red[4];
    const int i = blockIdx.x;
    const double ni = sqrt(G[(size_t)i * nK + i]);
    double s = 0.0;
    for (int j = threadIdx.x; j < nK; j += blockDim.x) {
        const double nj = sqrt(G[(size_t)j * nK + j]);
        const double r = G[(size_t)i * nK + j] / (ni * nj);
        s += r * r;
        Q[(size_t)i * nK + j] = (float)(-(2.0 / ni) * (r / nj));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        const double si = red[0] + red[1] + red[2] + red[3];
        srow[i] = si;
        const double r_ii = G[(size_t)i * nK + i] / (ni * ni);
        Q[(size_t)i * nK + i] = (float)(-(2.0 / ni) * (r_ii / ni - si / ni));
    }
}

// D_NC = 1/2 (K^2 - sum_i srow_i), summed in row order.
__global__ void nc_d_kernel(const double* __restrict__ srow, int nK, double* __restrict__ D) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < nK; ++i) s += srow[i];
        *D = 0.5 * ((double)nK * nK - s);
    }
}

}  // namespace

cudaError_t launch_nc_coeff(const double* G, int nK, double* srow, float* Q, double* D, cudaStream_t s) {
    nc_coeff_kernel<<<nK, 128, 0, s>>>(G, nK, srow, Q);
    nc_d_kernel<<<1, 32, 0, s>>>(srow, nK, D);
    count_launches(2);
    return cudaGetLastError();
}

int nc_gram_splits(const Geom& g, int nK) {
    const long long tiles = (long long)((nK + 15) / 16) * ((nK + 15) / 16);
    long long s = (4 * 152 + tiles - 1) / tiles;
    const long long max_s = (g.N + 63) / 64;
    if (s > max_s) s = max_s;
    if (s > 64) s = 64;
    return (int)(s < 1 ? 1 : s);
}

cudaError_t launch_nc_warp(const Stored& T, const Geom& g, const FrameSet& fs, const float* u, float* a, float* dT,
                           double* part, float* mu, cudaStream_t s) {
    long long bx = (g.N + 255) / 256;
    if (bx > 256) bx = 256;
    dim3 grid((unsigned)bx, (unsigned)fs.nK);
    with_store_type(T.type, [&](auto tag) {
        using TI = decltype(tag);
        const TI* Tp = static_cast<const TI*>(T.p);
        if (g.d == 2)
            nc_warp_kernel<2, TI><<<grid, 256, 0, s>>>(Tp, g, fs, u, a, dT, part);
        else
            nc_warp_kernel<3, TI><<<grid, 256, 0, s>>>(Tp, g, fs, u, a, dT, part);
        return 0;
    });
    nc_mean_kernel<<<fs.nK, 32, 0, s>>>(part, (int)bx, g.N, mu);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_nc_gram(const Geom& g, const float* a, const float* mu, int nK, double* part, double* G,
                           cudaStream_t s) {
    const int S = nc_gram_splits(g, nK);
    long long chunk = (g.N + S - 1) / S;
    chunk = (chunk + 63) / 64 * 64;
    dim3 grid((unsigned)((nK + 15) / 16), (unsigned)((nK + 15) / 16), (unsigned)S);
    nc_gram_kernel<<<grid, 256, 0, s>>>(a, mu, nK, g.N, chunk, part);
    nc_gram_sum_kernel<<<64, 256, 0, s>>>(part, S, nK, G);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_nc_grad(const Geom& g, const float* a, const float* mu, const float* Q, const float* dT, int nK,
                           float* gu, cudaStream_t s) {
    long long bx = (g.N + 255) / 256;
    if (bx > 1024) bx = 1024;
    dim3 grid((unsigned)bx, (unsigned)((nK + 15) / 16));
    const size_t smem = sizeof(float) * 16 * (size_t)nK;
    if (smem > 48 * 1024) return cudaErrorInvalidValue;
    if (g.d == 2)
        nc_grad_kernel<2><<<grid, 256, smem, s>>>(a, mu, Q, dT, nK, g.N, gu);
    else
        nc_grad_kernel<3><<<grid, 256, smem, s>>>(a, mu, Q, dT, nK, g.N, gu);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace stml
