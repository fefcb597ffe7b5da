// Learned temporal predictor: kernels of the convolutional encoder-decoder
// (forward, backward, Adam, weight packing).  The network proposes the field
// of a frame that the next temporal level adds (Sec. 3) from its two
// registered neighbours and three images; the registration keeps a proposal
// only where the objective of eq. (1) is lower there than at the classical
// predictor's.
//
// Convolutions are implicit GEMMs on the tensor cores, tcgen05.mma into
// tensor memory: forward and input gradient (conv3_kernel), weight gradient
// (wgrad_tc_kernel).
//   forward:        Y[p][co]  = sum_{tap, ci} X[p + off(tap)][ci] W[tap][ci][co]
//   input gradient: dX[p][ci] = sum_{tap, co} G[p + off(tap)][co] W[8 - tap][ci][co]
//                   (the same kernel with the flipped, transposed weights)
//   weight grad.:   dW[tap][ci][co] = sum_p X[p + off(tap)][ci] G[p][co]
//                   (split over pixel slices, slices summed in a fixed order)
#include <cuda_bf16.h>
#include <type_traits>
#include <cuda_fp16.h>

#include "net.h"

namespace stml {
// per-device caches of the SM count and of the dynamic shared-memory limit (k_transfer.cu)
int device_sms();
cudaError_t set_max_dynamic_smem(const void* kernel, int bytes);
}  // namespace stml

namespace stml {
namespace net {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// 16-byte global -> shared copy; src_bytes = 0 writes zeros (src unread).
__device__ __forceinline__ void cp16(void* dst, const void* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(src_bytes));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__device__ __forceinline__ float slope(float y) { return y > 0.f ? 1.f : kSlope; }
__device__ __forceinline__ float leaky(float z) { return z > 0.f ? z : kSlope * z; }

// Address of 8 input channels [ci, ci + 8) at pixel (n, yy, xx) of the
// stacked sources, or nullptr outside the image.
__device__ __forceinline__ const bf16* in_at(const ConvIn& in, int n, int yy, int xx, int H, int W,
                                             int ci) {
    if (yy < 0 || yy >= H || xx < 0 || xx >= W) return nullptr;
    if (ci < in.ca) {
        if (in.up)
            return in.a + (((long long)n * (H >> 1) + (yy >> 1)) * (W >> 1) + (xx >> 1)) * in.ca + ci;
        return in.a + (((long long)n * H + yy) * W + xx) * in.ca + ci;
    }
    return in.b + (((long long)n * H + yy) * W + xx) * in.cb + (ci - in.ca);
}

// Unpacks 8 BF16 values.
__device__ __forceinline__ void unpack8(const uint4& u, float (&f)[8]) {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float2 t = __bfloat1622float2(h[i]);
        f[2 * i] = t.x;
        f[2 * i + 1] = t.y;
    }
}
__device__ __forceinline__ uint4 pack8(const float (&f)[8]) {
    uint4 u;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
    return u;
}

}  // namespace

// ------------------------------------------------------------ convolution
// Blackwell tensor-core implicit GEMM on a halo tile.  A CTA computes a tile of
// 16 x 8 output pixels (M = 128) x BN output channels, accumulated in tensor
// memory (TMEM) by tcgen05.mma (kind::f16: BF16 operands, FP32 accumulator,
// M = 128, N = BN, K = 16 per instruction, issued by one thread).  Input
// channels run in chunks of 32: the chunk's 18 x 10 halo is gathered once
// (cp.async, zero-filled outside the image; the input may be a nearest-
// upsampled coarse map stacked with a skip map) into the no-swizzle K-major
// core-matrix layout [4 groups of 8 channels][180 halo pixels][8 channels],
// and the nine taps are nine shared-memory descriptors into the same halo:
// tap (dy, dx) starts ((1 + dy) 10 + 1 + dx) pixels in, 8-row groups (tile
// rows) 10 pixels apart, channel groups 180 pixels apart.  The chunk's
// weights arrive as [9 taps][4 groups][BN channels][8] (loaded once per CTA
// when the input has a single chunk).  A CTA runs a sequence of tiles; two
// stages: an item's 18 MMAs commit to its stage's mbarrier, which must
// complete before the stage is refilled.  Tiles alternate between two TMEM
// accumulators, and a tile's epilogue (tcgen05.ld; warp w owns lanes = tile
// rows 4w..4w+3) runs while the next tile's first MMAs execute.  Every wait
// is bounded; on expiry the kernel skips the remaining work, gives the MMAs
// still in flight one more bounded wait, sets *err (1, or 2 if that wait
// expired too: results undefined, discard the context) and frees its TMEM.
namespace {

constexpr int kHaloW = 10, kHaloH = 18, kHaloPx = kHaloW * kHaloH;   // 8 x 16 tile + 1-pixel border
constexpr int kTcStages = 2;
constexpr int kTcA = 4 * kHaloPx * 16;    // bytes of one halo stage: 4 channel groups x 180 px x 16 B

// Shared-memory matrix descriptor, no swizzle, K-major core matrices of
// 8 rows x 16 bytes: lbo = byte distance between core matrices along K,
// sbo = along M/N.
__device__ __forceinline__ uint64_t plain_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);   // start address
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;         // leading dimension byte offset
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;         // stride dimension byte offset
    d |= (uint64_t)1 << 46;                              // descriptor version
    return d;                                            // layout type 0: no swizzle
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count));
}

// Waits for the completion of phase `parity` of the mbarrier; false after
// 2^22 polls (well beyond any MMA chunk's latency).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (int i = 0; i < (1 << 22); ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                 : "memory");
}

// 32 consecutive columns of the thread's TMEM lane: the load and its wait in
// one asm statement, so no instruction can read the registers early.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace

// One CTA waits, with the convolution kernels' bound, on an mbarrier that
// nothing completes: the wait must give up and report it (*expired = 1).
__global__ void wait_probe_kernel(int* __restrict__ expired) {
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        *expired = mbar_wait(smem_u32(&bar), 0u) ? 0 : 1;
    }
}

cudaError_t launch_wait_probe(int* expired, cudaStream_t s) {
    wait_probe_kernel<<<1, 32, 0, s>>>(expired);
    return cudaGetLastError();
}

template <int BN>
struct TcCfg {
    static constexpr int B_BYTES = 9 * 4 * BN * 16;              // one weight stage
    static constexpr int TMEM_COLS = BN <= 32 ? 64 : BN <= 64 ? 128 : 256;   // two accumulators
    static constexpr int SMEM = 128 + kTcStages * (kTcA + B_BYTES) + 64;
    // instruction descriptor: F32 accumulator, BF16 A and B, both K-major, N, M = 128
    static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                      ((uint32_t)(128 >> 4) << 24);
};

template <int BN>
__global__ void __launch_bounds__(128) conv3_kernel(ConvIn in, const bf16* __restrict__ Wh, int Cin, int N, int B,
                                                    int H, int W, ConvOut out, int* __restrict__ err) {
    using C = TcCfg<BN>;
    extern __shared__ unsigned char tc_smem_raw[];
    const uint32_t raw = smem_u32(tc_smem_raw);
    const uint32_t base = (raw + 127u) & ~127u;
    unsigned char* gbase = tc_smem_raw + (base - raw);
    const uint32_t sA = base, sB = base + kTcStages * kTcA;
    const uint32_t bars = sB + kTcStages * C::B_BYTES;           // kTcStages mbarriers
    uint32_t* tslot = reinterpret_cast<uint32_t*>(gbase + (bars - base) + 8 * kTcStages);
    unsigned char* gA = gbase;
    unsigned char* gB = gbase + kTcStages * kTcA;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int tiles_x = (W + 7) >> 3, tiles_y = (H + 15) >> 4;
    const int tiles = B * tiles_y * tiles_x;
    const int n0 = blockIdx.y * BN;
    const int nch = Cin / 32;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                     "r"((uint32_t)C::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < kTcStages; ++i) mbar_init(bars + 8 * i, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    // tile index -> (image, first row, first column)
    auto tile_origin = [&](int t, int& pn, int& y0, int& x0) {
        const int tx = t % tiles_x;
        t /= tiles_x;
        x0 = tx * 8;
        y0 = (t % tiles_y) * 16;
        pn = t / tiles_y;
    };
    // with a single channel chunk the weights are the same for every item:
    // they are loaded once (with the first item) into stage 0's weight buffer
    const bool resident = nch == 1;
    auto load_stage = [&](int st, int tile, int c) {
        int pn, y0, x0;
        tile_origin(tile, pn, y0, x0);
        unsigned char* a_st = gA + st * kTcA;
        for (int s = tid; s < kHaloPx * 4; s += 128) {   // (halo pixel, channel group)
            const int hp = s >> 2, kg = s & 3;
            const int hy = hp / kHaloW, hx = hp - hy * kHaloW;
            const bf16* src = in_at(in, pn, y0 - 1 + hy, x0 - 1 + hx, H, W, c * 32 + kg * 8);
            cp16(a_st + (kg * kHaloPx + hp) * 16, src ? src : in.a, src ? 16 : 0);
        }
        if (resident && tile != (int)blockIdx.x) return;
        unsigned char* b_st = gB + st * C::B_BYTES;
        const bf16* wsrc = Wh + (long long)c * 36 * N * 8;     // [9 taps][4 groups][N][8] of this chunk
        for (int s = tid; s < 36 * BN; s += 128) {
            const int tg = s / BN, r = s - tg * BN;             // (tap, group), output channel
            cp16(b_st + s * 16, wsrc + ((long long)tg * N + n0 + r) * 8, 16);
        }
    };

    // Epilogue of the tile whose accumulator is TMEM buffer `buf`: TMEM lane
    // l = tile pixel (row l / 8, column l % 8); warp w reads lanes 32w..32w+31.
    auto epilogue = [&](int tile, int buf) {
        int pn, y0, x0;
        tile_origin(tile, pn, y0, x0);
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(buf * BN);
        const int y = y0 + (tid >> 3), x = x0 + (tid & 7);
        const bool valid = y < H && x < W;
        const long long m = ((long long)pn * H + y) * W + x;
        // 32 columns per TMEM load and wait
#pragma unroll 1
        for (int c32 = 0; c32 < BN; c32 += 32) {
        float vv[32];
        tc_ld32(trow + (uint32_t)c32, vv);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = vv[8 * i + j];
            const int c0 = c32 + 8 * i;
            if (!valid) continue;
            const int n = n0 + c0;
            if (out.mode == CONV_FWD) {
#pragma unroll
                for (int i = 0; i < 8; ++i) v[i] = leaky(v[i] + out.bias[n + i]);
                *reinterpret_cast<uint4*>(out.y + m * N + n) = pack8(v);
            } else if (out.mode == CONV_MASK) {
                float k[8];
                unpack8(*reinterpret_cast<const uint4*>(out.mask + m * N + n), k);
#pragma unroll
                for (int i = 0; i < 8; ++i) v[i] *= slope(k[i]);
                *reinterpret_cast<uint4*>(out.y + m * N + n) = pack8(v);
            } else {
                float* dst = n < out.n1 ? out.f1 + m * out.n1 + n : out.f2 + m * (N - out.n1) + (n - out.n1);
                reinterpret_cast<float4*>(dst)[0] = make_float4(v[0], v[1], v[2], v[3]);
                reinterpret_cast<float4*>(dst)[1] = make_float4(v[4], v[5], v[6], v[7]);
            }
        }
        }
        tc_fence_before();   // ordered before the barrier that precedes the buffer's next MMA
    };

    // The CTA's (tile, chunk) items run in one sequence q = 0, 1, ...: item q
    // uses stage q & 1 and commits to that stage's mbarrier (use q >> 1); the
    // k-th tile of the CTA accumulates in TMEM buffer k & 1, and its epilogue
    // runs while the MMAs of the (k+1)-th tile's first chunk execute.
    bool ok = true;
    int q = 0, k = 0, prev_tile = -1;
    if ((int)blockIdx.x < tiles) load_stage(0, blockIdx.x, 0);
    cp_commit();
    for (int tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x, ++k) {
        const int buf = k & 1;
        for (int c = 0; c < nch; ++c, ++q) {
            const int st = q & 1;
            cp_wait<0>();
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            // thread 0 waits for the MMAs of item q-1: their stage is refilled below,
            // and when c == 0 they finish the previous tile, whose epilogue follows
            if (tid == 0 && q >= 1 && ok) ok = mbar_wait(bars + 8 * ((q - 1) & 1), (uint32_t)(((q - 1) >> 1) & 1));
            if (!__syncthreads_and(ok)) {     // uniform: every thread leaves together
                ok = false;
                break;
            }
            tc_fence_after();
            if (tid == 0) {
                const uint32_t a0 = sA + st * kTcA, b0 = sB + (resident ? 0 : st * C::B_BYTES);
                const uint32_t dacc = tmem + (uint32_t)(buf * BN);
#pragma unroll 1
                for (int tap = 0; tap < 9; ++tap) {
                    const int dy = tap / 3, dx = tap - 3 * (tap / 3);
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
                        const uint64_t ad = plain_desc(a0 + ((2 * ks) * kHaloPx + dy * kHaloW + dx) * 16,
                                                       kHaloPx * 16, kHaloW * 16);
                        const uint64_t bd = plain_desc(b0 + ((tap * 4 + 2 * ks) * BN) * 16, BN * 16, 128);
                        tc_mma(dacc, ad, bd, C::IDESC, (c > 0 || tap > 0 || ks > 0) ? 1u : 0u);
                    }
                }
                tc_commit(bars + 8 * st);
            }
            // prefetch the next item (this tile's next chunk, or the next tile's
            // first) before the previous tile's epilogue, so that the copies
            // proceed while the epilogue reads TMEM
            if (c + 1 < nch)
                load_stage(st ^ 1, tile, c + 1);
            else if (tile + (int)gridDim.x < tiles)
                load_stage(st ^ 1, tile + gridDim.x, 0);
            cp_commit();
            if (c == 0 && prev_tile >= 0) epilogue(prev_tile, buf ^ 1);
        }
        prev_tile = tile;
    }
    // the last tile: wait for its MMAs, then drain it
    if (ok && prev_tile >= 0) {
        if (tid == 0) ok = mbar_wait(bars + 8 * ((q - 1) & 1), (uint32_t)(((q - 1) >> 1) & 1));
        ok = __syncthreads_and(ok) != 0;
        tc_fence_after();
        if (ok) epilogue(prev_tile, (k - 1) & 1);
    }
    cp_wait<0>();
    if (!ok && tid == 0) {
        // The wait that expired was for the MMAs of item q - 1, which may still
        // be running (writing TMEM, reading this CTA's shared memory).  They get
        // one more bounded wait before the TMEM is released; if that expires
        // too, *err = 2: results are undefined and the context should be
        // discarded.  Otherwise *err = 1 (the launch stopped early).
        const bool drained = q < 1 || mbar_wait(bars + 8 * ((q - 1) & 1), (uint32_t)(((q - 1) >> 1) & 1));
        atomicMax(err, drained ? 1 : 2);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                     "r"((uint32_t)C::TMEM_COLS)
                     : "memory");
    }
}

template <int BN>
static cudaError_t conv3_go(const ConvIn& in, const bf16* Wh, int Cin, int N, int B, int H, int W,
                            const ConvOut& out, int* err, cudaStream_t s) {
    using C = TcCfg<BN>;
    const cudaError_t e = set_max_dynamic_smem(reinterpret_cast<const void*>(conv3_kernel<BN>), C::SMEM);
    if (e != cudaSuccess) return e;
    const long long tiles = (long long)B * ((H + 15) / 16) * ((W + 7) / 8);
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    // a few CTAs per SM, each running a sequence of tiles (twice the CTAs
    // that fit at once: measured faster than one wave of resident CTAs)
    const long long per_sm = BN <= 32 ? 3 : BN <= 64 ? 2 : 1;
    const int sms = device_sms();
    long long ctas = (long long)(sms > 0 ? sms : 152) * per_sm * 2 / (N / BN);
    if (ctas < 1) ctas = 1;
    if (ctas > tiles) ctas = tiles;
    dim3 grid((unsigned)ctas, N / BN);
    conv3_kernel<BN><<<grid, 128, C::SMEM, s>>>(in, Wh, Cin, N, B, H, W, out, err);
    return cudaGetLastError();
}

cudaError_t launch_conv3(const ConvIn& in, const bf16* Wh, int Cin, int N, int B, int H, int W,
                         const ConvOut& out, int* err, cudaStream_t s) {
    if (Cin % 32 || N % 32 || in.ca % 32 || in.cb % 32 || in.ca + in.cb != Cin || B <= 0 || H <= 0 ||
        W <= 0 || (in.up && ((H | W) & 1)) || !err)
        return cudaErrorInvalidValue;
    if (N % 128 == 0) return conv3_go<128>(in, Wh, Cin, N, B, H, W, out, err, s);
    if (N % 96 == 0) return conv3_go<96>(in, Wh, Cin, N, B, H, W, out, err, s);
    if (N % 64 == 0) return conv3_go<64>(in, Wh, Cin, N, B, H, W, out, err, s);
    return conv3_go<32>(in, Wh, Cin, N, B, H, W, out, err, s);
}

// --------------------------------------------------------- weight gradient
// dW[tap][ci][co] = sum_p G[p][co] X[p + off(tap)][ci] as tensor-core GEMMs
// (tcgen05.mma kind::f16, BF16 operands, FP32 accumulators in TMEM), one per
// tap: M = 128 output channels (TMEM lanes; rows past the layer's channels
// are zero), N = 32 input channels, K = pixels.  A CTA owns one block of 128
// output channels, one chunk of 32 input channels and a run of 8 x 8 pixel
// tiles; the nine taps accumulate in TMEM columns 32 tap .. 32 tap + 31.  Per
// tile the output gradients G (64 pixels x 128 channels) and the input's
// 10 x 10 halo (32 channels) are gathered once by cp.async (zero outside the
// image) into no-swizzle MN-major core-matrix layouts: G as [8 tile rows]
// [16 channel groups][8 pixels][8 ch], the halo as [4 channel groups]
// [10 x 10 pixels][8 ch].  The B operand of tap (dy, dx) is the halo seen
// through a descriptor that starts at halo pixel (1 + dy, 1 + dx): its 8-pixel
// core-matrix rows are 8 consecutive halo pixels, the next tile row is 10
// pixels on, the next channel group 100 pixels on.  36 MMAs (9 taps x 4 steps
// of 16 pixels) per tile, issued by one thread and committed to the stage's
// mbarrier; three stages; every wait bounded (*err as in conv3_kernel).
namespace {
constexpr int kWgHalo = 10;                                   // 8 x 8 tile + 1-pixel border
constexpr int kWgHaloPx = kWgHalo * kWgHalo;
}  // namespace

struct WgCfg {
    static constexpr int STAGES = 3;
    static constexpr uint32_t A_SBO = 128;                    // between 8-channel groups (M)
    static constexpr uint32_t A_LBO = 16 * 128;               // between tile rows (K)
    static constexpr int A_BYTES = 8 * (int)A_LBO;            // 64 pixels x 128 channels
    static constexpr uint32_t B_LBO = kWgHalo * 16;           // next tile row in the halo (K)
    static constexpr uint32_t B_SBO = kWgHaloPx * 16;         // next channel group (N)
    static constexpr int B_BYTES = 4 * kWgHaloPx * 16;        // 10 x 10 pixels x 32 channels
    static constexpr int STAGE = A_BYTES + B_BYTES;
    // at least half the SM's shared memory: one CTA per SM, which owns all
    // 512 TMEM columns (nine accumulators of 32)
    static constexpr int SMEM_USED = 128 + STAGES * STAGE + 64;
    static constexpr int SMEM = SMEM_USED > 120 * 1024 ? SMEM_USED : 120 * 1024;
    static constexpr int TMEM_COLS = 512;
    // F32 accumulator, BF16 A and B, both MN-major (transposed), N = 32, M = 128
    static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                                      ((uint32_t)(32 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
};

__global__ void __launch_bounds__(128) wgrad_tc_kernel(ConvIn in, const bf16* __restrict__ G, int Cin, int N,
                                                       int B, int H, int W, int tiles_per_slice,
                                                       float* __restrict__ part, int* __restrict__ err) {
    using C = WgCfg;
    extern __shared__ unsigned char wg_smem_raw[];
    const uint32_t raw = smem_u32(wg_smem_raw);
    const uint32_t base = (raw + 127u) & ~127u;
    unsigned char* gbase = wg_smem_raw + (base - raw);
    const uint32_t bars = base + C::STAGES * C::STAGE;          // STAGES mbarriers
    uint32_t* tslot = reinterpret_cast<uint32_t*>(gbase + (bars - base) + 8 * C::STAGES);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int cch = blockIdx.x;                                  // input-channel chunk
    const int co0 = blockIdx.y * 128;                            // output-channel block
    const int ncol = N - co0 < 128 ? N - co0 : 128;              // real output channels (multiple of 8)
    const int tx = (W + 7) >> 3, ty = (H + 7) >> 3;
    const int ntiles = B * ty * tx;
    const int t_begin = blockIdx.z * tiles_per_slice;
    const int t_end = t_begin + tiles_per_slice < ntiles ? t_begin + tiles_per_slice : ntiles;
    const int nst = t_end > t_begin ? t_end - t_begin : 0;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                     "r"((uint32_t)C::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < C::STAGES; ++i) mbar_init(bars + 8 * i, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    // channel groups past the layer's channels stay zero in every stage
    for (int i = tid; i < C::STAGES * 64 * 16; i += 128) {   // (stage, tile row, pixel, channel group)
        const int g = i & 15, rest = i >> 4;
        if (g * 8 < ncol) continue;
        const int st = rest / 64, r = (rest % 64) >> 3, k = rest & 7;
        *reinterpret_cast<uint4*>(gbase + st * C::STAGE + r * C::A_LBO + g * C::A_SBO + k * 16) =
            make_uint4(0, 0, 0, 0);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    auto load_stage = [&](int st, int it) {
        int t = t_begin + it;
        const int txi = t % tx;
        t /= tx;
        const int tyi = t % ty;
        const int pn = t / ty;
        const int y0 = tyi * 8, x0 = txi * 8;
        unsigned char* a_st = gbase + st * C::STAGE;
        unsigned char* b_st = a_st + C::A_BYTES;
        const int ng = ncol >> 3;
        for (int i = tid; i < 64 * ng; i += 128) {              // G: (pixel, channel group)
            const int k = i / ng, g = i - k * ng;
            const int y = y0 + (k >> 3), x = x0 + (k & 7);
            const bool ok = y < H && x < W;
            const bf16* src = ok ? G + (((long long)pn * H + y) * W + x) * N + co0 + g * 8 : G;
            cp16(a_st + (k >> 3) * C::A_LBO + g * C::A_SBO + (k & 7) * 16, src, ok ? 16 : 0);
        }
        for (int i = tid; i < kWgHaloPx * 4; i += 128) {        // halo: (pixel, channel group)
            const int hp = i >> 2, g = i & 3;
            const int hy = hp / kWgHalo, hx = hp - hy * kWgHalo;
            const bf16* src = in_at(in, pn, y0 - 1 + hy, x0 - 1 + hx, H, W, cch * 32 + g * 8);
            cp16(b_st + g * C::B_SBO + hp * 16, src ? src : in.a, src ? 16 : 0);
        }
    };

    bool ok = true;
    int waited = -1;
#pragma unroll 1
    for (int sg = 0; sg < C::STAGES - 1; ++sg) {
        if (sg < nst) load_stage(sg, sg);
        cp_commit();
    }
#pragma unroll 1
    for (int it = 0; it < nst; ++it) {
        const int st = it % C::STAGES;
        cp_wait<C::STAGES - 2>();
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();   // every thread's copies of tile it have landed
        tc_fence_after();
        if (tid == 0) {
            const uint32_t a0 = base + st * C::STAGE, b0 = a0 + C::A_BYTES;
#pragma unroll 1
            for (int tap = 0; tap < 9; ++tap) {
                const int dy = tap / 3, dx = tap - 3 * (tap / 3);   // halo offsets 0..2
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {                    // tile rows 2 ks, 2 ks + 1
                    const uint64_t ad = plain_desc(a0 + 2 * ks * C::A_LBO, C::A_LBO, C::A_SBO);
                    const uint64_t bd =
                        plain_desc(b0 + ((2 * ks + dy) * kWgHalo + dx) * 16, C::B_LBO, C::B_SBO);
                    tc_mma(tmem + (uint32_t)(tap * 32), ad, bd, C::IDESC, (it > 0 || ks > 0) ? 1u : 0u);
                }
            }
            tc_commit(bars + 8 * st);
        }
        const int nx = it + C::STAGES - 1;
        if (nx < nst) {
            if (it >= 1) {   // the stage of tile it - 1 is refilled once its MMAs are done
                if (tid == 0)
                    ok = mbar_wait(bars + 8 * ((it - 1) % C::STAGES), (uint32_t)(((it - 1) / C::STAGES) & 1));
                if (!__syncthreads_and(ok)) {
                    ok = false;
                    break;
                }
                waited = it - 1;
            }
            load_stage(nx % C::STAGES, nx);
        }
        cp_commit();
    }
    if (ok && nst > 0) {
        const int j = nst - 1;
        if (tid == 0) ok = mbar_wait(bars + 8 * (j % C::STAGES), (uint32_t)((j / C::STAGES) & 1));
        ok = __syncthreads_and(ok) != 0;
        if (ok) waited = j;
    }
    tc_fence_after();
    if (ok) {
        // TMEM lane 32 w + l = output channel co0 + 32 w + l; column 32 tap + i = input channel cch * 32 + i
        const int co = co0 + warp * 32 + lane;
        const long long K = 9LL * Cin;
        float* dst = part + (long long)blockIdx.z * K * N;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int tap = 0; tap < 9; ++tap) {
            float v[32];
            if (nst > 0) {
                tc_ld32(trow + (uint32_t)(tap * 32), v);
            } else {
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = 0.f;
            }
            if (co < N) {
#pragma unroll
                for (int i = 0; i < 32; ++i) dst[((long long)tap * Cin + cch * 32 + i) * N + co] = v[i];
            }
        }
    }
    cp_wait<0>();
    if (!ok && tid == 0) {
        const int j = nst - 1;
        bool drained = true;
        if (j > waited && j >= 0) drained = mbar_wait(bars + 8 * (j % C::STAGES), (uint32_t)((j / C::STAGES) & 1));
        atomicMax(err, drained ? 1 : 2);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                     "r"((uint32_t)C::TMEM_COLS)
                     : "memory");
    }
}

cudaError_t launch_wgrad3(const ConvIn& in, const bf16* G, int Cin, int N, int B, int H, int W,
                          float* part, size_t part_cap, int* splits, int* err, cudaStream_t s) {
    if (Cin % 32 || N % 32 || in.ca % 32 || in.cb % 32 || in.ca + in.cb != Cin || B <= 0 || H <= 0 || W <= 0 ||
        (in.up && ((H | W) & 1)) || !err)
        return cudaErrorInvalidValue;
    const long long ntiles = (long long)B * ((H + 7) / 8) * ((W + 7) / 8);
    if (ntiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    const int cblocks = (N + 127) / 128;
    const long long ctas = (long long)(Cin / 32) * cblocks;
    const long long per = 9LL * Cin * N;
    const int sms = device_sms();
    long long S = ((sms > 0 ? sms : 152) + ctas - 1) / ctas;   // about one CTA per SM
    if (S > ntiles) S = ntiles;
    if (S > (long long)(part_cap / per)) S = (long long)(part_cap / per);
    if (S < 1) return cudaErrorInvalidValue;
    const long long tps = (ntiles + S - 1) / S;
    S = (ntiles + tps - 1) / tps;
    *splits = (int)S;
    using C = WgCfg;
    const cudaError_t e = set_max_dynamic_smem(reinterpret_cast<const void*>(wgrad_tc_kernel), C::SMEM);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)(Cin / 32), (unsigned)cblocks, (unsigned)S);
    wgrad_tc_kernel<<<grid, 128, C::SMEM, s>>>(in, G, Cin, N, B, H, W, (int)tps, part, err);
    return cudaGetLastError();
}

// ------------------------------------------------------------ column sums
__global__ void __launch_bounds__(256) colsum_kernel(const bf16* __restrict__ G, long long P, int N,
                                                     long long chunk, float* __restrict__ part) {
    __shared__ float red[256];
    const int R = 256 / N;
    const int c = threadIdx.x % N, r = threadIdx.x / N;
    const long long pb = (long long)blockIdx.x * chunk;
    const long long pe = pb + chunk < P ? pb + chunk : P;
    float acc = 0.f;
    if (r < R) {
#pragma unroll 8
        for (long long p = pb + r; p < pe; p += R) acc += __bfloat162float(G[p * N + c]);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < N) {
        float v = 0.f;
        for (int k = 0; k < R; ++k) v += red[k * N + threadIdx.x];
        part[(long long)blockIdx.x * N + threadIdx.x] = v;
    }
}

cudaError_t launch_colsum(const bf16* G, long long P, int N, float* part, size_t part_cap, int* splits,
                          cudaStream_t s) {
    if (N <= 0 || N > 256 || P <= 0) return cudaErrorInvalidValue;
    long long S = 256;
    if (S > (long long)(part_cap / N)) S = (long long)(part_cap / N);
    if (S > P) S = P;
    if (S < 1) return cudaErrorInvalidValue;
    const long long chunk = (P + S - 1) / S;
    S = (P + chunk - 1) / chunk;
    *splits = (int)S;
    colsum_kernel<<<(unsigned)S, 256, 0, s>>>(G, P, N, chunk, part);
    return cudaGetLastError();
}

// Fixed-order sum of the slice partials.  A block owns 32 consecutive output
// elements; warp w adds slices w, w + 8, w + 16, ... in order (each load a
// coalesced 128-byte row), and warp 0 adds the eight warp sums in order: the
// result depends only on the slice count, never on timing.
__global__ void __launch_bounds__(256) reduce_grad_kernel(const float* __restrict__ wpart, int ws, int cin,
                                                          int cin_real, int N, const float* __restrict__ bpart,
                                                          int bs, float* __restrict__ grad, long long w_off,
                                                          long long b_off) {
    __shared__ float red[8][33];
    const long long nW = 9LL * cin_real * N;
    const long long per = 9LL * cin * N;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (long long blk = blockIdx.x; blk * 32 < nW + N; blk += gridDim.x) {
        const long long i = blk * 32 + lane;
        float v = 0.f;
        if (i < nW) {
            const int co = (int)(i % N);
            const long long k = i / N;
            const int ci = (int)(k % cin_real);
            const int tap = (int)(k / cin_real);
            const float* src = wpart + ((long long)tap * cin + ci) * N + co;
#pragma unroll 4
            for (int sl = w; sl < ws; sl += 8) v += __ldg(src + (long long)sl * per);
        } else if (i < nW + N) {
            const float* src = bpart + (i - nW);
            for (int sl = w; sl < bs; sl += 8) v += __ldg(src + (long long)sl * N);
        }
        red[w][lane] = v;
        __syncthreads();
        if (w == 0 && i < nW + N) {
            float t = red[0][lane];
#pragma unroll
            for (int k = 1; k < 8; ++k) t += red[k][lane];
            grad[i < nW ? w_off + i : b_off + (i - nW)] = t;
        }
        __syncthreads();
    }
}

cudaError_t launch_reduce_grad(const float* wpart, int ws, int cin, int cin_real, int N,
                               const float* bpart, int bs, float* grad, long long w_off,
                               long long b_off, cudaStream_t s) {
    const long long nblk = (9LL * cin_real * N + N + 31) / 32;
    const unsigned blocks = (unsigned)(nblk < 8192 ? nblk : 8192);
    reduce_grad_kernel<<<blocks, 256, 0, s>>>(wpart, ws, cin, cin_real, N, bpart, bs, grad, w_off, b_off);
    return cudaGetLastError();
}

// ------------------------------------------------------ pooling and friends
__global__ void pool2_kernel(const bf16* __restrict__ x, bf16* __restrict__ y, int B, int H, int W,
                             int C) {
    const int Ho = H >> 1, Wo = W >> 1, C8 = C >> 3;
    const long long n = (long long)B * Ho * Wo * C8;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int c8 = (int)(i % C8);
        long long q = i / C8;
        const int xo = (int)(q % Wo);
        q /= Wo;
        const int yo = (int)(q % Ho);
        const int b = (int)(q / Ho);
        float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                const long long p = ((long long)b * H + 2 * yo + dy) * W + 2 * xo + dx;
                float f[8];
                unpack8(*reinterpret_cast<const uint4*>(x + p * C + c8 * 8), f);
#pragma unroll
                for (int k = 0; k < 8; ++k) s[k] += f[k];
            }
#pragma unroll
        for (int k = 0; k < 8; ++k) s[k] *= 0.25f;
        *reinterpret_cast<uint4*>(y + i * 8) = pack8(s);
    }
}

cudaError_t launch_pool2(const bf16* x, bf16* y, int B, int H, int W, int C, cudaStream_t s) {
    if (C % 8 || (H | W) & 1) return cudaErrorInvalidValue;
    const long long n = (long long)B * (H / 2) * (W / 2) * (C / 8);
    long long blocks = (n + 255) / 256;
    if (blocks > 65536) blocks = 65536;
    pool2_kernel<<<(unsigned)blocks, 256, 0, s>>>(x, y, B, H, W, C);
    return cudaGetLastError();
}

__global__ void combine_kernel(const float* __restrict__ dp, const float* __restrict__ skip,
                               const bf16* __restrict__ e, bf16* __restrict__ g, int B, int H, int W,
                               int C) {
    const int C8 = C >> 3;
    const long long n = (long long)B * H * W * C8;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int c8 = (int)(i % C8);
        const long long p = i / C8;
        const int x = (int)(p % W);
        const long long q = p / W;
        const int y = (int)(q % H);
        const int b = (int)(q / H);
        const long long pc = ((long long)b * (H >> 1) + (y >> 1)) * (W >> 1) + (x >> 1);
        const float4* d4 = reinterpret_cast<const float4*>(dp + pc * C + c8 * 8);
        const float4* s4 = reinterpret_cast<const float4*>(skip + p * C + c8 * 8);
        const float4 d0 = d4[0], d1 = d4[1], s0 = s4[0], s1 = s4[1];
        float ef[8];
        unpack8(*reinterpret_cast<const uint4*>(e + p * C + c8 * 8), ef);
        float v[8] = {0.25f * d0.x + s0.x, 0.25f * d0.y + s0.y, 0.25f * d0.z + s0.z,
                      0.25f * d0.w + s0.w, 0.25f * d1.x + s1.x, 0.25f * d1.y + s1.y,
                      0.25f * d1.z + s1.z, 0.25f * d1.w + s1.w};
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] *= slope(ef[k]);
        *reinterpret_cast<uint4*>(g + p * C + c8 * 8) = pack8(v);
    }
}

cudaError_t launch_combine(const float* dp, const float* skip, const bf16* e, bf16* g, int B, int H,
                           int W, int C, cudaStream_t s) {
    if (C % 8 || (H | W) & 1) return cudaErrorInvalidValue;
    const long long n = (long long)B * H * W * (C / 8);
    long long blocks = (n + 255) / 256;
    if (blocks > 65536) blocks = 65536;
    combine_kernel<<<(unsigned)blocks, 256, 0, s>>>(dp, skip, e, g, B, H, W, C);
    return cudaGetLastError();
}

__global__ void upback_kernel(const float* __restrict__ f, const bf16* __restrict__ d,
                              bf16* __restrict__ g, int B, int H, int W, int C) {
    const int Ho = H >> 1, Wo = W >> 1, C8 = C >> 3;
    const long long n = (long long)B * Ho * Wo * C8;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int c8 = (int)(i % C8);
        const long long pc = i / C8;
        const int xo = (int)(pc % Wo);
        const long long q = pc / Wo;
        const int yo = (int)(q % Ho);
        const int b = (int)(q / Ho);
        float v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                const long long p = ((long long)b * H + 2 * yo + dy) * W + 2 * xo + dx;
                const float4* f4 = reinterpret_cast<const float4*>(f + p * C + c8 * 8);
                const float4 a = f4[0], c = f4[1];
                v[0] += a.x; v[1] += a.y; v[2] += a.z; v[3] += a.w;
                v[4] += c.x; v[5] += c.y; v[6] += c.z; v[7] += c.w;
            }
        float df[8];
        unpack8(*reinterpret_cast<const uint4*>(d + pc * C + c8 * 8), df);
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] *= slope(df[k]);
        *reinterpret_cast<uint4*>(g + pc * C + c8 * 8) = pack8(v);
    }
}

cudaError_t launch_upback(const float* f, const bf16* d, bf16* g, int B, int H, int W, int C,
                          cudaStream_t s) {
    if (C % 8 || (H | W) & 1) return cudaErrorInvalidValue;
    const long long n = (long long)B * (H / 2) * (W / 2) * (C / 8);
    long long blocks = (n + 255) / 256;
    if (blocks > 65536) blocks = 65536;
    upback_kernel<<<(unsigned)blocks, 256, 0, s>>>(f, d, g, B, H, W, C);
    return cudaGetLastError();
}

// ------------------------------------------------------------- input / head
__device__ __forceinline__ float load_img(const void* p, int type, long long i) {
    if (type == 1) return __half2float(static_cast<const __half*>(p)[i]);
    if (type == 2) return __bfloat162float(static_cast<const bf16*>(p)[i]);
    return static_cast<const float*>(p)[i];
}

__global__ void assemble_kernel(const Sample* __restrict__ smp, int B, int H, int W, int H8, int W8,
                                bf16* __restrict__ x0, float* __restrict__ base,
                                float* __restrict__ tgt) {
    const long long n = (long long)B * H8 * W8;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(p % W8);
        const long long q = p / W8;
        const int y = (int)(q % H8);
        const int b = (int)(q / H8);
        float f[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        float b0 = 0.f, b1 = 0.f, t0 = 0.f, t1 = 0.f;
        if (y < H && x < W) {
            const Sample S = smp[b];
            const float ih = 1.f / S.h;
            const long long o = (long long)y * S.ld + x;
            const long long oi = (long long)y * S.ld_img + x;
            const float l0 = S.y_l[o], l1 = S.y_l[S.plane + o];
            const float r0 = S.y_r[o], r1 = S.y_r[S.plane + o];
            f[0] = l0 * ih;
            f[1] = l1 * ih;
            f[2] = r0 * ih;
            f[3] = r1 * ih;
            f[4] = load_img(S.T_l, S.img_type, oi);
            f[5] = load_img(S.T_k, S.img_type, oi);
            f[6] = load_img(S.T_r, S.img_type, oi);
            const float wr = 1.f - S.w_l;
            b0 = (S.w_l * l0 + wr * r0) * ih;
            b1 = (S.w_l * l1 + wr * r1) * ih;
            if (S.target) {
                t0 = S.target[o] * ih;
                t1 = S.target[S.plane + o] * ih;
            }
        }
        uint4* dst = reinterpret_cast<uint4*>(x0 + p * kInPad);
        dst[0] = pack8(f);
        const uint4 z = make_uint4(0, 0, 0, 0);
        dst[1] = z;
        dst[2] = z;
        dst[3] = z;
        reinterpret_cast<float2*>(base)[p] = make_float2(b0, b1);
        if (tgt) reinterpret_cast<float2*>(tgt)[p] = make_float2(t0, t1);
    }
}

cudaError_t launch_assemble(const Sample* smp, int B, int H, int W, int H8, int W8, bf16* x0,
                            float* base, float* tgt, cudaStream_t s) {
    const long long n = (long long)B * H8 * W8;
    long long blocks = (n + 255) / 256;
    if (blocks > 65536) blocks = 65536;
    assemble_kernel<<<(unsigned)blocks, 256, 0, s>>>(smp, B, H, W, H8, W8, x0, base, tgt);
    return cudaGetLastError();
}

constexpr int kHeadPart = 1 + kHeadIn * kOutCh + kOutCh;   // sum e^2, dW, db

__global__ void __launch_bounds__(256) head_kernel(const bf16* __restrict__ d0,
                                                   const float* __restrict__ th,
                                                   const float* __restrict__ base,
                                                   const float* __restrict__ tgt,
                                                   const Sample* __restrict__ smp, int B, int H, int W,
                                                   int H8, int W8, int train, float inv_count,
                                                   float* __restrict__ part, bf16* __restrict__ gd0) {
    __shared__ float sw[kHeadIn * kOutCh + kOutCh];
    __shared__ float red[8][kHeadPart];
    for (int i = threadIdx.x; i < kHeadIn * kOutCh + kOutCh; i += blockDim.x) sw[i] = th[i];
    __syncthreads();
    float acc[kHeadPart];
#pragma unroll
    for (int i = 0; i < kHeadPart; ++i) acc[i] = 0.f;
    const long long n = (long long)B * H8 * W8;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(p % W8);
        const long long q = p / W8;
        const int y = (int)(q % H8);
        const int b = (int)(q / H8);
        float d[kHeadIn];
#pragma unroll
        for (int k = 0; k < kHeadIn / 8; ++k) {
            float f[8];
            unpack8(reinterpret_cast<const uint4*>(d0 + p * kHeadIn)[k], f);
#pragma unroll
            for (int j = 0; j < 8; ++j) d[8 * k + j] = f[j];
        }
        float dl0 = sw[kHeadIn * kOutCh], dl1 = sw[kHeadIn * kOutCh + 1];
#pragma unroll
        for (int j = 0; j < kHeadIn; ++j) {
            dl0 += sw[2 * j] * d[j];
            dl1 += sw[2 * j + 1] * d[j];
        }
        const bool inside = y < H && x < W;
        const float2 bs = reinterpret_cast<const float2*>(base)[p];
        if (!train) {
            if (inside) {
                const Sample& S = smp[b];
                const long long o = (long long)y * S.ld + x;
                S.out[o] = S.h * (bs.x + dl0);
                S.out[S.plane + o] = S.h * (bs.y + dl1);
            }
            continue;
        }
        float g0 = 0.f, g1 = 0.f;
        if (inside) {
            const float2 tg = reinterpret_cast<const float2*>(tgt)[p];
            const float e0 = bs.x + dl0 - tg.x, e1 = bs.y + dl1 - tg.y;
            acc[0] += e0 * e0 + e1 * e1;
            g0 = 2.f * e0 * inv_count;
            g1 = 2.f * e1 * inv_count;
        }
        float gv[kHeadIn];
#pragma unroll
        for (int j = 0; j < kHeadIn; ++j) {
            acc[1 + 2 * j] += d[j] * g0;
            acc[2 + 2 * j] += d[j] * g1;
            gv[j] = (sw[2 * j] * g0 + sw[2 * j + 1] * g1) * slope(d[j]);
        }
        acc[1 + kHeadIn * kOutCh] += g0;
        acc[2 + kHeadIn * kOutCh] += g1;
#pragma unroll
        for (int k = 0; k < kHeadIn / 8; ++k) {
            float f[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) f[j] = gv[8 * k + j];
            reinterpret_cast<uint4*>(gd0 + p * kHeadIn)[k] = pack8(f);
        }
    }
    if (!train) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < kHeadPart; ++i) {
        float v = acc[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][i] = v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kHeadPart; i += blockDim.x) {
        float v = 0.f;
        for (int w = 0; w < 8; ++w) v += red[w][i];
        part[(long long)blockIdx.x * kHeadPart + i] = v;
    }
}

cudaError_t launch_head(const bf16* d0, const float* theta_head, const float* base, const float* tgt,
                        const Sample* smp, int B, int H, int W, int H8, int W8, int train,
                        float inv_count, float* part, int* blocks, bf16* gd0, cudaStream_t s) {
    const long long n = (long long)B * H8 * W8;
    long long nb = (n + 255) / 256;
    if (nb > 1024) nb = 1024;
    if (blocks) *blocks = (int)nb;
    head_kernel<<<(unsigned)nb, 256, 0, s>>>(d0, theta_head, base, tgt, smp, B, H, W, H8, W8, train,
                                            inv_count, part, gd0);
    return cudaGetLastError();
}

__global__ void reduce_head_kernel(const float* __restrict__ part, int blocks, float* __restrict__ grad,
                                   long long off, float inv_count, double* loss) {
    for (int i = threadIdx.x; i < kHeadPart; i += blockDim.x) {
        float v = 0.f;
        for (int b = 0; b < blocks; ++b) v += part[(long long)b * kHeadPart + i];
        if (i == 0) {
            if (loss) *loss = (double)v * (double)inv_count;
        } else {
            grad[off + i - 1] = v;
        }
    }
}

cudaError_t launch_reduce_head(const float* part, int blocks, float* grad, long long off, float inv_count,
                               double* loss, cudaStream_t s) {
    reduce_head_kernel<<<1, 128, 0, s>>>(part, blocks, grad, off, inv_count, loss);
    return cudaGetLastError();
}

// ------------------------------------------------------------ Adam, packing
__global__ void adam_kernel(float* __restrict__ th, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, long long n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        th[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

cudaError_t launch_adam(float* theta, float* m, float* v, const float* g, long long n, float lr,
                        float b1, float b2, float eps, float c1, float c2, cudaStream_t s) {
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    adam_kernel<<<(unsigned)blocks, 256, 0, s>>>(theta, m, v, g, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

// Weights in the layout of conv3_kernel: [Cin / 32 chunks][9 taps][4 groups
// of 8 input channels][N][8], forward (N = cout, input channel ci) and, for
// the input gradient, flipped and transposed (N = cin, input channel co of
// W[8 - tap][ci][co]).
__global__ void pack_kernel(const float* __restrict__ th, PackTable t, long long total) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        long long r = i;
        int l = 0;
        bool flip = false;
        for (; l < t.n; ++l) {
            const long long nf = 9LL * t.cin[l] * t.cout[l];
            if (r < nf) break;
            r -= nf;
            if (t.wd[l]) {
                if (r < nf) {
                    flip = true;
                    break;
                }
                r -= nf;
            }
        }
        if (l >= t.n) continue;
        const int cin = t.cin[l], cout = t.cout[l], cr = t.cin_real[l];
        const int Nn = flip ? cin : cout;
        // r = (((chunk * 9 + tap) * 4 + group) * Nn + n) * 8 + e
        const int e = (int)(r & 7);
        long long q = r >> 3;
        const int n = (int)(q % Nn);
        q /= Nn;
        const int grp = (int)(q % 4);
        q /= 4;
        const int tap = (int)(q % 9);
        const int chunk = (int)(q / 9);
        const int k = chunk * 32 + grp * 8 + e;   // input channel of this GEMM
        float v = 0.f;
        if (!flip) {
            if (k < cr) v = th[t.w_off[l] + ((long long)tap * cr + k) * cout + n];
        } else {
            if (n < cr) v = th[t.w_off[l] + ((long long)(8 - tap) * cr + n) * cout + k];
        }
        (flip ? t.wd[l] : t.wf[l])[r] = __float2bfloat16_rn(v);
    }
}

cudaError_t launch_pack(const float* theta, const PackTable& t, cudaStream_t s) {
    long long total = 0;
    for (int l = 0; l < t.n; ++l) total += 9LL * t.cin[l] * t.cout[l] * (t.wd[l] ? 2 : 1);
    long long blocks = (total + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    pack_kernel<<<(unsigned)blocks, 256, 0, s>>>(theta, t, total);
    return cudaGetLastError();
}

__global__ void to_bf16_kernel(const float* __restrict__ src, bf16* __restrict__ dst, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = __float2bfloat16_rn(src[i]);
}
__global__ void from_bf16_kernel(const bf16* __restrict__ src, float* __restrict__ dst, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = __bfloat162float(src[i]);
}

cudaError_t launch_to_bf16(const float* src, bf16* dst, long long n, cudaStream_t s) {
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    to_bf16_kernel<<<(unsigned)blocks, 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}
cudaError_t launch_from_bf16(const bf16* src, float* dst, long long n, cudaStream_t s) {
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    from_bf16_kernel<<<(unsigned)blocks, 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

}  // namespace net
}  // namespace stml
