// Learned temporal predictor: launchers of the network's kernels (internal).
//
// Tensors are channels-last BF16 maps [pixel][channel] over a batch of B
// canvases of H8 x W8 pixels (the images zero-padded to multiples of 8);
// pixel index p = (n H8 + y) W8 + x.  Level l of the network has H8 / 2^l x
// W8 / 2^l pixels per canvas.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace stml {
namespace net {

typedef __nv_bfloat16 bf16;

constexpr float kSlope = 0.1f;     // leaky ReLU
constexpr int kInCh = 7;           // [y_l / h (2), y_r / h (2), T_l, T_k, T_r]
constexpr int kInPad = 32;         // x0 is stored with 32 channels (the rest zero)
constexpr int kHeadIn = 32;
constexpr int kOutCh = 2;

// One sample of a batch: the two registered neighbours' fields (2 component
// planes each, `plane` floats apart, rows `ld` apart), the three images
// (`img_type`: 0 f32, 1 f16, 2 bf16; rows `ld_img` apart), the left weight
// w_l = (r - k) / (r - l) and the level's cell width h.  `target` (may be
// null) and `out` are fields of the same layout as y_l.
struct Sample {
    const float* y_l;
    const float* y_r;
    const void* T_l;
    const void* T_k;
    const void* T_r;
    const float* target;
    float* out;
    long long plane;
    int ld;
    int ld_img;
    int img_type;
    float w_l;
    float h;
};

// Sources of a convolution's input: `a` (ca channels; at half resolution and
// upsampled by nearest neighbour when up = 1) followed by `b` (cb channels,
// cb = 0 for none).  ca and cb are multiples of 32.
struct ConvIn {
    const bf16* a;
    int ca;
    int up;
    const bf16* b;
    int cb;
};

// What the convolution epilogue does with the FP32 accumulator.
//   FWD:   y = bf16(leaky(acc + bias))                      -> y  [P][N]
//   MASK:  y = bf16(acc * slope(mask))                      -> y  [P][N]
//   SPLIT: channels [0, n1) -> f1 [P][n1], [n1, N) -> f2 [P][N - n1]  (FP32)
enum ConvMode { CONV_FWD = 0, CONV_MASK = 1, CONV_SPLIT = 2 };
struct ConvOut {
    int mode;
    const float* bias;
    bf16* y;
    const bf16* mask;
    float* f1;
    float* f2;
    int n1;
};

// Layer table of the packing kernel: parameter offsets and packed weights.
constexpr int kLayers = 14;
struct PackTable {
    int cin_real[kLayers], cin[kLayers], cout[kLayers];
    long long w_off[kLayers];           // offset of W[ky][kx][ci][co] in theta
    bf16* wf[kLayers];                  // [cin/32][9][4][cout][8] (input channels >= cin_real zero)
    bf16* wd[kLayers];                  // [cout/32][9][4][cin][8] of W[8 - tap] (null: not needed)
    int n;
};

// x0 [P][32] bf16, base [P][2] and tgt [P][2] (FP32, cells) from the samples
// (device array `smp` of B entries), canvases H8 x W8 with the real H x W.
cudaError_t launch_assemble(const Sample* smp, int B, int H, int W, int H8, int W8, bf16* x0,
                            float* base, float* tgt, cudaStream_t s);
// 3x3 convolution of the B x H x W maps of `in` with weights Wh in the
// [Cin/32][9][4][N][8] layout of launch_pack; *err (device) is set to 1 if a
// bounded wait expired.
cudaError_t launch_conv3(const ConvIn& in, const bf16* Wh, int Cin, int N, int B, int H, int W,
                         const ConvOut& out, int* err, cudaStream_t s);
// Partial weight gradients: part[s][9 Cin][N] (FP32) = sum over the s-th slice
// of pixels of im2col(in)^T G (tcgen05 tensor cores); returns the number of
// slices used in *splits; *err (device) as for launch_conv3.
cudaError_t launch_wgrad3(const ConvIn& in, const bf16* G, int Cin, int N, int B, int H, int W,
                          float* part, size_t part_cap, int* splits, int* err, cudaStream_t s);
// Partial column sums part[s][N] of G [P][N].
cudaError_t launch_colsum(const bf16* G, long long P, int N, float* part, size_t part_cap,
                          int* splits, cudaStream_t s);
// grad[w_off + (tap cin_real + ci) N + co] = sum_s wpart[s][tap cin + ci][co]
// (ci < cin_real) and grad[b_off + co] = sum_s bpart[s][co].
cudaError_t launch_reduce_grad(const float* wpart, int ws, int cin, int cin_real, int N,
                               const float* bpart, int bs, float* grad, long long w_off,
                               long long b_off, cudaStream_t s);
// y [B][H/2][W/2][C] = bf16(mean of 2x2 blocks of x [B][H][W][C]).
cudaError_t launch_pool2(const bf16* x, bf16* y, int B, int H, int W, int C, cudaStream_t s);
// g [B][H][W][C] = bf16((dp[n][y/2][x/2][c] / 4 + skip[n][y][x][c]) * slope(e)).
cudaError_t launch_combine(const float* dp, const float* skip, const bf16* e, bf16* g, int B, int H,
                           int W, int C, cudaStream_t s);
// g [B][H/2][W/2][C] = bf16(sum of 2x2 blocks of f [B][H][W][C] * slope(d)).
cudaError_t launch_upback(const float* f, const bf16* d, bf16* g, int B, int H, int W, int C,
                          cudaStream_t s);
// Head (1x1 conv 32 -> 2 in FP32): z = h (base + delta) to the samples' `out`
// (train = 0); with train = 1 also the loss terms and gradients: part
// [blocks][67] = {sum e^2, dW[32][2], db[2]} and gd0 = bf16(W gdelta * slope(d0)).
cudaError_t launch_head(const bf16* d0, const float* theta_head, const float* base,
                        const float* tgt, const Sample* smp, int B, int H, int W, int H8, int W8,
                        int train, float inv_count, float* part, int* blocks, bf16* gd0,
                        cudaStream_t s);
// Sums the head partials: grad[off .. off + 66) and *loss (sum e^2 / count).
cudaError_t launch_reduce_head(const float* part, int blocks, float* grad, long long off,
                               float inv_count, double* loss, cudaStream_t s);
// Adam (FP32): m, v, theta updated in place; c1 = 1 / (1 - b1^t), c2 = 1 / (1 - b2^t).
cudaError_t launch_adam(float* theta, float* m, float* v, const float* g, long long n, float lr,
                        float b1, float b2, float eps, float c1, float c2, cudaStream_t s);
// One CTA waiting, with the convolutions' bound, on an mbarrier nothing
// completes; *expired (device) = 1 when the wait gave up as designed.
cudaError_t launch_wait_probe(int* expired, cudaStream_t s);
// BF16 copies of every layer's weights in the GEMM layouts.
cudaError_t launch_pack(const float* theta, const PackTable& t, cudaStream_t s);
// dst[i] = bf16(src[i]) and back.
cudaError_t launch_to_bf16(const float* src, bf16* dst, long long n, cudaStream_t s);
cudaError_t launch_from_bf16(const bf16* src, float* dst, long long n, cudaStream_t s);

}  // namespace net
}  // namespace stml

// ---------------------------------------------------------- host runtime
struct stml_net;

namespace stml {
namespace net {
// True when a level of H x W pixels fits the network's canvas.
bool fits(const ::stml_net* n, int H, int W);
int max_batch(const ::stml_net* n);
// True (and the flag cleared) if a convolution's bounded wait expired; synchronous.
bool timed_out(::stml_net* n);
// Proposals of B <= max_batch samples (host descriptors) on stream s.
cudaError_t forward_on(::stml_net* n, const Sample* host_smp, int B, int H, int W, cudaStream_t s);
}  // namespace net
}  // namespace stml
