/* Learned temporal predictor of the STML library.
 *
 * The predictors of Sec. 3 (linear interpolation on the coarsest level, the
 * least-squares predictor of eq. (2) on finer ones) propose the field of every
 * frame k that the next temporal level K_{q+1} adds, from the fields
 * registered on K_q.  A stml_net is a convolutional encoder-decoder that
 * proposes it instead from the two registered neighbours l < k < r of k and
 * the three images:
 *
 *   z_k = h (base + delta),  base = (w_l y_l + (1 - w_l) y_r) / h,
 *   delta = N_theta(y_l / h, y_r / h, T_l, T_k, T_r),  w_l = (r - k) / (r - l),
 *
 * h the cell width of the level.  Attached to a context (stml_set_predictor_net)
 * it is used at every predictor step of a 2-D STML registration whose level fits
 * its canvas: the proposals replace the classical ones only when the objective
 * of eq. (1) over the next temporal set (over all frames for the fill after the
 * stopping rule of eq. (3)) is lower there.
 *
 * Network (2-D, 906274 parameters): four levels of two 3x3 convolutions with
 * 32, 64, 96 and 128 channels (2x2 mean pooling between them), a decoder of
 * nearest-neighbour upsampling, skip connections and two 3x3 convolutions per
 * level (96, 64, 32 channels), leaky ReLU (slope 0.1) after every 3x3
 * convolution, and a 1x1 head to 2 channels.  The input is zero-padded to
 * multiples of 8 pixels.  Convolutions multiply BF16 operands (weights,
 * activations and the gradients with respect to pre-activations) and
 * accumulate in FP32; the head, the loss and Adam run in FP32.
 *
 * Parameter vector (FP32, host memory in this interface): for each of the 14
 * convolutions in the order e0a (7->32), e0b (32->32), e1a (32->64),
 * e1b (64->64), e2a (64->96), e2b (96->96), ba (96->128), bb (128->128),
 * d2a (224->96), d2b (96->96), d1a (160->64), d1b (64->64), d0a (96->32),
 * d0b (32->32): its weights W[ky][kx][ci][co] then its bias[co]; then the
 * head's W[ci][co] (32 x 2) and bias[2].  Input channels of e0a: y_l / h (2),
 * y_r / h (2), T_l, T_k, T_r; the decoder's first convolutions take
 * [upsampled coarser map, encoder map of the same level].
 *
 * Errors follow stml.h: STML_EINVAL for bad arguments (nothing launched),
 * STML_ECUDA when a CUDA call failed (destroy the network).  A network is used
 * by one host thread at a time; its calls run on the stream given at creation
 * (inside a registration: on the context's stream).
 */
#ifndef STML_NET_H
#define STML_NET_H

#include <stddef.h>

#include "stml.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct stml_net stml_net;   /* opaque; owns its device memory */

/* One sample: device pointers to FP32 arrays.  Fields are (2, H, .) with
 * component planes `plane` floats apart and rows `ld` floats apart (a crop of
 * a larger field is a pointer to its first pixel); images are (H, .) with rows
 * `ld_img` floats apart. */
typedef struct {
    const float* y_l;        /* left neighbour's field (physical units of the level) */
    const float* y_r;        /* right neighbour's field */
    const float* T_l;        /* images of frames l, k, r at the level */
    const float* T_k;
    const float* T_r;
    const float* target;     /* registered field of frame k (training), or NULL */
    float* out;              /* proposal z_k (stml_net_forward), or NULL */
    long long plane;
    int ld;
    int ld_img;
    float w_l;               /* (r - k) / (r - l), in [0, 1] */
    float h;                 /* cell width of the level, > 0 */
} stml_net_sample;

typedef struct {
    double lr, beta1, beta2, eps;    /* Adam (Kingma & Ba): defaults 1e-3, 0.9, 0.999, 1e-8 */
} stml_adam;

/* Number of parameters (906274). */
size_t stml_net_param_count(void);

/* Creates a network with parameters `params` (host, stml_net_param_count()
 * floats) and buffers for batches of up to max_batch samples of up to
 * max_h x max_w pixels, on `cuda_stream` (NULL: legacy default stream). */
stml_status stml_net_create(const float* params, size_t n_params, int max_batch, int max_h, int max_w,
                            void* cuda_stream, stml_net** out);
void stml_net_destroy(stml_net* net);
const char* stml_net_last_error(const stml_net* net);

/* Replaces the parameters (host array) and resets Adam's moments and step. */
stml_status stml_net_set_params(stml_net* net, const float* params, size_t n_params);
/* Copies the parameters to the host array (synchronises the stream). */
stml_status stml_net_get_params(stml_net* net, float* params, size_t n_params);

/* Proposals z_k of B samples (host array of descriptors) of H x W pixels,
 * written to each sample's `out` (asynchronous on the stream). */
stml_status stml_net_forward(stml_net* net, const stml_net_sample* samples, int B, int H, int W);

/* Loss L = mean over the B x 2 x H x W outputs of (z_k - target)^2 / h^2 (in
 * cells) and, when grad is not NULL, dL/dtheta (host, stml_net_param_count()
 * floats).  Synchronises the stream. */
stml_status stml_net_loss_grad(stml_net* net, const stml_net_sample* samples, int B, int H, int W,
                               double* loss, float* grad);

/* One Adam step on the loss of the batch (opt NULL: the defaults).  With
 * loss not NULL the stream is synchronised and the batch's loss (before the
 * step) is returned; otherwise the call is asynchronous. */
stml_status stml_net_train_step(stml_net* net, const stml_net_sample* samples, int B, int H, int W,
                                const stml_adam* opt, double* loss);

/* One 3x3 convolution of the network's kind on channels-last FP32 device
 * arrays, for checking the convolution kernels layer by layer.  Inputs are
 * rounded to BF16 on entry (like the network's operands); W is
 * [ky][kx][ci][co] (9 Cin Cout floats), Cin and Cout multiples of 32:
 *   mode 0 (forward):        y (B,H,W,Cout) = bf16(leaky(conv3(x, W) + b)),  x (B,H,W,Cin)
 *   mode 1 (input gradient): y (B,H,W,Cin)  = conv3 adjoint of x (B,H,W,Cout), FP32
 *   mode 2 (weight gradient): y = [dW (9 Cin Cout), db (Cout)] of <x, conv3(a, W) + b>
 *                             for x (B,H,W,Cout) and a (B,H,W,Cin), FP32
 * Allocates and frees its own scratch memory; synchronises `cuda_stream`. */
stml_status stml_net_conv3_block(int mode, const float* x, const float* a, const float* W, const float* b,
                                 float* y, int B, int H, int W_, int Cin, int Cout, void* cuda_stream);

/* Failure-detection self-check: one CTA waits, with the bound of the
 * convolution kernels' mbarrier waits, on an mbarrier that nothing completes;
 * *expired = 1 when the wait gave up and the kernel returned (the designed
 * behaviour: the network calls then report STML_ETIMEOUT).  Takes up to a
 * second; synchronises `cuda_stream`.  A convolution whose wait expires
 * gives its tensor-core work still in flight one more bounded wait before it
 * releases its tensor memory; if that wait expires as well, the error text of
 * STML_ETIMEOUT says so, results are undefined and the CUDA context should be
 * discarded. */
stml_status stml_check_bounded_wait(void* cuda_stream, int* expired);

/* Attaches a network to a context as its temporal predictor (NULL detaches).
 * The network must outlive the attachment and serve one context at a time;
 * stml_register_batch refuses contexts that share a network. */
stml_status stml_set_predictor_net(stml_ctx* ctx, stml_net* net);

#ifdef __cplusplus
}
#endif

#endif /* STML_NET_H */
