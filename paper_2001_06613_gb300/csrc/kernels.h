// Host-side launchers of the STML kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <initializer_list>

#include <string>

#include "common.cuh"

namespace stml {

// A stored array and its element type (StoreType).
struct Stored {
    const void* p;
    int type;
};

// Calls f with a value of the element type named by a StoreType.
template <typename F>
auto with_store_type(int st, F&& f) {
    if (st == ST_F16) return f(__half{});
    if (st == ST_BF16) return f(__nv_bfloat16{});
    return f(float{});
}

// Launch attributes of a programmatic dependent launch on stream s: the
// kernel may start its CTAs while the previous kernel of the stream is still
// finishing (it waits in pdl_enter until that kernel has completed).  This
// hides the ~2 us between the end of one kernel and the start of the next in
// a chain of dependent launches.  Left out while s is being captured into a
// graph, where the launches keep plain stream order.  Returns the number of
// attributes written to at (0 or 1).
inline unsigned pdl_attr(cudaStream_t s, cudaLaunchAttribute* at) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        (void)cudaGetLastError();
        return 0;
    }
    at->id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at->val.programmaticStreamSerializationAllowed = 1;
    return 1;
}

// Launches kernel k (whose first statement is pdl_enter()) on `grid` x
// `block` threads with `smem` bytes of dynamic shared memory on stream s as
// a programmatic dependent launch.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
    cudaLaunchConfig_t lc = {};
    lc.gridDim = grid;
    lc.blockDim = block;
    lc.dynamicSmemBytes = smem;
    lc.stream = s;
    cudaLaunchAttribute at[1];
    lc.numAttrs = pdl_attr(s, at);
    lc.attrs = at;
    return cudaLaunchKernelEx(&lc, k, static_cast<KArgs>(args)...);
}

// Sets the text stml_last_error(NULL) returns (errors of context-free calls).
void set_context_free_error(const std::string& msg);

// Every launcher adds the number of kernels it launched to this counter.
long long launches_total();
void count_launches(int k);

// CTAs of a grid-stride launch of `kernel` at kThreads per CTA: the CTAs
// that are resident at once (SMs x CTAs per SM at the kernel's register and
// shared-memory use, queried once per kernel), at most `items` and at most
// `cap`.  A grid larger than that runs in waves, and a CTA of the second wave
// works on items far from those in flight, losing the L2 reuse of the
// neighbouring frames and rows.
// Cached per (device, kernel), so a process that uses several GPUs sizes each
// grid for the device it launches on.
unsigned resident_grid(const void* kernel, long long items, unsigned cap);

// Streaming multiprocessors of the current device (cached per device; 0 if
// the query fails).
int device_sms();

// Raises the dynamic shared-memory limit of `kernel` on the current device to
// `bytes` (cudaFuncSetAttribute is per device; done once per device and kernel).
cudaError_t set_max_dynamic_smem(const void* kernel, int bytes);

// Geometry of a level from its shape (nz, ny, nx), dimension and cell width.
Geom make_geom(const int shape3[3], int d, float h);

// Divisors of a level's pixel index (x, y, z).
PixIndex make_pix_index(const Geom& g);

// CTAs for n work items at `threads` per CTA, capped for grid-stride loops.
inline unsigned blocks_for(long long n, int threads = kThreads, long long cap = 1 << 20) {
    long long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (unsigned)b;
}

// Pixels per CTA of the kernels that loop over the frames of a pixel: one
// warp-wide row of pixels, the frames split over the 8 warps of the CTA.
constexpr int kPixPerCta = 32;
constexpr int kFrameGroups = kThreads / kPixPerCta;

// ------------------------------------------------------------ affine (Sec. 4)
// Centre c (finest-level pixels, per array axis) and 1 / rho of the affine
// parametrisation u_k(x) = W_k (x - c) / rho + b_k.
struct AffineFrame {
    float c[3];
    float inv_rho;
};
// u (nK, d, N) from theta (nK, d(d+1)) on the device.
cudaError_t launch_affine_field(const Geom& g, const AffineFrame& af, const float* theta, int nK, float* u,
                                cudaStream_t s);
// out (nK, d(d+1), FP64) = projection of the field gradient gu (nK, d, N);
// part holds nK * affine_project_blocks(g) * d(d+1) doubles.
int affine_project_blocks(const Geom& g);
cudaError_t launch_affine_project(const Geom& g, const AffineFrame& af, const float* gu, int nK, double* part,
                                  double* out, cudaStream_t s);

// Normalised-correlation distance of the affine variant: warped frames a
// (nK x N), grad T (nK x d x N), per-frame means mu (part: nK * 256 * 2
// doubles); Gram matrix G (nK x nK doubles) about the means (part:
// nc_gram_splits * nK^2 doubles); gu = (Q (a - mu)) grad T for the K x K Q.
cudaError_t launch_nc_warp(const Stored& T, const Geom& g, const FrameSet& fs, const float* u, float* a, float* dT,
                           double* part, float* mu, cudaStream_t s);
int nc_gram_splits(const Geom& g, int nK);
cudaError_t launch_nc_gram(const Geom& g, const float* a, const float* mu, int nK, double* part, double* G,
                           cudaStream_t s);
cudaError_t launch_nc_grad(const Geom& g, const float* a, const float* mu, const float* Q, const float* dT, int nK,
                           float* gu, cudaStream_t s);
// From the Gram matrix G: srow_i = sum_j rho_ij^2, the gradient matrix Q and
// D_NC (device double) -- the host needs no step between Gram and gradient.
cudaError_t launch_nc_coeff(const double* G, int nK, double* srow, float* Q, double* D, cudaStream_t s);

// ---------------------------------------------------------- transfer ops
// 2^d block mean of `planes` stored arrays of 2 gc (type: StoreType).
cudaError_t launch_restrict(const void* fine, void* coarse, int type, int planes, const Geom& gc,
                            cudaStream_t s);
// float <-> stored type, n values.
cudaError_t launch_to_store(const float* src, void* dst, int type, long long n, cudaStream_t s);
cudaError_t launch_from_store(const void* src, int type, float* dst, long long n, cudaStream_t s);
cudaError_t launch_prolong(const float* coarse, float* fine, int planes, const Geom& gc,
                           cudaStream_t s);
cudaError_t launch_prolong_adjoint(const float* fine, float* coarse, int planes, const Geom& gc,
                                   cudaStream_t s);

// Linear temporal predictor: for every target t, out[dst_t] = wl_t * in[src_l] + wr_t * in[src_r].
struct LinTap {
    int dst, src_l, src_r, pad;
    float wl, wr;
};
cudaError_t launch_predict_linear(const float* in, float* out, const LinTap* taps, int nT,
                                  size_t plane_elems, cudaStream_t s);

// Thomas sweep for eq. (2): factors cp, inv_den, sub (n floats each) and
// kidx (n ints, index into eta or -1) in device memory.
cudaError_t launch_predict_ls(const float* eta, const float* omega, float* zeta, const float* cp,
                              const float* inv_den, const float* sub, const int* kidx, int n,
                              size_t ncomp, cudaStream_t s);

// Copies planes: dst[j] = src[idx[j]] (gather) for j < nK, each plane_elems floats.
cudaError_t launch_gather_planes(const float* src, float* dst, const int* idx, int nK,
                                 size_t plane_elems, cudaStream_t s);
// dst[idx[j]] = src[j] (scatter).
cudaError_t launch_scatter_planes(const float* src, float* dst, const int* idx, int nK,
                                  size_t plane_elems, cudaStream_t s);

cudaError_t launch_corr_coeff(const void* img, int type, int n, long long N, double* rho_dev, cudaStream_t s);

// ---------------------------------------------------------- objective (k_eval.cu)
// Objective pass at u (or u + t du): J, D, S, P, |u|^2 to out[0..3], out[5]
// (out[4] = 0), and the per-pixel frame means abar (N) and ubar (d N).
// With gdot (requires du) the pass also reduces <gdot, du> and |du|^2 into out[6], out[7].
// Armijo trial k (t = 2^-k) of a line search decided on the device: the
// trial does nothing once an earlier one was accepted (or trial 0 found no
// descent); its last CTA applies J(u + t d) <= J + c t <g, d> and records the
// outcome in S (ls_*).  Trial 0 must carry gdot.
struct LineSearchArgs {
    DevScalars* S;
    int k;
    double J;
    double c;
};
// Launch shape of the objective pass: pixels per lane (4, 2 or 1; 1 or 2 in
// 3-D) and frame splits (1..8, one thread-block cluster per pixel run).
struct ObjShapeChoice {
    int vec;
    int splits;
};
// The shapes an autotuner may try for this level and frame count.
int obj_shape_candidates(const Geom& g, int nK, ObjShapeChoice* out, int cap);
cudaError_t launch_objective(const Stored& T, const Geom& g, const FrameSet& fs, const Coef& cf, const float* u,
                             const float* du, float t, const float* gdot, float* abar, float* ubar, double* partials,
                             size_t partials_cap, unsigned int* ticket, double* out, cudaStream_t s,
                             const LineSearchArgs* ls = nullptr, const ObjShapeChoice* shape = nullptr);
// Gradient pass at u (or u + t du) with abar, ubar of the same point: g and
// grad T, optionally the point itself (unew); |g|^2 and |u|^2 to out[4], out[5].
// With gate != nullptr it runs only if gate->ls_accepted, with t = gate->ls_t.
// grad T is written as float (dT_type ST_F32) or in the image's storage type.
cudaError_t launch_gradient(const Stored& T, const Geom& g, const FrameSet& fs, const Coef& cf, const float* u,
                            const float* du, float t, const float* abar, const float* ubar, float* grad, void* dT,
                            int dT_type, float* unew, double* partials, size_t partials_cap, unsigned int* ticket,
                            double* out, cudaStream_t s, const DevScalars* gate = nullptr);
// Doubles of partial sums the evaluation kernels need.
size_t eval_partials(const Geom& g, int nK);

// ---------------------------------------------------------- Hessian product
struct HessWork {
    float* mean_s;     // N
    float* sum_v;      // d * N
    double* partials;
    size_t partials_cap;
};

// Hv and <v, Hv> (to out[0]) for a given v: per-pixel frame sums, then the
// stencil stream.  With pcg != nullptr the launch is a step of the device-side
// PCG: it does nothing once cg_active is 0, and its last CTA sets
// alpha = rho / <p, Hp> (or flags a breakdown).
cudaError_t launch_hessvec(const Geom& g, const FrameSet& fs, const Coef& cf, const float* dT,
                           const float* v, float* Hv, HessWork& w, unsigned int* ticket,
                           double* out, DevScalars* pcg, cudaStream_t s);

// Doubles of partial sums the Gauss-Newton kernels need for a problem of this size.
size_t gn_partials(const Geom& g, int nK);

// The two halves of the Hessian product (k_gn.cu): per-pixel frame sums of v
// (mean of grad T . v, sum of v) and the stencil stream that uses them.
cudaError_t launch_hess_sums(const Geom& g, const FrameSet& fs, const float* dT, const float* v, float* mean_s,
                             float* sum_v, cudaStream_t s, const int* gate = nullptr);
cudaError_t launch_hess_apply(const Geom& g, const FrameSet& fs, const Coef& cf, const float* dT, const float* v,
                              const float* mean_s, const float* sum_v, float* Hv, double* partials,
                              size_t partials_cap, unsigned int* ticket, double* out, DevScalars* pcg,
                              cudaStream_t s);

// ---------------------------------------------------------- PCG vector ops
struct PcgArgs {
    float tol_cg;
    int max_cg;
};
// Vectors of one PCG solve (all n d N floats unless noted).  The streaming
// solve keeps its direction in p[0] and the direction's frame sums in
// ms_z / sv_z.  The cooperative solve keeps z = M^-1 r in z and its sums in
// ms_z / sv_z, and double-buffers the direction and its sums: iteration k
// writes p[k & 1] from p[(k + 1) & 1]; p_0 = z_0 lands in p[0] either way.
struct PcgBufs {
    float* x;
    float* r;
    float* z;                      // M^-1 r (cooperative solve)
    float* q;                      // H p
    float* p[2];
    float* ms_z;                   // frame sums: mean of grad T . w (N) ...
    float* sv_z;                   // ... and sum of w (d N)
    float* ms_p[2];                // frame sums of p (cooperative solve)
    float* sv_p[2];
};
// r = -g, p = M^-1 r, x = 0, the frame sums of p; rho = <r, M^-1 r>, |r|^2.
// With gate != nullptr the start runs only if *gate is nonzero (otherwise
// cg_active keeps its value, 0 after any finished solve).
cudaError_t launch_pcg_init(const Geom& g, const FrameSet& fs, const Coef& cf, const float* grad, const Stored& dT,
                            const PcgBufs& b, double* partials, size_t partials_cap, DevScalars* S, PcgArgs a,
                            cudaStream_t s, const int* gate = nullptr);
// q = H p (from p and its frame sums); alpha = rho / <p, q>.
cudaError_t launch_pcg_apply(const Geom& g, const FrameSet& fs, const Coef& cf, const Stored& dT, const PcgBufs& b,
                             double* partials, size_t partials_cap, DevScalars* S, cudaStream_t s);
// x += alpha p, r -= alpha q; rho, the convergence test and beta.
cudaError_t launch_pcg_update(const Geom& g, const FrameSet& fs, const Coef& cf, const Stored& dT, const PcgBufs& b,
                              double* partials, size_t partials_cap, DevScalars* S, PcgArgs a, cudaStream_t s);
// p = M^-1 r + beta p and the frame sums of the new p.
cudaError_t launch_pcg_direction(const Geom& g, const FrameSet& fs, const Coef& cf, const Stored& dT,
                                 const PcgBufs& b, DevScalars* S, cudaStream_t s);
// The whole PCG solve (start, iterations, exit) in one cooperative launch, for
// small problems where launch latency dominates; the final CG state goes to S.
bool pcg_coop_preferred(const Geom& g, int nK);
cudaError_t launch_pcg_coop(const Geom& g, const FrameSet& fs, const Coef& cf, const float* grad, const Stored& dT,
                            const PcgBufs& b, double* partials, size_t partials_cap, DevScalars* S, PcgArgs a,
                            cudaStream_t s, const int* gate = nullptr);

// ---------------------------------------------------------- batched solver (k_batch.cu)
// One sequence of a batched stage: its level geometry and frame set, the
// solver buffers of its context (all nK d N floats unless noted) and the
// counts of its work items.
struct BatchSeq {
    Geom g;
    PixIndex pi;
    FrameSet fs;
    Coef cf;
    FastDiv cpf;             // chunks of kThreads * VEC pixels per frame (Hessian-product items)
    unsigned eval_tiles;     // tiles of 32 VEC pixels (objective and gradient)
    unsigned pcg_tiles;      // tiles of TPR VEC pixels (PCG start and update)
    unsigned chunks;         // nK * cpf
    const void* T;           // images of the level, all frames (storage type of the batch)
    float* u[2];             // the iterate and the next point (they swap at every accepted step)
    float* grad;
    void* dT;                // grad T in the image storage type
    float *x, *r, *z, *q;
    float* p[2];
    float *ms_z, *sv_z;      // frame sums of z: mean of grad T . z (N), sum of z (d N)
    float* ms_p[2];
    float* sv_p[2];
    float *abar, *ubar;      // per-pixel frame means (N, d N)
    double target;           // target objective of this GIR (0: none), see stml_params.target_J
    double target_tol;
};

// Phases of a sequence's state machine.
// LAND: objective at u + t d during the regula falsi that shortens the step
// crossing the target objective.
enum BatchPhase { BPH_EVAL0 = 0, BPH_INIT, BPH_APPLY, BPH_UPDATE, BPH_TRIAL, BPH_GRAD, BPH_LAND, BPH_DONE };

// Device state of one sequence (written by the first CTA of its range only).
struct BatchState {
    int phase, cur;          // next phase; u[cur] is the iterate
    int it, cg_total, ls_total;
    int ls_k, dir_p0;        // Armijo trial index; the direction is p[0] (first CG step broke down)
    int status;              // stml_status of the GIR
    int cg_k, cg_iter, cg_flag, cg_active;
    float cg_rho, cg_bnorm2, cg_rnorm2, cg_pq, cg_alpha, cg_beta;
    float t;                 // step of the current / accepted trial
    int pad;
    double J0, J, Jold, D, S, P, gnorm2, unorm2, step;
    double gTd, dnorm2;
    double Jt, Dt, St, Pt;   // totals of the last trial
    // landing on the target: the bracket [la, lb] of the step, J - target at
    // its ends, the best point so far; land_final: the next GRAD ends the GIR
    double la, lfa, lb, lfb, best_t, best_f, best_J, best_D, best_S, best_P;
    int side, land_it, land_final, land_pad;
};

// Solver parameters of the batch (stml_params of its contexts).
struct BatchCtl {
    float tol_cg;
    int max_cg, max_gn, max_ls;
    double armijo_c, tol_J, tol_Y, tol_G, g_abs;
};

// Barrier words and the error flag (bit 0: a bounded wait expired); zero at launch.
struct BatchSync {
    unsigned count, gen, err, steps;
};

// Launch shapes of the batched kernel: CTAs per SM and lanes per pixel row
// of the PCG tiles (4 or 16; the evaluation tiles are one warp wide).
struct BatchShape {
    int ctas_per_sm;
    int tpr;
};
// VEC: 4 when every sequence has nx % 4 == 0 and 16-byte aligned buffers, else 1.
// d: 2 or 3; img_type: StoreType of images and grad T.  part: gridDim * 8
// float2 slots (batch_partials); the launch is cooperative (all CTAs resident).
size_t batch_partials(int ctas);
int batch_grid(int d, int vec, int img_type, const BatchShape& sh);
// Self-check of the bounded grid barrier: one CTA waits on a barrier that
// expects two; *expired (device int) = 1 when the wait gave up (about 2 s).
cudaError_t launch_batch_barrier_probe(BatchSync* sync, int* expired, cudaStream_t s);
cudaError_t launch_batch_gir(const BatchSeq* seqs_dev, int nseq, BatchState* states, const BatchCtl& ctl, int d,
                             int vec, int img_type, const BatchShape& sh, float2* part, BatchSync* sync,
                             int max_steps, cudaStream_t s);

// ------------------------------------------------- coarse displacement grid (k_ugrid.cu)
// The image grid (nx, ny, nz; N cells per plane) and the grid of the
// unknowns, coarser by F = 2^s per axis (cx, cy, cz; Nc cells per plane).
struct UGrid {
    int nx, ny, nz;
    int cx, cy, cz;
    int d, F;
    float inv_F;
    long long N, Nc;
};
UGrid make_ugrid(const Geom& fine, int s);
// Device-resident state of a coarse-grid PCG solve: the coefficients (FP64,
// applied in float), the stopping threshold tol_cg ||g||, the step count and
// the CG_* flag.  `mirror` (may be null) receives `active` as well, for the
// image-grid kernels of the Hessian product that are gated on it.
struct UgCg {
    double rho, thr, alpha, beta, pq, rnorm2;
    int active, iter, flag, max_cg;
    int* mirror;
};
// u = P_s (w + t dw) for `planes` planes (dw may be null); nothing when
// gate != null and *gate == 0.
cudaError_t launch_ugrid_prolong(const float* w, const float* dw, float t, float* u, long long planes,
                                 const UGrid& ug, cudaStream_t s, const int* gate = nullptr);
// out = P_s^T f (fixed-order gather per coarse value); gated like the prolongation.
cudaError_t launch_ugrid_adjoint(const float* f, float* out, long long planes, const UGrid& ug, cudaStream_t s,
                                 const int* gate = nullptr);
// Minv = 1 / Jacobi diagonal of the coarse-grid Hessian from the image-grid
// grad T (float), cf the image grid's and cw the coarse grid's coefficients.
cudaError_t launch_ugrid_jacobi(const float* dT, float* Minv, const UGrid& ug, const FrameSet& fs, const Coef& cf,
                                const Coef& cw, cudaStream_t s);
// S and P on the coarse grid gw at w + t dw; mode 0: objective sums (5
// values to out) and, with gout, the gradient gin + regulariser/penalty
// gradient; mode 1: gout = gin + their Hessian product, out[0] = <w, gout>;
// with cg (mode 1, a PCG step): nothing once cg->active is 0, and the last
// CTA takes alpha = rho / <p, Hp> or the breakdown decision.
cudaError_t launch_ugrid_reg(int mode, const Geom& gw, const FrameSet& fs, const Coef& cw, const float* w,
                             const float* dw, float t, const float* gin, float* gout, double* partials,
                             size_t partials_cap, unsigned int* ticket, double* out, cudaStream_t s,
                             UgCg* cg = nullptr);
enum UgridVecMode { VEC_INIT = 0, VEC_STEP = 1, VEC_DIR = 2, VEC_DOT = 3, VEC_AXPY = 4 };
// PCG vector steps and dot products over n coarse values (see k_ugrid.cu).
// With cg: VEC_INIT starts the solve (thr = tol_cg ||g||), VEC_STEP and
// VEC_DIR take alpha / beta from it and do nothing once it stopped, and
// VEC_STEP's last CTA takes the stopping decision.
cudaError_t launch_ugrid_vec(int mode, long long n, float a, const float* Minv, float* x, float* r, float* z,
                             float* p, const float* q, const float* g, double* partials, size_t partials_cap,
                             unsigned int* ticket, double* out, cudaStream_t s, UgCg* cg = nullptr,
                             double thr = 0.0, int max_cg = 0);

}  // namespace stml
