/*
 * stml.h -- C ABI of the GB300 spatio-temporal multilevel (STML) registration library.
 *
 * The library registers an image sequence groupwise (Sec. 2, eq. 1 of
 * Aggrawal & Modersitzki, "Accelerating the Registration of Image Sequences by
 * Spatio-temporal Multilevel Strategies") with the predictor-corrector sweep
 * over a spatial pyramid and a temporal binary tree (Sec. 3, Fig. 1, eqs. 2-3).
 * Every step of the computation runs in CUDA kernels on one GPU; this header
 * uses plain pointers and sizes only.
 *
 * Conventions shared by all entry points
 * --------------------------------------
 * - Grids are cell-centred.  `shape` lists the cells per axis in C order
 *   (2-D: {ny, nx}; 3-D: {nz, ny, nx}); x varies fastest in memory.  Level 0 is
 *   the coarsest of `n_levels` spatial levels; level l has cell width
 *   h = 2^(n_levels-1-l) finest pixels and shape = finest_shape / h.
 * - Images: float32, layout [frame][z][y][x].
 * - Displacement fields: float32, layout [frame][component][z][y][x] in finest
 *   pixel units; component c moves along axis c of `shape` (2-D: c=0 is y,
 *   c=1 is x).  The transformation of frame k is y_k(x) = x + u_k(x).
 * - Frame subsets (`frames`, `K`) are host int arrays of strictly increasing
 *   0-based frame numbers.
 * - Pointers documented as "device" must point to device memory of the GPU
 *   that was current when the context was created; "host" pointers to host
 *   memory.  Device field arrays passed to stml_eval, stml_hessvec, stml_gir
 *   and stml_hessvec_noalloc must be 16-byte aligned (cudaMalloc and torch
 *   allocations are); others return STML_EINVAL.  The library never takes
 *   ownership of caller memory.
 * - All work is ordered on the CUDA stream given to stml_create (or passed to
 *   the context-free operators); calls that return host values synchronise
 *   that stream only.
 * - No C++ exception crosses this boundary.  Every entry point returns a
 *   stml_status; on error, stml_last_error() describes it.  A context stays
 *   usable after STML_EINVAL; after STML_ECUDA it should be destroyed.
 */
#ifndef STML_H
#define STML_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct stml_ctx stml_ctx;   /* opaque; owns all device memory it allocates */

typedef enum {
    STML_OK = 0,
    STML_EINVAL = -1,        /* bad argument or shape */
    STML_ENOMEM = -2,        /* device allocation failed */
    STML_ECUDA = -3,         /* a CUDA call failed */
    STML_ENONFINITE = -4,    /* a NaN or Inf appeared in the objective */
    STML_EBREAKDOWN = -5,    /* PCG met p^T H p <= 0 */
    STML_ELINESEARCH = -6,   /* Armijo found no acceptable step */
    STML_ETIMEOUT = -7,      /* a bounded device wait expired */
    STML_ESTATE = -8         /* call out of order (e.g. no sequence loaded) */
} stml_status;

typedef enum { STML_MODE_STML = 0, STML_MODE_SPML = 1 } stml_mode;

/* Storage of the image pyramid and of the solver's image gradient grad T
 * (mixed precision): every value is computed in FP32 and rounded to nearest
 * even when stored; objective terms, PCG coefficients and the Armijo test keep
 * their double-float / FP64 reductions.  Fields are always FP32. */
typedef enum { STML_DTYPE_F32 = 0, STML_DTYPE_F16 = 1, STML_DTYPE_BF16 = 2 } stml_dtype;

/* Solver parameters.  Objective terms (Sec. 2, eq. 1):
 *   J = hd/2 sum_k ||a_k - mean_j a_j||^2                       (distance, a_k = R_k o y_k)
 *     + alpha/2 hd sum_k sum_c sum_i ||d_i u_{k,c}||^2           (spatial diffusion S)
 *     + alpha_t/2 hd sum_{consecutive k<k' in K} ||u_k' - u_k||^2 / (k'-k)^2
 *     + lambda hd ||(1/|K|) sum_j u_j||^2                         (penalty P)
 * with hd the cell volume of the level.  beta weighs eq. (2); eps_stop is the
 * relative per-frame tolerance of the stopping rule eq. (3). */
typedef struct {
    double alpha, alpha_t, lambda;
    double beta;
    double eps_stop;
    int stop_rule;           /* 1: apply eq. (3) for q > 0 */
    int n_levels;            /* spatial levels L >= 1 */
    int n_tlevels;           /* temporal levels Q >= 1 (q = 0..Q-1) */
    double tol_J, tol_Y, tol_G, g_abs;   /* Gauss-Newton stopping tests */
    int max_gn;
    double tol_cg;           /* PCG stops when ||r|| <= tol_cg ||g|| */
    int max_cg;
    int max_ls;              /* Armijo trials */
    double armijo_c;
    int image_dtype;         /* stml_dtype; fixed for a sequence when it is loaded */
    int pcg_cooperative;     /* 1: small levels solve PCG in one cooperative launch;
                              * 0: always the streaming kernels (required by
                              * stml_register_batch) */
    int autotune;            /* 1: the first call of each (level, frame count)
                              * times the objective pass's launch shapes and,
                              * for levels up to 2^23 pixel-frames, a
                              * cooperative against a
                              * streaming PCG solve, and keeps the fastest for
                              * the context (reproducible within a context);
                              * 0: built-in choices (default) */
    int transform;           /* 0: non-parametric fields (Gauss-Newton-PCG, the default);
                              * 1: one affine-linear map per frame (Sec. 4), solved by
                              * L-BFGS (Sec. 2); see stml_eval_affine */
    int lbfgs_m;             /* L-BFGS memory (pairs kept), 1..64 */
    int max_lbfgs;           /* L-BFGS iterations per GIR */
    int distance;            /* 0: sum of squared differences (eq. 1 as above);
                              * 1 (transform 1 only): normalised correlation,
                              * D = 1/2 sum_{i,j in K} (1 - rho_ij^2) with rho_ij the
                              * correlation of the warped frames i and j over the
                              * grid -- a reading of the SqN distance named in Sec. 2
                              * (1/2 (|K|^2 - sum of sigma^4 of the matrix of
                              * normalised frames)); S and P unchanged */
    double target_J;         /* > 0: the last GIR over all frames on the finest
                              * level (and stml_gir) stops where its objective
                              * first reaches target_J: the step that crosses it
                              * is shortened (regula falsi on its length) until
                              * |J - target_J| <= target_tol * target_J; a GIR
                              * that starts at or below target_J takes no step.
                              * Lets registrations that follow different paths
                              * end at the same objective.  0: off (default) */
    double target_tol;       /* relative tolerance of that landing (default 1e-5) */
    int u_coarsen;           /* s in 0..4: the unknown fields of every level live on its image
                              * grid coarsened by 2^s per axis (cell width 2^s h) and warp the
                              * images through u = P_s w, P_s the cell-centred multilinear
                              * interpolation with clamp-to-edge; the distance of eq. (1) is
                              * taken on the image grid, S and P of Sec. 2 on the coarse grid,
                              * and the gradient gathers the image-grid distance gradient
                              * through P_s^T (a reading of Sec. 2, which leaves the
                              * discretisation of the transformation to FAIR).  Fields
                              * (stml_get_field, stml_gir) are then on the coarse grid.  s > 0
                              * needs transform 0, image_dtype F32 and target_J 0; the
                              * predictor network is not used and stml_batch_register
                              * refuses the context; every image axis must be a multiple of
                              * 2^(n_levels-1+s).  0: the image grid (default) */
} stml_params;

typedef struct {
    int level, tlevel, n_frames;
    int gn_iters, cg_iters, ls_trials;
    int stopped_early;       /* eq. (3) ended this level after this temporal level */
    int status;              /* stml_status of the GIR (0, ELINESEARCH, EBREAKDOWN ...) */
    double J0, J, D, S, P;   /* objective at start and end of the GIR */
    double seconds;          /* wall time of the GIR on the stream */
    /* learned predictor (stml_net.h): -1 no learned proposal was made, 0 the
     * classical proposal was kept, 1 the learned one (lower objective) */
    int pred_learned;        /* for the start of this GIR */
    int fill_learned;        /* for the fill after eq. (3) ended the level here */
    double J0_classic;       /* objective at the classical start (pred_learned >= 0) */
    double J_fill_classic;   /* objective over all frames at the classical fill */
    double J_fill;           /* ... and at the kept fill (fill_learned >= 0) */
} stml_stats;

/* Fills *p with the library defaults (alpha 0.02, lambda 1, beta 1e-5, ...). */
void stml_default_params(stml_params* p);

/* Creates a context that will work on `cuda_stream` (a cudaStream_t, or NULL
 * for the legacy default stream) of the current device.  Returns STML_EINVAL
 * for invalid parameters. */
stml_status stml_create(const stml_params* p, void* cuda_stream, stml_ctx** out);

/* Frees every device allocation of the context. NULL is ignored. */
void stml_destroy(stml_ctx* ctx);

/* Text of the last error on ctx, or of the last context-free call when ctx is NULL. */
const char* stml_last_error(const stml_ctx* ctx);

/* Replaces the parameters (level counts must match the loaded sequence, if any). */
stml_status stml_set_params(stml_ctx* ctx, const stml_params* p);

/* ------------------------------------------------------------------ data */

/* Copies n_frames images of `shape` (dim = 2 or 3) from `frames` (host, or
 * device when on_device != 0) into library memory.  Every axis must be
 * divisible by 2^(n_levels-1) and have at most 65535 cells, and an image at
 * most 2^31 - 1 cells (pixel indices are 32-bit).  Allocates all level
 * buffers. */
stml_status stml_load_sequence(stml_ctx* ctx, const float* frames, int on_device,
                               int n_frames, int dim, const int* shape);

/* Builds the image pyramid by 2^d block means (Sec. 3; Sec. 4: smoothing in
 * space only) and the temporal sets K_q (Fig. 1). */
stml_status stml_build_pyramid(stml_ctx* ctx);

/* Shape (3 ints, z first; 1 for a missing axis) and cell width of a level. */
stml_status stml_level_info(const stml_ctx* ctx, int level, int* shape3, double* h);

/* Frames of K_q (Fig. 1): *count receives |K_q|; up to cap numbers are written. */
stml_status stml_temporal_set(const stml_ctx* ctx, int tlevel, int* frames, int cap, int* count);

/* Copies the images of all frames at `level` to dst (n * N floats). */
stml_status stml_get_images(stml_ctx* ctx, int level, float* dst, int dst_on_device);

/* Copies y_{level,all} (n * d * N floats) to dst / from src. */
stml_status stml_get_field(stml_ctx* ctx, int level, float* dst, int dst_on_device);
stml_status stml_set_field(stml_ctx* ctx, int level, const float* src, int src_on_device);

/* --------------------------------------------------------------- drivers */

/* Registers the loaded sequence from the coarsest to the finest level.
 * STML: predictor-corrector sweep over K_0..K_T at every level (Sec. 3) with
 * the stopping rule eq. (3); SpML: one GIR over all frames per level.
 * Per-GIR statistics go to stats[0..cap) and their number to *n_written
 * (either may be NULL).  The result is available via stml_get_field. */
stml_status stml_register(stml_ctx* ctx, stml_mode mode, stml_stats* stats, int cap,
                          int* n_written);

/* Registers the sequences of n_ctx contexts concurrently (batched serving of
 * many sequences of uneven length and size): up to max_threads host threads
 * (<= 0: one per context) each run stml_register on one context, whose work
 * goes to that context's own stream, so small sequences share the GPU.
 * Every context must hold a built pyramid and have pcg_cooperative = 0
 * (a cooperative launch needs the whole GPU), else STML_EINVAL before any
 * work starts; contexts must not share a stream.  status (host, n_ctx
 * entries, may be NULL) receives each context's result; the return value is
 * STML_OK or the first failure in context order.  Results equal those of
 * stml_register on each context alone. */
stml_status stml_register_batch(stml_ctx* const* ctxs, int n_ctx, stml_mode mode, int max_threads,
                                stml_status* status);

/* One predictor step of the STML sweep (Sec. 3): start values z_{l,q} on all
 * frames -- Id (level 0, q = 0), the prolongated y_{l-1,all} (q = 0), the
 * linear rule (level 0) or eq. (2) (finer levels) from y_{l,q-1}. */
stml_status stml_predict(stml_ctx* ctx, int level, int tlevel);

/* One corrector step: y_{l,q} = GIR(l, K_q) from z_{l,q}; applies eq. (3) for
 * q > 0 and, when it fires or q = T, completes y_{l,all}.  *finished (may be
 * NULL) is set to 1 when the level is complete. */
stml_status stml_correct(stml_ctx* ctx, int level, int tlevel, stml_stats* stats, int* finished);

/* --------------------------------------------- building blocks (device) */

/* Objective of eq. (1) with S and P on the level-`level` images of `frames`
 * at fields u (device, nK * d * N floats).  out (host, 6 doubles) receives
 * J, D, S, P, ||g||^2, ||u||^2.  g and dT (device, nK * d * N floats each)
 * receive the gradient and grad T_k(x + u_k(x)); pass NULL for both to
 * evaluate the objective only (then out[4] = 0). */
stml_status stml_eval(stml_ctx* ctx, int level, const int* frames, int nK, const float* u,
                      double* out, float* g, float* dT);

/* Objective at the trial point u + t d of an Armijo line search (the
 * objective of eq. (1) plus S and P as in stml_eval, no array formed), in the
 * launch the solver uses.  out (host, 8 doubles): J, D, S, P, 0, |u + t d|^2,
 * <gd, d>, |d|^2; the last two only when gd (the gradient at u, device,
 * same layout as u) is given, else 0.  u, d, gd are device arrays of
 * nK * d * N floats, 16-byte aligned. */
stml_status stml_eval_trial(stml_ctx* ctx, int level, const int* frames, int nK, const float* u,
                            const float* d, double t, const float* gd, double* out);

/* Gauss-Newton Hessian product Hv = J^T J v + alpha hd B^T B v + alpha_t hd L_t v
 * + 2 lambda hd / |K|^2 sum_j v_j (device arrays of nK * d * N floats, dT as
 * returned by stml_eval).  *vHv (host, may be NULL) receives <v, Hv>. */
stml_status stml_hessvec(stml_ctx* ctx, int level, const int* frames, int nK,
                         const float* dT, const float* v, float* Hv, double* vHv);

/* Runs the Gauss-Newton/PCG/Armijo scheme on the frames of K starting from
 * u (device, nK * d * N floats, overwritten with the result; with
 * params.u_coarsen = s > 0 the fields are on the coarse grid, nK * d * N / 2^(s d)
 * floats). */
stml_status stml_gir(stml_ctx* ctx, int level, const int* frames, int nK, float* u,
                     stml_stats* stats);

/* Coarse displacement grid (params.u_coarsen = s > 0; see stml_params).  The
 * unknowns w (device, nK * d * Nc floats, Nc = N / 2^(s d) cells of the
 * coarse grid of the level, layout [frame][component][cells]) warp the images
 * through u = P_s w.  stml_eval_ugrid: out (host, 6 doubles) = J, D, S, P,
 * ||g||^2, ||w||^2 with D the distance of eq. (1) at u on the image grid and S,
 * P of Sec. 2 on the coarse grid; g (coarse, may be NULL) = P_s^T (hd r_k grad
 * T_k) + alpha hd_w B^T B w_k + alpha_t hd_w (L_t w)_k + 2 lambda hd_w wbar / |K|
 * (hd_w = (2^s h)^d); dT (image grid, nK * d * N floats, may be NULL) = grad T
 * at the warped positions; Minv (coarse, may be NULL) = the inverse Jacobi
 * diagonal of the Gauss-Newton Hessian, (P_s o P_s)^T of the image-grid
 * distance diagonal plus the regulariser and penalty diagonal.
 * stml_hessvec_ugrid: Hv = P_s^T H_D P_s v + alpha hd_w B^T B v + alpha_t hd_w
 * L_t v + 2 lambda hd_w / |K|^2 sum_j v_j (H_D the distance part of the
 * image-grid Hessian at dT); Hv must not alias v; *vHv (host, may be NULL)
 * = <v, Hv>.  STML_EINVAL when u_coarsen is 0. */
stml_status stml_eval_ugrid(stml_ctx* ctx, int level, const int* frames, int nK, const float* w,
                            double* out, float* g, float* dT, float* Minv);
stml_status stml_hessvec_ugrid(stml_ctx* ctx, int level, const int* frames, int nK, const float* dT,
                               const float* v, float* Hv, double* vHv);

/* Affine-linear variant (params.transform = 1; Sec. 4 transformations, Sec. 2
 * L-BFGS).  Frame k's displacement is u_k(x) = W_k (x - c) / rho + b_k with x
 * a cell centre in finest-level pixels, c the centre of the finest grid
 * (extent / 2 per axis), rho half of its largest extent; theta_k = (W_k row
 * by row, b_k): d (d + 1) doubles per frame, the same on every level.  The
 * objective is J of eq. (1) at these fields (the parameters' gradient is the
 * projection of the field gradient).  L-BFGS: two-loop recursion with
 * H0 = (s^T y / y^T y) I of the newest pair, lbfgs_m pairs (pairs with
 * s^T y <= 1e-12 |s||y| dropped), first step -g scaled to move no parameter
 * by more than one pixel, Armijo back-tracking, the Gauss-Newton stopping
 * tests in parameter space, at most max_lbfgs iterations.  Multilevel:
 * stml_register runs STML / SpML over theta (linear predictor on the
 * coarsest level, eq. (2) per parameter on finer ones, eq. (3)); afterwards
 * every level's fields (stml_get_field) are the affine fields of the result.
 * The step API (stml_predict / stml_correct) serves transform 0 only. */

/* J, D, S, P (out[0..3]) at the affine fields of theta (host, nK x d(d+1))
 * for the frames of K on `level`, and dJ/dtheta (host, same shape) when grad
 * is not NULL.  Synchronises the stream. */
stml_status stml_eval_affine(stml_ctx* ctx, int level, const int* frames, int nK, const double* theta,
                             double* out, double* grad);
/* The affine fields u (device, nK x d x N) of theta (host) on `level`. */
stml_status stml_affine_field(stml_ctx* ctx, int level, const int* frames, int nK, const double* theta,
                              float* u);
/* GIR(K) over the affine parameters (L-BFGS) from theta_io (host, updated);
 * stats->gn_iters counts L-BFGS iterations, cg_iters is 0. */
stml_status stml_gir_affine(stml_ctx* ctx, int level, const int* frames, int nK, double* theta_io,
                            stml_stats* stats);
/* The parameters of all frames after an affine stml_register (host,
 * n x d(d+1) doubles; cap = capacity in doubles). */
stml_status stml_get_affine(const stml_ctx* ctx, double* theta, size_t cap);

/* Correlation coefficients rho_{k,k+1} of consecutive frames at `level`
 * (Sec. 4, Table 1); rho (host) receives n - 1 doubles. */
stml_status stml_corr_coeff(stml_ctx* ctx, int level, double* rho);

/* ------------------------------------ context-free operators (device) */

/* 2^d block mean of `planes` images of fine_shape into coarse (Sec. 3). */
stml_status stml_restrict(const float* fine, float* coarse, int planes, int dim,
                          const int* fine_shape, void* cuda_stream);

/* Cell-centred multilinear prolongation P (clamp at the border) of `planes`
 * scalar planes of coarse_shape to 2 * coarse_shape. */
stml_status stml_prolong(const float* coarse, float* fine, int planes, int dim,
                         const int* coarse_shape, void* cuda_stream);

/* Transpose P^T of stml_prolong, as a gather with a fixed summation order. */
stml_status stml_prolong_adjoint(const float* fine, float* coarse, int planes, int dim,
                                 const int* coarse_shape, void* cuda_stream);

/* The interpolation P_s of the coarse displacement grid (params.u_coarsen):
 * `planes` planes of fine_shape / 2^s (s in 1..4, every axis of fine_shape a
 * multiple of 2^s) to fine_shape; per axis, fine cell j takes
 * (1 - f) w[clamp(i0)] + f w[clamp(i0 + 1)] with i0 + f = (j + 1/2) / 2^s - 1/2.
 * stml_ugrid_adjoint is its transpose P_s^T, a gather over the 2^(s+1) fine
 * cells per axis of every coarse cell in a fixed order (no atomics).  Device
 * arrays; STML_EINVAL for bad shapes. */
stml_status stml_ugrid_prolong(const float* w, float* u, int planes, int dim, const int* fine_shape, int s,
                               void* cuda_stream);
stml_status stml_ugrid_adjoint(const float* u, float* w, int planes, int dim, const int* fine_shape, int s,
                               void* cuda_stream);

/* Linear temporal predictor (Sec. 3, coarsest level): for every target frame
 * t in `targets` (host, nT frames) z[t] = yK[t] if t is in K, else the linear
 * interpolation of its neighbours left(t), right(t) in K.  yK holds nK planes
 * of plane_elems floats in the order of K, z holds nT planes in the order of
 * targets (device). */
stml_status stml_predict_linear(const float* yK, const int* K, int nK, float* z,
                                const int* targets, int nT, size_t plane_elems,
                                void* cuda_stream);

/* Least-squares temporal predictor, eq. (2), for n_comp independent
 * (pixel, component) series: eta (device, nK * n_comp floats, frames of K in
 * order), omega and zeta (device, n * n_comp floats, frame-major).  Solved by
 * Thomas' algorithm with one factorisation of D_K + beta L for all series. */
stml_status stml_predict_ls(const float* eta, const int* K, int nK, const float* omega,
                            float* zeta, int n, double beta, size_t n_comp,
                            void* cuda_stream);

/* ------------------------------------------ batched persistent solver */

/* A batch of contexts solved together (batched serving of many sequences of
 * uneven frame counts and sizes; the paper has no counterpart).  For every
 * (spatial level, temporal level) stage of the multilevel sweep, the
 * predictors, gathers and the stopping rule eq. (3) run per context on its own
 * stream, and the GIRs of all contexts run in ONE persistent cooperative
 * kernel: each sequence's Gauss-Newton / PCG / Armijo loop is a state machine
 * on the device, every step of the kernel splits the grid into contiguous CTA
 * ranges (one per active sequence, sized by the bytes its current phase
 * moves) that stride over the sequence's (tile or frame-chunk) items, and the
 * first CTA of each range reduces its range's sums in a fixed order and takes
 * the sequence's decisions; the grid barriers are bounded (STML_ETIMEOUT).
 * Each stage's uploads, kernel and download replay a CUDA graph captured on
 * the stage's first use.  With params.autotune = 1 the first stage of every
 * level times four launch shapes (1 or 2 CTAs per SM, 4 or 16 lanes per
 * PCG tile row) and keeps the fastest for the batch.
 *
 * stml_batch_create: ctxs (host array of n_ctx distinct contexts of one
 * device, not sharing a predictor network) stay owned by the caller and must
 * outlive the batch.  stml_batch_register: every context must hold a built
 * pyramid; all need the same dimension, image storage, level counts and
 * solver parameters (alpha, alpha_t, lambda, tolerances, iteration limits),
 * transform 0, and at most 2 x SMs sequences (target_J may differ: each
 * sequence's last GIR stops at its own target); else
 * STML_EINVAL before any work.  status (host, n_ctx entries, may be NULL)
 * receives each context's result; the return value is STML_OK or the first
 * failure.  Decisions are those of stml_register (same tests on the same
 * kinds of totals); results agree with it to rounding.  Per-GIR statistics:
 * stml_last_stats on each context.  stml_batch_report writes a JSON array
 * (per stage: level, tlevel, sequences, kernel steps, ms, launch shape; the
 * autotuner's trials) to buf (host, cap bytes, NUL-terminated; *needed gets
 * the full length plus one).  Errors of batch calls: stml_batch_last_error. */
typedef struct stml_batch stml_batch;
stml_status stml_batch_create(stml_ctx* const* ctxs, int n_ctx, stml_batch** out);
stml_status stml_batch_register(stml_batch* batch, stml_mode mode, stml_status* status);
stml_status stml_batch_report(const stml_batch* batch, char* buf, size_t cap, size_t* needed);
const char* stml_batch_last_error(const stml_batch* batch);
void stml_batch_destroy(stml_batch* batch);

/* Failure-detection self-check of the batched solver's bounded grid
 * barrier: one CTA enters a barrier that expects two CTAs, so nothing
 * completes it; *expired (host) = 1 when the wait gave up after its bound
 * (about 2 s) and reported it -- the behaviour a stalled batched solve shows
 * as STML_ETIMEOUT.  Synchronises `cuda_stream`. */
stml_status stml_check_batch_barrier(void* cuda_stream, int* expired);

/* Statistics of every GIR of the context's last registration (stml_register
 * or stml_batch_register), in order: stats (host, cap entries, may be NULL),
 * *n_written (may be NULL) the number of GIRs. */
stml_status stml_last_stats(const stml_ctx* ctx, stml_stats* stats, int cap, int* n_written);

/* ----------------------------------------------- allocation-free variant */

/* Gauss-Newton Hessian product (as stml_hessvec) for callers that cannot
 * allocate device memory: code running inside a framework that owns all
 * device memory through its own pool, or code that may only touch the buffers
 * it is handed.  The paper has no counterpart; this is a library service.
 * No context is needed and nothing is allocated: dT, v and Hv (device,
 * nK * dim * N floats of the level grid `shape` with cell width h) are the
 * caller's; frames (host, nK increasing numbers) only set the temporal
 * weights; p supplies alpha, alpha_t and lambda; *vHv (host, may be NULL)
 * receives <v, Hv>.  All scratch comes from one static 24 MiB device array per
 * GPU that loads the library (held until the process exits); a problem that
 * needs more returns STML_EINVAL.  The first call on a device looks up that
 * array's device address (make that first call before any stream capture);
 * the address is kept per CUDA context, so after cudaDeviceReset the next
 * call looks it up again.  Frame numbers and weights reach the array as
 * kernel arguments (no host-to-device copy); with vHv != NULL the call copies
 * <v, Hv> to the host and synchronises `cuda_stream`.  Calls share the array,
 * so calls that overlap on the GPU race; run them on one stream.  Errors are
 * reported through stml_last_error(NULL). */
stml_status stml_hessvec_noalloc(const float* dT, const float* v, float* Hv, int dim,
                                 const int* shape, double h, const int* frames, int nK,
                                 const stml_params* p, double* vHv, void* cuda_stream);

/* ------------------------------------------------------------ profiling */

/* CUDA-event timing of solver launches on the context's stream, grouped by
 * kernel class and level: 1 times every launch, 2 only the Gauss-Newton
 * Hessian-product launches, 0 none.  Resets the counters. */
stml_status stml_profile_enable(stml_ctx* ctx, int enable);

/* Reads the counters: launches, summed device milliseconds, summed
 * algorithmic bytes (read v, read grad T, write Hv: 12 d bytes per
 * pixel-frame) and summed pixel-frames.  Synchronises the stream. */
stml_status stml_profile_read(stml_ctx* ctx, long long* launches, double* ms, double* bytes,
                              double* pixel_frames);

/* Per kernel class and level: launches, summed device milliseconds, summed
 * algorithmic bytes and pixel-frames of every launch since
 * stml_profile_enable(ctx, 1), as a JSON array written to buf (host, cap
 * bytes, NUL-terminated, truncated if short); *needed (may be NULL) receives
 * the full length plus one.  Synchronises the stream. */
stml_status stml_profile_report(stml_ctx* ctx, char* buf, size_t cap, size_t* needed);

/* The choices params.autotune made so far in this context, as JSON text:
 * [{"what": "objective_shape", "level": l, "frames": n, "variant": v,
 *   "vec": w, "splits": s}, {"what": "pcg_path", "level": l, "frames": n,
 * "cooperative": 0|1}, ...] (variant 0 objective, 1 Armijo trial, 2 trial
 * with <g, d>).  Same buffer protocol as stml_profile_report. */
stml_status stml_tuning_report(const stml_ctx* ctx, char* buf, size_t cap, size_t* needed);

/* Number of this library's kernel launches since the context was created. */
long long stml_launch_count(const stml_ctx* ctx);

/* Latency floor of one CG step of the cooperative PCG solve (the Jacobi-PCG
 * inner iterations of the Gauss-Newton GIR, Sec. 2, run in one launch on
 * small levels): times `iters` iterations of the solve's synchronisation
 * alone -- per iteration two rounds of CTA partial sums, a grid-wide barrier
 * and the fixed-order total of the partials in every CTA, with no vector
 * work -- in one cooperative launch of `blocks` CTAs of 256 threads (at most
 * two per SM, as the solve), after one untimed launch, and writes the
 * microseconds per iteration to *us_per_iter (host).  A measurement utility;
 * the paper has no counterpart.  No context is needed; the call allocates
 * and frees its own small buffers, runs on a stream of its own on the current
 * device and synchronises it.  blocks beyond what can be resident at once,
 * blocks or iters below 1, or a NULL pointer return STML_EINVAL; errors are
 * reported through stml_last_error(NULL). */
stml_status stml_coop_sync_floor(int blocks, int iters, double* us_per_iter);

#ifdef __cplusplus
}
#endif

#endif /* STML_H */
