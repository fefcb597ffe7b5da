// Host runtime of the STML library: context and memory plan, the
// Gauss-Newton/PCG/Armijo registration of a frame subset (the GIR of Sec. 2),
// the spatio-temporal predictor-corrector sweep (Sec. 3, eqs. 2-3), the
// spatial-only multilevel baseline and the C ABI of include/stml.h.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <array>
#include <functional>
#include <initializer_list>
#include <map>
#include <string>
#include <thread>
#include <atomic>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/stml.h"
#include "../../include/stml_net.h"
#include "kernels.h"
#include "net.h"

using namespace stml;

namespace {

thread_local std::string g_free_error;   // error text of the context-free calls

// NVTX range for profilers (no cost without one attached): spatial level,
// temporal level / GIR, Gauss-Newton iteration, learned proposals.
struct Range {
    template <typename... A>
    explicit Range(const char* fmt, A... a) {
        char buf[96];
        std::snprintf(buf, sizeof(buf), fmt, a...);
        nvtxRangePushA(buf);
    }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

struct LevelBuf {
    Geom g{};
    int shape3[3] = {1, 1, 1};
    void* img = nullptr;     // n * N values of the context's image storage type
    float* y = nullptr;      // n * d * N  (y_{l,all})
};

}  // namespace

void stml::set_context_free_error(const std::string& msg) { g_free_error = msg; }

struct stml_ctx {
    stml_params p{};
    cudaStream_t stream = nullptr;
    int device = 0;
    int n = 0, d = 0;
    int img_type = ST_F32;               // storage of the image pyramid and of the solver's grad T
    int shape[3] = {1, 1, 1};            // finest level (z, y, x)
    std::vector<LevelBuf> lv;
    std::vector<std::vector<int>> sets;  // K_0 .. K_T
    bool loaded = false, built = false;

    // workspace, sized for the finest level and all frames
    float *w_u = nullptr, *w_g = nullptr, *w_dT = nullptr, *w_x = nullptr, *w_r = nullptr,
          *w_p = nullptr, *w_q = nullptr, *w_ut = nullptr;
    float *w_abar = nullptr, *w_ubar = nullptr;    // per-pixel frame means of the last objective pass
    float *w_m1 = nullptr, *w_m2 = nullptr;        // per-pixel frame sums of a Hessian-product field / of z
    float *w_p2 = nullptr, *w_cz = nullptr;        // second PCG direction buffer, PCG z = M^-1 r
    float *w_sp0 = nullptr, *w_sp1 = nullptr;      // frame sums of the PCG direction ((1 + d) N each)
    float *w_z = nullptr, *w_z2 = nullptr;     // predictor state z_{l,q,all}
    double* partials = nullptr;
    size_t partials_cap = 0;                   // in doubles
    DevScalars* S = nullptr;                   // device scalars
    DevScalars* Sh = nullptr;                  // pinned host mirror
    int* d_frames = nullptr;
    float* d_wnext = nullptr;
    int* d_idx = nullptr;
    float* d_lsf = nullptr;                    // cp | inv_den | sub
    int* d_kidx = nullptr;
    LinTap* d_taps = nullptr;
    double* d_rho = nullptr;

    // STML sweep state
    int cur_level = -1, last_q = -1;
    double dhat_prev = 0.0;
    bool level_done = false;

    // profiling: CUDA events around every launch of the solver, per kernel
    // class and level (key = class * 64 + level), with algorithmic bytes
    bool prof = false;
    bool prof_hess_only = false;
    struct ProfEvent {
        int key;
        cudaEvent_t a, b;
    };
    std::vector<ProfEvent> ev;
    size_t ev_used = 0;
    std::map<int, std::array<double, 3>> pacc;   // key -> launches, bytes, pixel-frames
    // autotuned choices (params.autotune): objective-pass launch shape per
    // (level, nK, variant) and cooperative (1) or streaming (0) PCG per (level, nK)
    std::map<std::array<int, 3>, ObjShapeChoice> obj_tuned;
    std::map<std::array<int, 2>, int> coop_tuned;

    // affine variant (params.transform = 1): parameters of all frames (host),
    // device and pinned staging buffers for one evaluation
    std::vector<double> theta;
    float* d_theta = nullptr;
    double *d_gth = nullptr, *d_aff_part = nullptr;
    float* h_theta = nullptr;
    double* h_gth = nullptr;
    int aff_cap = 0;                  // frames the affine buffers hold
    // one evaluation of the affine objective (upload, field, objective,
    // gradient, projection, download) as a CUDA graph per (level, nK, grad);
    // captured on a private stream, launched on the context's stream
    cudaStream_t cap_stream = nullptr;
    std::map<std::array<int, 3>, cudaGraphExec_t> aff_graphs;
    // normalised-correlation distance: frame means, Gram matrix, D_NC with
    // the row sums and the Gram partials, the K x K gradient matrix, and a
    // pinned slot for D_NC
    float *d_mu = nullptr, *d_Q = nullptr;
    double *d_G = nullptr, *d_gpart = nullptr, *h_G = nullptr;

    // learned temporal predictor (stml_set_predictor_net) and its last decisions
    ::stml_net* net = nullptr;
    int pred_learned = -1;
    double J0_classic = 0.0;

    // coarse displacement grid (params.u_coarsen > 0): vectors on the coarse
    // grid of the finest level for all frames (gradient, PCG x, r, z, p, q,
    // Jacobi inverse, accepted point) and the reduction scratch of its passes
    float *ug_g = nullptr, *ug_x = nullptr, *ug_r = nullptr, *ug_z = nullptr, *ug_p = nullptr, *ug_q = nullptr,
          *ug_m = nullptr, *ug_w = nullptr;
    double *ug_part = nullptr, *ug_out = nullptr, *ug_outh = nullptr;
    size_t ug_part_cap = 0;
    unsigned int* ug_tk = nullptr;
    UgCg *ug_cg = nullptr, *ug_cgh = nullptr;   // device state of the coarse-grid PCG solve, pinned host copy
    size_t ug_cap = 0;                           // floats each coarse-grid vector holds

    std::vector<stml_stats> last_stats;   // per GIR of the last registration
    std::string err;
};

namespace {

stml_status fail(stml_ctx* c, stml_status s, const std::string& msg) {
    if (c)
        c->err = msg;
    else
        g_free_error = msg;
    return s;
}

stml_status cuda_fail(stml_ctx* c, cudaError_t e, const char* what) {
    return fail(c, STML_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(ctx, call)                                              \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call); \
    } while (0)

#define TRY(call)                           \
    do {                                    \
        stml_status s_ = (call);            \
        if (s_ != STML_OK) return s_;       \
    } while (0)

template <class T>
cudaError_t dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void**)p, count * sizeof(T));
}

template <class T>
void dfree(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

bool valid_params(const stml_params* p, std::string& why) {
    if (!p) { why = "params is NULL"; return false; }
    if (p->n_levels < 1 || p->n_levels > 12) { why = "n_levels must be in 1..12"; return false; }
    if (p->n_tlevels < 1 || p->n_tlevels > 20) { why = "n_tlevels must be in 1..20"; return false; }
    if (!(p->alpha >= 0) || !(p->alpha_t >= 0) || !(p->lambda >= 0) || !(p->beta >= 0)) {
        why = "alpha, alpha_t, lambda and beta must be >= 0";
        return false;
    }
    if (p->max_gn < 0 || p->max_cg < 0 || p->max_ls < 1) { why = "iteration limits out of range"; return false; }
    if (!(p->tol_cg > 0) || !(p->armijo_c > 0 && p->armijo_c < 1)) { why = "tol_cg > 0 and 0 < armijo_c < 1"; return false; }
    if (p->pcg_cooperative != 0 && p->pcg_cooperative != 1) { why = "pcg_cooperative must be 0 or 1"; return false; }
    if (p->autotune != 0 && p->autotune != 1) { why = "autotune must be 0 or 1"; return false; }
    if (p->transform != 0 && p->transform != 1) { why = "transform must be 0 or 1"; return false; }
    if (p->distance != 0 && p->distance != 1) { why = "distance must be 0 or 1"; return false; }
    if (p->distance == 1 && p->transform != 1) { why = "distance 1 (normalised correlation) needs transform 1"; return false; }
    if (p->lbfgs_m < 1 || p->lbfgs_m > 64 || p->max_lbfgs < 0) {
        why = "lbfgs_m must be in 1..64 and max_lbfgs >= 0";
        return false;
    }
    if (!(p->target_J >= 0) || !(p->target_tol > 0 && p->target_tol < 1)) {
        why = "target_J must be >= 0 and 0 < target_tol < 1";
        return false;
    }
    if (p->image_dtype < STML_DTYPE_F32 || p->image_dtype > STML_DTYPE_BF16) {
        why = "image_dtype must be STML_DTYPE_F32, _F16 or _BF16";
        return false;
    }
    if (p->u_coarsen < 0 || p->u_coarsen > 4) { why = "u_coarsen must be in 0..4"; return false; }
    if (p->u_coarsen > 0 && (p->transform != 0 || p->image_dtype != STML_DTYPE_F32 || p->target_J != 0.0)) {
        why = "u_coarsen > 0 needs transform 0, image_dtype STML_DTYPE_F32 and target_J 0";
        return false;
    }
    return true;
}

Coef make_coef(const Geom& g, const stml_params& p, int nK) {
    Coef c;
    const double hd = g.hd;
    c.alpha_hd = (float)(p.alpha * hd);
    c.alphat_hd = (float)(p.alpha_t * hd);
    c.pen_g = (float)(2.0 * p.lambda * hd / nK);
    c.pen_h = (float)(2.0 * p.lambda * hd / ((double)nK * nK));
    c.lam_hd = (float)(p.lambda * hd);
    c.half_hd = (float)(0.5 * hd);
    c.hd = (float)hd;
    c.inv_h2 = (float)(1.0 / ((double)g.h * g.h));
    c.inv_nK = (float)(1.0 / nK);
    c.diag_D = (float)(hd * (1.0 - 1.0 / nK));
    return c;
}

// Grid the fields of a level live on: its image grid, or with u_coarsen =
// s > 0 that grid coarsened by 2^s per axis (cell width 2^s h).
Geom field_geom(const stml_ctx* c, int level) {
    const Geom& g = c->lv[level].g;
    const int s = c->p.u_coarsen;
    if (s == 0) return g;
    int sh3[3] = {g.d == 3 ? g.nz >> s : 1, g.ny >> s, g.nx >> s};
    return make_geom(sh3, g.d, g.h * (float)(1 << s));
}

void free_buffers(stml_ctx* c) {
    for (auto& L : c->lv) {
        dfree(L.img);
        dfree(L.y);
    }
    c->lv.clear();
    dfree(c->w_u); dfree(c->w_g); dfree(c->w_dT); dfree(c->w_x); dfree(c->w_r);
    dfree(c->w_p); dfree(c->w_q); dfree(c->w_ut); dfree(c->w_abar); dfree(c->w_ubar); dfree(c->w_m1);
    dfree(c->w_m2); dfree(c->w_z); dfree(c->w_z2); dfree(c->partials);
    dfree(c->w_p2); dfree(c->w_cz); dfree(c->w_sp0); dfree(c->w_sp1);
    for (float** fp : {&c->ug_g, &c->ug_x, &c->ug_r, &c->ug_z, &c->ug_p, &c->ug_q, &c->ug_m, &c->ug_w}) dfree(*fp);
    dfree(c->ug_part);
    dfree(c->ug_out);
    dfree(c->ug_tk);
    dfree(c->ug_cg);
    if (c->ug_outh) cudaFreeHost(c->ug_outh);
    if (c->ug_cgh) cudaFreeHost(c->ug_cgh);
    c->ug_outh = nullptr;
    c->ug_cgh = nullptr;
    c->ug_cap = 0;
    c->ug_part_cap = 0;
    dfree(c->d_frames); dfree(c->d_wnext); dfree(c->d_idx); dfree(c->d_lsf);
    dfree(c->d_kidx); dfree(c->d_taps); dfree(c->d_rho);
    dfree(c->d_theta); dfree(c->d_gth); dfree(c->d_aff_part);
    if (c->h_theta) cudaFreeHost(c->h_theta);
    if (c->h_gth) cudaFreeHost(c->h_gth);
    c->h_theta = nullptr;
    c->h_gth = nullptr;
    c->aff_cap = 0;
    for (auto& kv : c->aff_graphs) cudaGraphExecDestroy(kv.second);
    c->aff_graphs.clear();
    dfree(c->d_mu); dfree(c->d_Q); dfree(c->d_G); dfree(c->d_gpart);
    if (c->h_G) cudaFreeHost(c->h_G);
    c->h_G = nullptr;
    c->loaded = c->built = false;
}

std::vector<std::vector<int>> make_sets(int n, int Q) {
    // K_q takes every 2^(T-q)-th frame; the last frame always belongs to K_q.
    std::vector<std::vector<int>> sets;
    const int T = Q - 1;
    for (int q = 0; q < Q; ++q) {
        const long long stride = 1LL << (T - q);
        std::vector<int> K;
        for (long long k = 0; k < n; k += stride) K.push_back((int)k);
        if (K.back() != n - 1) K.push_back(n - 1);
        sets.push_back(K);
    }
    return sets;
}

stml_status check_frames(stml_ctx* c, const int* frames, int nK) {
    if (!frames || nK < 1 || nK > c->n) return fail(c, STML_EINVAL, "frame subset size out of range");
    for (int j = 0; j < nK; ++j) {
        if (frames[j] < 0 || frames[j] >= c->n) return fail(c, STML_EINVAL, "frame number out of range");
        if (j > 0 && frames[j] <= frames[j - 1]) return fail(c, STML_EINVAL, "frames must increase strictly");
    }
    return STML_OK;
}

bool al16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

stml_status check_aligned(stml_ctx* c, std::initializer_list<const void*> ptrs) {
    for (const void* p : ptrs)
        if (p && !al16(p)) return fail(c, STML_EINVAL, "device arrays must be 16-byte aligned");
    return STML_OK;
}

stml_status check_level(stml_ctx* c, int level) {
    if (!c->built) return fail(c, STML_ESTATE, "no pyramid: call stml_load_sequence and stml_build_pyramid");
    if (level < 0 || level >= (int)c->lv.size()) return fail(c, STML_EINVAL, "level out of range");
    return STML_OK;
}

// Uploads K and the temporal weights 1/(k_{j+1} - k_j)^2.
stml_status upload_frameset(stml_ctx* c, const std::vector<int>& K, FrameSet& fs) {
    std::vector<float> w(K.size(), 0.f);
    for (size_t j = 0; j + 1 < K.size(); ++j) {
        const double dk = (double)(K[j + 1] - K[j]);
        w[j] = (float)(1.0 / (dk * dk));
    }
    CK(c, cudaMemcpyAsync(c->d_frames, K.data(), K.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaMemcpyAsync(c->d_wnext, w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    fs.frames = c->d_frames;
    fs.w_next = c->d_wnext;
    fs.nK = (int)K.size();
    return STML_OK;
}

stml_status read_scalars(stml_ctx* c) {
    CK(c, cudaMemcpyAsync(c->Sh, c->S, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (c->Sh->err_flags & 1u) return fail(c, STML_ETIMEOUT, "a bounded device wait expired (bulk copy not completed)");
    return STML_OK;
}

enum ProfClass {
    PC_HESS = 0, PC_EVAL, PC_TRIAL, PC_PCG_INIT, PC_PCG_UPDATE, PC_PCG_P, PC_PCG_COOP,
    PC_PRED_LS, PC_PRED_LIN, PC_PROLONG, PC_GATHER, PC_RESTRICT, PC_PRED_NET, PC_AFFINE, PC_COUNT
};
const char* const kProfNames[PC_COUNT] = {
    "gn_hessian_product", "gradient_pass", "objective_pass", "pcg_init", "pcg_update",
    "pcg_direction", "pcg_solve_cooperative", "predict_ls_eq2", "predict_linear", "prolong", "gather_scatter",
    "restrict", "predict_learned", "affine_projection"};

// Starts an event pair (returns its index, or -1 when profiling is off).
long prof_begin(stml_ctx* c, int cls, int level) {
    if (!c->prof || (c->prof_hess_only && cls != PC_HESS)) return -1;
    if (c->ev_used == c->ev.size()) {
        stml_ctx::ProfEvent pe{0, nullptr, nullptr};
        if (cudaEventCreate(&pe.a) != cudaSuccess || cudaEventCreate(&pe.b) != cudaSuccess) return -1;
        c->ev.push_back(pe);
    }
    const long i = (long)c->ev_used++;
    c->ev[i].key = cls * 64 + level;
    cudaEventRecord(c->ev[i].a, c->stream);
    return i;
}

void prof_end(stml_ctx* c, long i, double bytes, double pixel_frames) {
    if (i < 0) return;
    cudaEventRecord(c->ev[i].b, c->stream);
    auto& acc = c->pacc[c->ev[i].key];
    acc[0] += 1;
    acc[1] += bytes;
    acc[2] += pixel_frames;
}

// Removes `n` launches of a class that returned at once (a stopped PCG solve,
// a line-search trial or step that was not needed) from the byte and launch
// counts; their (short) event time stays in the class total.
void prof_discount(stml_ctx* c, int cls, int level, double n, double bytes_each, double pf_each) {
    if (!c->prof || (c->prof_hess_only && cls != PC_HESS) || n <= 0) return;
    auto it = c->pacc.find(cls * 64 + level);
    if (it == c->pacc.end()) return;
    it->second[0] -= n;
    it->second[1] -= n * bytes_each;
    it->second[2] -= n * pf_each;
}

stml_status hessvec_launch(stml_ctx* c, int level, const Geom& g, const FrameSet& fs, const Coef& cf,
                           const float* dT, const float* v, float* Hv, DevScalars* pcg) {
    HessWork hw{c->w_m1, c->w_m2, c->partials, c->partials_cap};
    const long pe = prof_begin(c, PC_HESS, level);
    CK(c, launch_hessvec(g, fs, cf, dT, v, Hv, hw, &c->S->ticket[1], c->S->dots + 4, pcg, c->stream));
    const double pf = (double)fs.nK * (double)g.N;
    prof_end(c, pe, pf * 12.0 * g.d, pf);
    return STML_OK;
}

// ------------------------------------------------------------------ autotuning
// Launch shape of the objective pass for (level, nK, variant: 0 plain, 1
// trial, 2 trial with <g, d>): nullptr (the built-in choice) unless
// params.autotune.  The first call of a key times every candidate shape on
// these very arguments (one warm-up and two timed launches each, CUDA events
// on the context's stream) and keeps the fastest for the context's lifetime,
// so results stay reproducible within a context.
const ObjShapeChoice* obj_choice(stml_ctx* c, int level, const Geom& g, const FrameSet& fs, const Coef& cf,
                                 const Stored& T, const float* u, const float* du, float t, const float* gdot,
                                 int variant) {
    if (!c->p.autotune) return nullptr;
    const std::array<int, 3> key{level, fs.nK, variant};
    auto it = c->obj_tuned.find(key);
    if (it != c->obj_tuned.end()) return &it->second;
    ObjShapeChoice cand[16];
    const int nc = obj_shape_candidates(g, fs.nK, cand, 16);
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return nullptr;
    float best = 1e30f;
    ObjShapeChoice pick{0, 0};
    for (int i = 0; i < nc; ++i) {
        // scratch outputs: the frame means and totals of queued launches stay
        // untouched (w_m1 / w_m2 are rewritten by every PCG start)
        auto go = [&]() {
            return launch_objective(T, g, fs, cf, u, du, t, gdot, c->w_m1, c->w_m2, c->partials, c->partials_cap,
                                    &c->S->ticket[0], c->S->dots, c->stream, nullptr, &cand[i]);
        };
        if (go() != cudaSuccess) {   // a shape these arrays do not allow
            cudaGetLastError();
            continue;
        }
        cudaEventRecord(a, c->stream);
        const bool ok = go() == cudaSuccess && go() == cudaSuccess;
        cudaEventRecord(b, c->stream);
        float ms = 0.f;
        if (!ok || cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (ms < best) {
            best = ms;
            pick = cand[i];
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (pick.vec == 0) return nullptr;
    return &(c->obj_tuned[key] = pick);
}

// ------------------------------------------------------------------ GIR
// Gauss-Newton on the frames K of `level`, from and into u (nK * d * N floats).
// With target > 0 the GIR stops as soon as an accepted step reaches
// J <= target, after shortening that step (Illinois regula falsi on its
// length) so that J lands within params.target_tol * target of the target; a
// start with J0 <= target takes no step.
stml_status run_gir_ugrid(stml_ctx* c, int level, const std::vector<int>& K, float* w_io, stml_stats* st);

stml_status run_gir(stml_ctx* c, int level, const std::vector<int>& K, float* u_io, stml_stats* st,
                    double target = 0.0) {
    if (c->p.u_coarsen > 0) return run_gir_ugrid(c, level, K, u_io, st);
    Range rg("GIR level %d |K| %d", level, (int)K.size());
    const auto t_start = std::chrono::steady_clock::now();
    LevelBuf& L = c->lv[level];
    const Geom& g = L.g;
    const int nK = (int)K.size();
    const size_t M = (size_t)nK * g.d * g.N;
    const stml_params& p = c->p;
    FrameSet fs;
    TRY(upload_frameset(c, K, fs));
    const Coef cf = make_coef(g, p, nK);
    float* u = u_io;
    float* ut = c->w_ut;
    DevScalars* S = c->S;
    const PcgArgs pa{(float)p.tol_cg, p.max_cg};

    stml_stats s{};
    s.level = level;
    s.n_frames = nK;
    s.status = STML_OK;

    const double pfK = (double)nK * (double)g.N;
    // Algorithmic bytes per pixel-frame of each pass (every array read or
    // written once; images and grad T in their storage type of bS bytes).
    const double bS = (double)store_bytes(c->img_type), d = g.d;
    const double B_obj = bS + 4.0 * d;                        // T, u
    const double B_trial0 = bS + 16.0 * d, B_trial = bS + 8.0 * d;   // T, u, d (, g and d again)
    const double B_grad0 = bS + (8.0 + bS) * d;               // T, u; g, grad T
    const double B_grad = bS + (16.0 + bS) * d;               // T, u, d; g, grad T, u + t d
    const double B_apply = (8.0 + bS) * d;                    // p, grad T; Hp
    const double B_update = (24.0 + bS) * d;                  // x, p, r, q, grad T; x, r
    const double B_dir = (12.0 + bS) * d;                     // r, grad T, p; p
    const double B_init = (16.0 + bS) * d;                    // g, grad T; r, p, x
    // objective + gradient at u (start of the GIR)
    auto eval_full = [&]() -> stml_status {
        long pe = prof_begin(c, PC_TRIAL, level);
        const ObjShapeChoice* sh0 = obj_choice(c, level, g, fs, cf, Stored{L.img, c->img_type}, u, nullptr, 0.f,
                                               nullptr, 0);
        CK(c, launch_objective(Stored{L.img, c->img_type}, g, fs, cf, u, nullptr, 0.f, nullptr, c->w_abar, c->w_ubar,
                               c->partials, c->partials_cap, &S->ticket[0], S->red, c->stream, nullptr, sh0));
        prof_end(c, pe, pfK * B_obj, pfK);
        pe = prof_begin(c, PC_EVAL, level);
        CK(c, launch_gradient(Stored{L.img, c->img_type}, g, fs, cf, u, nullptr, 0.f, c->w_abar, c->w_ubar, c->w_g,
                              c->w_dT, c->img_type, nullptr, c->partials, c->partials_cap, &S->ticket[4], S->red,
                              c->stream));
        prof_end(c, pe, pfK * B_grad0, pfK);
        return read_scalars(c);
    };

    TRY(eval_full());
    const double J0 = c->Sh->red[0];
    double J = J0, D = c->Sh->red[1], Sv = c->Sh->red[2], Pv = c->Sh->red[3];
    double gnorm2 = c->Sh->red[4], unorm2 = c->Sh->red[5];
    s.J0 = J0;
    double J_old = 0.0, step_norm = 0.0;
    int it = 0;
    int predict_cg = 8;        // CG steps launched in the first chunk of a solve
    int launched = 0;
    long pe = -1;

    // Stopping tests of the Gauss-Newton loop at the current iterate.
    auto should_stop = [&]() -> bool {
        if (!std::isfinite(J) || !std::isfinite(gnorm2)) {
            s.status = STML_ENONFINITE;
            return true;
        }
        const double gnorm = std::sqrt(gnorm2);
        if (it > 0) {
            const bool c1 = std::fabs(J_old - J) <= p.tol_J * (1.0 + std::fabs(J0));
            const bool c2 = step_norm <= p.tol_Y * (1.0 + std::sqrt(unorm2));
            const bool c3 = gnorm <= p.tol_G * (1.0 + std::fabs(J0));
            if (c1 && c2 && c3) return true;
        }
        return gnorm <= p.g_abs * (1.0 + std::fabs(J0)) || it >= p.max_gn;
    };
    // PCG vectors of this level: the direction sums live at [0, N) (mean of
    // grad T . p) and [N, (1 + d) N) (sum of p) of w_sp0 / w_sp1
    const Stored dTs{c->w_dT, c->img_type};   // the solver's grad T, in the image storage type
    const PcgBufs pb{c->w_x, c->w_r, c->w_cz, c->w_q, {c->w_p, c->w_p2}, c->w_m1, c->w_m2,
                     {c->w_sp0, c->w_sp1}, {c->w_sp0 + g.N, c->w_sp1 + g.N}};
    // PCG iterations (Hessian product, update, direction), `n` of them, queued.
    auto launch_cg = [&](int n) -> stml_status {
        for (int i = 0; i < n; ++i) {
            pe = prof_begin(c, PC_HESS, level);
            CK(c, launch_pcg_apply(g, fs, cf, dTs, pb, c->partials, c->partials_cap, S, c->stream));
            prof_end(c, pe, pfK * B_apply, pfK);
            pe = prof_begin(c, PC_PCG_UPDATE, level);
            CK(c, launch_pcg_update(g, fs, cf, dTs, pb, c->partials, c->partials_cap, S, pa, c->stream));
            prof_end(c, pe, pfK * B_update, pfK);
            pe = prof_begin(c, PC_PCG_P, level);
            CK(c, launch_pcg_direction(g, fs, cf, dTs, pb, S, c->stream));
            prof_end(c, pe, pfK * B_dir, pfK);
        }
        launched += n;
        return STML_OK;
    };
    // Start of a PCG solve for H d = -g plus its first chunk of steps (small
    // levels: the whole solve in one cooperative launch).
    // Launches of a streaming solve that returned at once (after the solve
    // stopped, or because its gated start did not run) leave the profile.
    auto discount_cg = [&](int queued, int ran_apply, int ran_update, int ran_dir, bool init_ran) {
        prof_discount(c, PC_HESS, level, queued - ran_apply, pfK * B_apply, pfK);
        prof_discount(c, PC_PCG_UPDATE, level, queued - ran_update, pfK * B_update, pfK);
        prof_discount(c, PC_PCG_P, level, queued - ran_dir, pfK * B_dir, pfK);
        if (!init_ran) prof_discount(c, PC_PCG_INIT, level, 1, pfK * B_init, pfK);
    };
    // With gate != nullptr the solve starts only if the device accepted a step.
    bool coop = p.pcg_cooperative && pcg_coop_preferred(g, nK);
    auto start_cg = [&](const int* gate = nullptr) -> stml_status {
        if (coop) {
            pe = prof_begin(c, PC_PCG_COOP, level);
            CK(c, launch_pcg_coop(g, fs, cf, c->w_g, dTs, pb, c->partials, c->partials_cap, S, pa, c->stream,
                                  gate));
            prof_end(c, pe, 0.0, pfK);
            launched = p.max_cg;
            return STML_OK;
        }
        pe = prof_begin(c, PC_PCG_INIT, level);
        CK(c, launch_pcg_init(g, fs, cf, c->w_g, dTs, pb, c->partials, c->partials_cap, S, pa, c->stream,
                              gate));
        prof_end(c, pe, pfK * B_init, pfK);
        launched = 0;
        return launch_cg(std::min(p.max_cg, std::max(2, predict_cg)));
    };

    // params.autotune: time a cooperative and a streaming solve of the first
    // system of this (level, nK) and keep the faster path for the context
    auto tune_coop = [&]() -> stml_status {
        const std::array<int, 2> key{level, nK};
        const auto it = c->coop_tuned.find(key);
        if (it != c->coop_tuned.end()) {
            coop = it->second != 0;
            return STML_OK;
        }
        cudaEvent_t a = nullptr, b = nullptr;
        CK(c, cudaEventCreate(&a));
        CK(c, cudaEventCreate(&b));
        float t_coop = 1e30f, t_str = 1e30f;
        CK(c, cudaEventRecord(a, c->stream));
        CK(c, launch_pcg_coop(g, fs, cf, c->w_g, dTs, pb, c->partials, c->partials_cap, S, pa, c->stream));
        CK(c, cudaEventRecord(b, c->stream));
        CK(c, cudaEventSynchronize(b));
        CK(c, cudaEventElapsedTime(&t_coop, a, b));
        CK(c, cudaEventRecord(a, c->stream));
        CK(c, launch_pcg_init(g, fs, cf, c->w_g, dTs, pb, c->partials, c->partials_cap, S, pa, c->stream));
        int done = 0;
        for (int chunk = std::min(p.max_cg, std::max(2, predict_cg)); done < p.max_cg;
             chunk = std::min(4, p.max_cg - done)) {
            for (int i = 0; i < chunk; ++i) {
                CK(c, launch_pcg_apply(g, fs, cf, dTs, pb, c->partials, c->partials_cap, S, c->stream));
                CK(c, launch_pcg_update(g, fs, cf, dTs, pb, c->partials, c->partials_cap, S, pa, c->stream));
                CK(c, launch_pcg_direction(g, fs, cf, dTs, pb, S, c->stream));
            }
            done += chunk;
            TRY(read_scalars(c));
            if (!c->Sh->cg_active) break;
        }
        CK(c, cudaEventRecord(b, c->stream));
        CK(c, cudaEventSynchronize(b));
        CK(c, cudaEventElapsedTime(&t_str, a, b));
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        coop = t_coop <= t_str;
        c->coop_tuned[key] = coop ? 1 : 0;
        return STML_OK;
    };

    const bool targeted = target > 0.0;
    bool started = false;     // a PCG solve (with its first chunk) is already queued and read
    if (!(targeted && J0 <= target) && !should_stop()) {
        if (p.autotune && p.pcg_cooperative && (long long)g.N * nK <= (1LL << 23)) TRY(tune_coop());
        TRY(start_cg());
        TRY(read_scalars(c));
        started = true;
    }
    while (started) {
        Range rit("Gauss-Newton iteration %d", it);
        // --- finish the PCG solve: all coefficients stay on the device; chunks of
        // launches whose kernels return at once when the device cleared cg_active
        while (c->Sh->cg_active && launched < p.max_cg) {
            TRY(launch_cg(std::min(4, p.max_cg - launched)));
            TRY(read_scalars(c));
        }
        s.cg_iters += c->Sh->cg_iter;
        predict_cg = c->Sh->cg_iter;
        if (!coop) {   // launches of this solve that did work
            const int n_it = c->Sh->cg_iter, fl = c->Sh->cg_flag;
            const bool brk = fl == CG_BREAKDOWN;
            const int ran_apply = fl == CG_ZERO ? 0 : n_it + (brk ? 1 : 0);
            const int ran_dir = brk ? n_it : std::max(n_it - 1, 0);
            discount_cg(launched, ran_apply, n_it, ran_dir, true);
        }
        if (c->Sh->cg_flag == CG_BREAKDOWN && c->Sh->cg_iter == 0)   // preconditioned gradient step p_0
            CK(c, cudaMemcpyAsync(c->w_x, c->w_p, M * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));

        // --- Armijo back-tracking, decided on the device.  Trials t = 1 and
        // t = 1/2 are queued together (the second returns at once if the first
        // is accepted), then the gradient pass at the accepted point and the
        // next PCG start, both gated on acceptance: one host wait per
        // Gauss-Newton step unless both trials fail.
        bool accepted = false, descent = true;
        int ls_next = 0;              // next trial to queue
        auto queue_trial = [&](int k) -> stml_status {
            const double t = std::ldexp(1.0, -k);
            const LineSearchArgs la{S, k, J, p.armijo_c};
            const ObjShapeChoice* sh = obj_choice(c, level, g, fs, cf, Stored{L.img, c->img_type}, u, c->w_x,
                                                  (float)t, k == 0 ? c->w_g : nullptr, k == 0 ? 2 : 1);
            pe = prof_begin(c, PC_TRIAL, level);
            CK(c, launch_objective(Stored{L.img, c->img_type}, g, fs, cf, u, c->w_x, (float)t, k == 0 ? c->w_g : nullptr,
                                   c->w_abar, c->w_ubar, c->partials, c->partials_cap, &S->ticket[0], S->trial,
                                   c->stream, &la, sh));
            prof_end(c, pe, pfK * (k == 0 ? B_trial0 : B_trial), pfK);
            return STML_OK;
        };
        // gradient pass at the accepted point (writes u + t d to ut, g, grad T)
        // and the speculative start of the next solve
        // (with a target the direction must survive the step: no speculative start)
        const bool next_solve = it + 1 < p.max_gn && !targeted;
        auto drop_accept = [&]() {   // a queued gated step and start that did not run
            prof_discount(c, PC_EVAL, level, 1, pfK * B_grad, pfK);
            if (next_solve && !coop) discount_cg(launched, 0, 0, 0, false);
            if (next_solve && coop) prof_discount(c, PC_PCG_COOP, level, 1, 0.0, pfK);
        };
        auto queue_accept = [&]() -> stml_status {
            pe = prof_begin(c, PC_EVAL, level);
            CK(c, launch_gradient(Stored{L.img, c->img_type}, g, fs, cf, u, c->w_x, 1.0f, c->w_abar, c->w_ubar,
                                  c->w_g, c->w_dT, c->img_type, ut, c->partials, c->partials_cap, &S->ticket[4],
                                  S->red, c->stream, S));
            prof_end(c, pe, pfK * B_grad, pfK);
            if (next_solve) TRY(start_cg(&S->ls_accepted));
            return STML_OK;
        };
        for (; ls_next < std::min(2, p.max_ls); ++ls_next) TRY(queue_trial(ls_next));
        TRY(queue_accept());
        TRY(read_scalars(c));
        while (!c->Sh->ls_nodescent && !c->Sh->ls_accepted && ls_next < p.max_ls) {
            drop_accept();
            TRY(queue_trial(ls_next++));
            TRY(queue_accept());
            TRY(read_scalars(c));
        }
        if (!c->Sh->ls_accepted) drop_accept();
        // queued trials that returned at once
        prof_discount(c, PC_TRIAL, level, ls_next - c->Sh->ls_trials, pfK * B_trial, pfK);
        s.ls_trials += c->Sh->ls_trials;
        descent = !c->Sh->ls_nodescent;
        accepted = c->Sh->ls_accepted != 0;
        if (!descent) {
            s.status = STML_EBREAKDOWN;
            break;
        }
        if (!accepted) {
            s.status = STML_ELINESEARCH;
            break;
        }
        std::swap(u, ut);
        step_norm = (double)c->Sh->ls_t * std::sqrt(c->Sh->ls_dnorm2);
        J_old = J;
        J = c->Sh->trial[0];
        D = c->Sh->trial[1];
        Sv = c->Sh->trial[2];
        Pv = c->Sh->trial[3];
        ++it;
        gnorm2 = c->Sh->red[4];
        unorm2 = c->Sh->red[5];
        if (targeted && J <= target) {
            // land on the target between the previous iterate (now in ut) and
            // the accepted point: J(ut + s x) for s in (0, t]
            auto phi = [&](double sv, double* out4) -> stml_status {
                const ObjShapeChoice* sh = obj_choice(c, level, g, fs, cf, Stored{L.img, c->img_type}, ut, c->w_x,
                                                      (float)sv, nullptr, 1);
                pe = prof_begin(c, PC_TRIAL, level);
                CK(c, launch_objective(Stored{L.img, c->img_type}, g, fs, cf, ut, c->w_x, (float)sv, nullptr,
                                       c->w_abar, c->w_ubar, c->partials, c->partials_cap, &S->ticket[0], S->trial,
                                       c->stream, nullptr, sh));
                prof_end(c, pe, pfK * B_trial, pfK);
                TRY(read_scalars(c));
                for (int i = 0; i < 4; ++i) out4[i] = c->Sh->trial[i];
                return STML_OK;
            };
            const double tol = p.target_tol * target;
            double a = 0.0, fa = J_old - target, b = c->Sh->ls_t, fb = J - target;
            double best_t = b, best_f = std::fabs(fb), cur[4] = {J, D, Sv, Pv}, best4[4] = {J, D, Sv, Pv};
            int side = 0;
            for (int i = 0; i < 40 && best_f > tol; ++i) {
                const double tv = (a * fb - b * fa) / (fb - fa);
                TRY(phi(tv, cur));
                const double ft = cur[0] - target;
                if (std::fabs(ft) < best_f) {
                    best_f = std::fabs(ft);
                    best_t = tv;
                    for (int k = 0; k < 4; ++k) best4[k] = cur[k];
                }
                if (ft > 0.0) {
                    a = tv;
                    fa = ft;
                    if (side == 1) fb *= 0.5;
                    side = 1;
                } else {
                    b = tv;
                    fb = ft;
                    if (side == -1) fa *= 0.5;
                    side = -1;
                }
            }
            if (best_t != c->Sh->ls_t) {
                // the landed point: objective (abar, ubar) then gradient pass writing u = ut + s x
                double chk[4];
                if ((double)(float)best_t != (double)(float)c->Sh->ls_t) {
                    TRY(phi(best_t, chk));
                    pe = prof_begin(c, PC_EVAL, level);
                    CK(c, launch_gradient(Stored{L.img, c->img_type}, g, fs, cf, ut, c->w_x, (float)best_t, c->w_abar,
                                          c->w_ubar, c->w_g, c->w_dT, c->img_type, u, c->partials, c->partials_cap,
                                          &S->ticket[4], S->red, c->stream));
                    prof_end(c, pe, pfK * B_grad, pfK);
                    TRY(read_scalars(c));
                    for (int k = 0; k < 4; ++k) best4[k] = chk[k];
                    gnorm2 = c->Sh->red[4];
                    unorm2 = c->Sh->red[5];
                }
            }
            J = best4[0];
            D = best4[1];
            Sv = best4[2];
            Pv = best4[3];
            break;
        }
        // the next solve was queued before |g| of the new iterate was known; it
        // is dropped if the stopping tests fire
        started = next_solve;
        if (should_stop()) {
            started = false;
        } else if (targeted) {
            TRY(start_cg());
            TRY(read_scalars(c));
            started = true;
        }
    }
    if (u != u_io) {
        CK(c, cudaMemcpyAsync(u_io, u, M * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
    }
    s.gn_iters = it;
    s.J = J;
    s.D = D;
    s.S = Sv;
    s.P = Pv;
    s.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (st) *st = s;
    return STML_OK;
}

// ------------------------------------------------------- coarse displacement grid
// Buffers of the coarse-grid solver (allocated on first use, sized for the
// finest level and all frames).
stml_status ensure_ugrid(stml_ctx* c) {
    const size_t M = (size_t)c->n * c->d * field_geom(c, (int)c->lv.size() - 1).N;
    if (c->ug_g && c->ug_cap >= M) return STML_OK;
    if (c->ug_g) {   // u_coarsen was lowered since the buffers were made: make them again, larger
        CK(c, cudaStreamSynchronize(c->stream));
        for (float** fp : {&c->ug_g, &c->ug_x, &c->ug_r, &c->ug_z, &c->ug_p, &c->ug_q, &c->ug_m, &c->ug_w}) dfree(*fp);
        dfree(c->ug_part);
        dfree(c->ug_out);
        dfree(c->ug_tk);
        dfree(c->ug_cg);
        if (c->ug_outh) cudaFreeHost(c->ug_outh);
        if (c->ug_cgh) cudaFreeHost(c->ug_cgh);
        c->ug_outh = nullptr;
        c->ug_cgh = nullptr;
    }
    c->ug_cap = 0;
    bool ok = true;
    for (float** fp : {&c->ug_g, &c->ug_x, &c->ug_r, &c->ug_z, &c->ug_p, &c->ug_q, &c->ug_m, &c->ug_w})
        ok = ok && dalloc(fp, M) == cudaSuccess;
    c->ug_part_cap = (size_t)152 * 8 * 8;
    ok = ok && dalloc(&c->ug_part, c->ug_part_cap) == cudaSuccess;
    ok = ok && dalloc(&c->ug_out, 16) == cudaSuccess;
    ok = ok && dalloc(&c->ug_tk, 8) == cudaSuccess;
    ok = ok && cudaMallocHost((void**)&c->ug_outh, 16 * sizeof(double)) == cudaSuccess;
    ok = ok && dalloc(&c->ug_cg, 1) == cudaSuccess;
    ok = ok && cudaMallocHost((void**)&c->ug_cgh, sizeof(UgCg)) == cudaSuccess;
    if (!ok) return fail(c, STML_ENOMEM, "device allocation of the coarse-grid solver buffers failed");
    c->ug_cap = M;
    CK(c, cudaMemsetAsync(c->ug_tk, 0, 8 * sizeof(unsigned int), c->stream));
    // the PCG state mirrors its `active` word into the context's cg_active,
    // which gates the image-grid kernels of the Hessian product
    std::memset(c->ug_cgh, 0, sizeof(UgCg));
    c->ug_cgh->mirror = &c->S->cg_active;
    CK(c, cudaMemcpyAsync(c->ug_cg, c->ug_cgh, sizeof(UgCg), cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return STML_OK;
}

// The first n reduced values of the coarse-grid passes (ug_out) on the host.
stml_status ug_read(stml_ctx* c, int n) {
    CK(c, cudaMemcpyAsync(c->ug_outh, c->ug_out, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return STML_OK;
}

// One objective evaluation with the unknowns w on the coarse grid of the
// level: u = P_s w on the image grid, the distance of eq. (1) there (with
// the gradient: hd r grad T, gathered to the coarse grid by P_s^T), S and P
// on the coarse grid.  o6 = J, D, S, P, |g|^2, |w|^2.  With grad the coarse
// gradient goes to c->ug_g and grad T (image grid) to c->w_dT; with dw the
// objective is taken at w + t dw (no gradient).
struct UgEval {
    stml_ctx* c;
    int level;
    Geom g, gw;
    UGrid ug;
    FrameSet fs;
    Coef cf0, cw;
    long long planes;

    stml_status run(const float* w, const float* dw, float t, bool grad, double* o6) {
        const LevelBuf& L = c->lv[level];
        const Stored img{L.img, c->img_type};
        const double pf = (double)fs.nK * (double)g.N;
        long pe = prof_begin(c, PC_PROLONG, level);
        CK(c, launch_ugrid_prolong(w, dw, t, c->w_ut, planes, ug, c->stream));
        prof_end(c, pe, 4.0 * g.d * pf, pf);
        pe = prof_begin(c, PC_TRIAL, level);
        CK(c, launch_objective(img, g, fs, cf0, c->w_ut, nullptr, 0.f, nullptr, c->w_abar, c->w_ubar, c->partials,
                               c->partials_cap, &c->S->ticket[0], c->S->red, c->stream));
        prof_end(c, pe, pf * (4.0 + 4.0 * g.d), pf);
        if (grad) {
            pe = prof_begin(c, PC_EVAL, level);
            CK(c, launch_gradient(img, g, fs, cf0, c->w_ut, nullptr, 0.f, c->w_abar, c->w_ubar, c->w_g, c->w_dT,
                                  ST_F32, nullptr, c->partials, c->partials_cap, &c->S->ticket[4], c->S->red,
                                  c->stream));
            prof_end(c, pe, pf * (4.0 + 20.0 * g.d), pf);
            pe = prof_begin(c, PC_PROLONG, level);
            CK(c, launch_ugrid_adjoint(c->w_g, c->ug_g, planes, ug, c->stream));
            prof_end(c, pe, 4.0 * g.d * pf, pf);
        }
        CK(c, launch_ugrid_reg(0, gw, fs, cw, w, dw, t, grad ? c->ug_g : nullptr, grad ? c->ug_g : nullptr,
                               c->ug_part, c->ug_part_cap, &c->ug_tk[0], c->ug_out, c->stream));
        TRY(read_scalars(c));
        TRY(ug_read(c, 5));
        const stml_params& p = c->p;
        const double* r = c->ug_outh;
        const double hdw = gw.hd, inv_h2 = 1.0 / ((double)gw.h * gw.h), K = fs.nK;
        const double D = c->Sh->red[1];
        const double Sv = 0.5 * p.alpha * hdw * inv_h2 * r[0] + 0.5 * p.alpha_t * hdw * r[1];
        const double Pv = p.lambda * hdw * r[2] / (K * K);
        o6[0] = D + Sv + Pv;
        o6[1] = D;
        o6[2] = Sv;
        o6[3] = Pv;
        o6[4] = grad ? r[3] : 0.0;
        o6[5] = r[4];
        return STML_OK;
    }

    // q = H p (coarse grid): P_s^T H_D P_s p + the regulariser and penalty
    // Hessian; *pq = <p, q>.
    stml_status hess(const float* pv, float* qv, double* pq) {
        const double pf = (double)fs.nK * (double)g.N;
        long pe = prof_begin(c, PC_PROLONG, level);
        CK(c, launch_ugrid_prolong(pv, nullptr, 0.f, c->w_p, planes, ug, c->stream));
        prof_end(c, pe, 4.0 * g.d * pf, pf);
        TRY(hessvec_launch(c, level, g, fs, cf0, c->w_dT, c->w_p, c->w_q, nullptr));
        pe = prof_begin(c, PC_PROLONG, level);
        CK(c, launch_ugrid_adjoint(c->w_q, qv, planes, ug, c->stream));
        prof_end(c, pe, 4.0 * g.d * pf, pf);
        CK(c, launch_ugrid_reg(1, gw, fs, cw, pv, nullptr, 0.f, qv, qv, c->ug_part, c->ug_part_cap, &c->ug_tk[1],
                               c->ug_out + 5, c->stream));
        if (pq) {
            CK(c, cudaMemcpyAsync(c->ug_outh + 5, c->ug_out + 5, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
            CK(c, cudaStreamSynchronize(c->stream));
            *pq = c->ug_outh[5];
        }
        return STML_OK;
    }

    // One PCG step's Hessian product q = H p, every launch gated on the solve
    // still running; the last CTA of the regulariser pass takes alpha.
    stml_status hess_step(const float* pv, float* qv) {
        const double pf = (double)fs.nK * (double)g.N;
        const int* gate = &c->S->cg_active;
        long pe = prof_begin(c, PC_PROLONG, level);
        CK(c, launch_ugrid_prolong(pv, nullptr, 0.f, c->w_p, planes, ug, c->stream, gate));
        prof_end(c, pe, 4.0 * g.d * pf, pf);
        TRY(hessvec_launch(c, level, g, fs, cf0, c->w_dT, c->w_p, c->w_q, c->S));
        pe = prof_begin(c, PC_PROLONG, level);
        CK(c, launch_ugrid_adjoint(c->w_q, qv, planes, ug, c->stream, gate));
        prof_end(c, pe, 4.0 * g.d * pf, pf);
        CK(c, launch_ugrid_reg(1, gw, fs, cw, pv, nullptr, 0.f, qv, qv, c->ug_part, c->ug_part_cap, &c->ug_tk[1],
                               c->ug_out + 5, c->stream, c->ug_cg));
        return STML_OK;
    }

    stml_status jacobi() {
        CK(c, launch_ugrid_jacobi(c->w_dT, c->ug_m, ug, fs, cf0, cw, c->stream));
        return STML_OK;
    }
};

stml_status ug_setup(stml_ctx* c, int level, const std::vector<int>& K, UgEval& E) {
    TRY(ensure_ugrid(c));
    E.c = c;
    E.level = level;
    E.g = c->lv[level].g;
    E.gw = field_geom(c, level);
    E.ug = make_ugrid(E.g, c->p.u_coarsen);
    TRY(upload_frameset(c, K, E.fs));
    stml_params p0 = c->p;
    p0.alpha = p0.alpha_t = p0.lambda = 0.0;
    E.cf0 = make_coef(E.g, p0, (int)K.size());
    E.cw = make_coef(E.gw, c->p, (int)K.size());
    E.planes = (long long)K.size() * E.g.d;
    return STML_OK;
}

// Deterministic dot product of two coarse-grid vectors of n values.
stml_status ug_dot(stml_ctx* c, long long n, const float* a, const float* b, double* out) {
    CK(c, launch_ugrid_vec(VEC_DOT, n, 0.f, nullptr, const_cast<float*>(a), nullptr, nullptr, const_cast<float*>(b),
                           nullptr, nullptr, c->ug_part, c->ug_part_cap, &c->ug_tk[3], c->ug_out + 8, c->stream));
    CK(c, cudaMemcpyAsync(c->ug_outh + 8, c->ug_out + 8, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    *out = c->ug_outh[8];
    return STML_OK;
}

// GIR(K) with the unknowns on the coarse grid (u_coarsen = s > 0): the same
// Gauss-Newton / Jacobi-PCG / Armijo scheme and stopping tests as run_gir;
// the PCG coefficients and stopping decisions are taken on the device (FP64
// from the deterministic reductions), the host reads the solve's state once
// per chunk of queued steps.
stml_status run_gir_ugrid(stml_ctx* c, int level, const std::vector<int>& K, float* w_io, stml_stats* st) {
    Range rg("GIR on the coarse field grid, level %d |K| %d", level, (int)K.size());
    const auto t_start = std::chrono::steady_clock::now();
    UgEval E;
    TRY(ug_setup(c, level, K, E));
    const stml_params& p = c->p;
    const long long M = E.planes * E.gw.N;
    stml_stats s{};
    s.level = level;
    s.n_frames = (int)K.size();
    s.status = STML_OK;
    float* w = w_io;
    float* wt = c->ug_w;
    double ev[6];
    TRY(E.run(w, nullptr, 0.f, true, ev));
    const double J0 = ev[0];
    double J = ev[0], gnorm2 = ev[4], wnorm2 = ev[5], J_old = 0.0, step_norm = 0.0;
    s.J0 = J0;
    int it = 0, predict_cg = 8;
    double last[4] = {ev[0], ev[1], ev[2], ev[3]};
    for (;;) {
        if (!std::isfinite(J) || !std::isfinite(gnorm2)) {
            s.status = STML_ENONFINITE;
            break;
        }
        const double gnorm = std::sqrt(gnorm2);
        if (it > 0) {
            const bool c1 = std::fabs(J_old - J) <= p.tol_J * (1.0 + std::fabs(J0));
            const bool c2 = step_norm <= p.tol_Y * (1.0 + std::sqrt(wnorm2));
            const bool c3 = gnorm <= p.tol_G * (1.0 + std::fabs(J0));
            if (c1 && c2 && c3) break;
        }
        if (gnorm <= p.g_abs * (1.0 + std::fabs(J0)) || it >= p.max_gn) break;
        // --- Jacobi-PCG for H x = -g from x = 0
        Range rit("Gauss-Newton iteration %d", it);
        TRY(E.jacobi());
        int steps = 0;
        if (gnorm > 0.0) {
            // the coefficients stay on the device; the host queues the
            // previous solve's step count, then chunks of 4, and reads the
            // state once per chunk (launches after the stop return at once)
            CK(c, launch_ugrid_vec(VEC_INIT, M, 0.f, c->ug_m, c->ug_x, c->ug_r, c->ug_z, c->ug_p, nullptr, c->ug_g,
                                   c->ug_part, c->ug_part_cap, &c->ug_tk[2], c->ug_out + 6, c->stream, c->ug_cg,
                                   p.tol_cg * gnorm, p.max_cg));
            int launched = 0, chunk = std::max(2, predict_cg);
            for (;;) {
                const int nq = std::min(chunk, p.max_cg - launched);
                for (int i = 0; i < nq; ++i) {
                    TRY(E.hess_step(c->ug_p, c->ug_q));
                    CK(c, launch_ugrid_vec(VEC_STEP, M, 0.f, c->ug_m, c->ug_x, c->ug_r, c->ug_z, c->ug_p, c->ug_q,
                                           nullptr, c->ug_part, c->ug_part_cap, &c->ug_tk[2], c->ug_out + 6,
                                           c->stream, c->ug_cg));
                    CK(c, launch_ugrid_vec(VEC_DIR, M, 0.f, nullptr, nullptr, nullptr, c->ug_z, c->ug_p, nullptr,
                                           nullptr, c->ug_part, c->ug_part_cap, &c->ug_tk[2], c->ug_out + 6,
                                           c->stream, c->ug_cg));
                }
                launched += nq;
                CK(c, cudaMemcpyAsync(c->ug_cgh, c->ug_cg, sizeof(UgCg), cudaMemcpyDeviceToHost, c->stream));
                CK(c, cudaStreamSynchronize(c->stream));
                if (!c->ug_cgh->active || launched >= p.max_cg) break;
                chunk = 4;
            }
            steps = c->ug_cgh->iter;
            predict_cg = steps;
            // breakdown on the first step: the preconditioned gradient
            if (c->ug_cgh->flag == CG_BREAKDOWN && steps == 0)
                CK(c, cudaMemcpyAsync(c->ug_x, c->ug_z, (size_t)M * sizeof(float), cudaMemcpyDeviceToDevice,
                                      c->stream));
        } else {
            CK(c, cudaMemsetAsync(c->ug_x, 0, (size_t)M * sizeof(float), c->stream));
        }
        s.cg_iters += steps;
        double gTd = 0.0, dd = 0.0;
        TRY(ug_dot(c, M, c->ug_g, c->ug_x, &gTd));
        if (!(gTd < 0.0)) {
            s.status = STML_EBREAKDOWN;
            break;
        }
        TRY(ug_dot(c, M, c->ug_x, c->ug_x, &dd));
        // --- Armijo back-tracking on t = 1, 1/2, ...
        bool accepted = false;
        double t = 1.0, tr[6];
        for (int k = 0; k < p.max_ls; ++k) {
            TRY(E.run(w, c->ug_x, (float)t, false, tr));
            ++s.ls_trials;
            if (tr[0] <= J + p.armijo_c * t * gTd) {
                accepted = true;
                break;
            }
            if (k + 1 < p.max_ls) t *= 0.5;
        }
        if (!accepted) {
            s.status = STML_ELINESEARCH;
            break;
        }
        CK(c, launch_ugrid_vec(VEC_AXPY, M, (float)t, nullptr, w, nullptr, wt, c->ug_x, nullptr, nullptr, c->ug_part,
                               c->ug_part_cap, &c->ug_tk[2], c->ug_out + 6, c->stream));
        std::swap(w, wt);
        step_norm = t * std::sqrt(dd);
        J_old = J;
        TRY(E.run(w, nullptr, 0.f, true, ev));
        J = ev[0];
        gnorm2 = ev[4];
        wnorm2 = ev[5];
        for (int i = 0; i < 4; ++i) last[i] = ev[i];
        ++it;
    }
    if (w != w_io) {
        CK(c, cudaMemcpyAsync(w_io, w, (size_t)M * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
    }
    s.gn_iters = it;
    s.J = last[0];
    s.D = last[1];
    s.S = last[2];
    s.P = last[3];
    s.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (st) *st = s;
    return STML_OK;
}

// ------------------------------------------------------------------ predictors
stml_status upload_idx(stml_ctx* c, const std::vector<int>& K) {
    CK(c, cudaMemcpyAsync(c->d_idx, K.data(), K.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    return STML_OK;
}

// Linear taps: target frame k gets the registered field if k is in K, else
// the interpolation between its neighbours in K.  Indices src_* point into
// the compact (K-ordered) array; dst is the frame number (or target index).
std::vector<LinTap> linear_taps(const std::vector<int>& K, const std::vector<int>& targets, bool dst_is_frame) {
    std::vector<LinTap> taps;
    for (size_t t = 0; t < targets.size(); ++t) {
        const int k = targets[t];
        LinTap tp{};
        tp.dst = dst_is_frame ? k : (int)t;
        auto it = std::lower_bound(K.begin(), K.end(), k);
        if (it != K.end() && *it == k) {
            tp.src_l = tp.src_r = (int)(it - K.begin());
            tp.wl = 1.f;
            tp.wr = 0.f;
        } else {
            const int r = (int)(it - K.begin()), l = r - 1;
            const double kl = K[l], kr = K[r];
            tp.src_l = l;
            tp.src_r = r;
            tp.wl = (float)((kr - k) / (kr - kl));
            tp.wr = (float)((k - kl) / (kr - kl));
        }
        taps.push_back(tp);
    }
    return taps;
}

// Factors of D_K + beta L for Thomas' algorithm, computed in double.
void ls_factors(int n, const std::vector<int>& K, double beta, std::vector<float>& tab, std::vector<int>& kidx) {
    std::vector<double> diag(n, 0.0), sub(n, 0.0), sup(n, 0.0);
    kidx.assign(n, -1);
    for (size_t i = 0; i < K.size(); ++i) {
        diag[K[i]] += 1.0;
        kidx[K[i]] = (int)i;
    }
    for (int k = 0; k + 1 < n; ++k) {
        diag[k] += beta;
        diag[k + 1] += beta;
        sup[k] -= beta;
        sub[k + 1] -= beta;
    }
    tab.assign(3 * (size_t)n, 0.f);
    double cp_prev = 0.0;
    for (int k = 0; k < n; ++k) {
        const double den = k == 0 ? diag[0] : diag[k] - sub[k] * cp_prev;
        const double cp = sup[k] / den;
        tab[k] = (float)cp;
        tab[n + k] = (float)(1.0 / den);
        tab[2 * n + k] = (float)sub[k];
        cp_prev = cp;
    }
}

stml_status run_predict_ls(stml_ctx* c, const std::vector<int>& K, const float* eta, const float* omega,
                           float* zeta, size_t ncomp) {
    std::vector<float> tab;
    std::vector<int> kidx;
    ls_factors(c->n, K, c->p.beta, tab, kidx);
    CK(c, cudaMemcpyAsync(c->d_lsf, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaMemcpyAsync(c->d_kidx, kidx.data(), kidx.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    const long pe = prof_begin(c, PC_PRED_LS, c->cur_level < 0 ? 0 : c->cur_level);
    CK(c, launch_predict_ls(eta, omega, zeta, c->d_lsf, c->d_lsf + c->n, c->d_lsf + 2 * c->n, c->d_kidx, c->n,
                            ncomp, c->stream));
    prof_end(c, pe, (double)ncomp * (16.0 * c->n + 8.0 * K.size()), (double)ncomp * c->n / c->d);
    return STML_OK;
}

stml_status run_predict_linear(stml_ctx* c, const std::vector<int>& K, const std::vector<int>& targets,
                               const float* in, float* out, size_t plane) {
    std::vector<LinTap> taps = linear_taps(K, targets, true);
    CK(c, cudaMemcpyAsync(c->d_taps, taps.data(), taps.size() * sizeof(LinTap), cudaMemcpyHostToDevice, c->stream));
    const long pe = prof_begin(c, PC_PRED_LIN, c->cur_level < 0 ? 0 : c->cur_level);
    CK(c, launch_predict_linear(in, out, c->d_taps, (int)taps.size(), plane, c->stream));
    prof_end(c, pe, 12.0 * plane * taps.size(), (double)plane * taps.size() / c->d);
    return STML_OK;
}

// ----------------------------------------------------------- learned predictor
// Objective of eq. (1) over the frames K of `full` (fields of all frames).
stml_status objective_of(stml_ctx* c, int level, const std::vector<int>& K, const float* full, double* J) {
    LevelBuf& L = c->lv[level];
    const size_t plane = (size_t)L.g.d * L.g.N;
    TRY(upload_idx(c, K));
    CK(c, launch_gather_planes(full, c->w_ut, c->d_idx, (int)K.size(), plane, c->stream));
    FrameSet fs;
    TRY(upload_frameset(c, K, fs));
    const Coef cf = make_coef(L.g, c->p, (int)K.size());
    CK(c, launch_objective(Stored{L.img, c->img_type}, L.g, fs, cf, c->w_ut, nullptr, 0.f, nullptr, c->w_abar,
                           c->w_ubar, c->partials, c->partials_cap, &c->S->ticket[0], c->S->red, c->stream));
    TRY(read_scalars(c));
    *J = c->Sh->red[0];
    return STML_OK;
}

// With a network attached: proposes the fields of `targets` (frames outside
// Kp) from their registered neighbours in Kp (fields in K order in yK) and the
// images, and keeps them in `dst` (fields of all frames, holding the classical
// proposals) only if the objective over the frames Kj is lower with them.
// *decision: -1 no proposal (no network, a 3-D sequence, a level larger than
// the network's canvas, no target between two frames of Kp), 0 classical
// kept, 1 learned kept; *J_classic and *J_kept the two objectives.
stml_status learned_fill(stml_ctx* c, int level, const std::vector<int>& Kp, const float* yK,
                         const std::vector<int>& targets, float* dst, const std::vector<int>& Kj, int* decision,
                         double* J_classic, double* J_kept) {
    *decision = -1;
    LevelBuf& L = c->lv[level];
    if (!c->net || c->d != 2 || c->p.u_coarsen || targets.empty() || !net::fits(c->net, L.g.ny, L.g.nx))
        return STML_OK;
    const size_t plane = (size_t)L.g.d * L.g.N;
    const size_t img_frame = (size_t)L.g.N * store_bytes(c->img_type);
    const char* img = static_cast<const char*>(L.img);
    std::vector<net::Sample> smp;
    std::vector<int> used;
    for (int k : targets) {
        auto it = std::upper_bound(Kp.begin(), Kp.end(), k);
        if (it == Kp.begin() || it == Kp.end() || *(it - 1) == k) continue;
        const int r = *it, l = *(it - 1);
        const size_t il = (size_t)(it - 1 - Kp.begin()), ir = (size_t)(it - Kp.begin());
        smp.push_back(net::Sample{yK + il * plane, yK + ir * plane, img + (size_t)l * img_frame,
                                  img + (size_t)k * img_frame, img + (size_t)r * img_frame, nullptr,
                                  c->w_z2 + (size_t)k * plane, (long long)L.g.N, L.g.nx, L.g.nx, c->img_type,
                                  (float)(r - k) / (float)(r - l), (float)L.g.h});
        used.push_back(k);
    }
    if (smp.empty()) return STML_OK;
    Range rn("learned proposals level %d: %d frames", level, (int)smp.size());
    const long pe = prof_begin(c, PC_PRED_NET, level);
    CK(c, cudaMemcpyAsync(c->w_z2, dst, (size_t)c->n * plane * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
    const int mb = net::max_batch(c->net);
    for (size_t b = 0; b < smp.size(); b += mb) {
        const int nb = (int)std::min(smp.size() - b, (size_t)mb);
        CK(c, net::forward_on(c->net, smp.data() + b, nb, L.g.ny, L.g.nx, c->stream));
    }
    prof_end(c, pe, 0.0, (double)smp.size() * L.g.N);
    double Jc = 0.0, Jn = 0.0;
    TRY(objective_of(c, level, Kj, dst, &Jc));
    TRY(objective_of(c, level, Kj, c->w_z2, &Jn));
    if (net::timed_out(c->net)) return fail(c, STML_ETIMEOUT, "a convolution of the predictor network timed out");
    *J_classic = Jc;
    if (std::isfinite(Jn) && Jn < Jc) {
        for (int k : used)
            CK(c, cudaMemcpyAsync(dst + (size_t)k * plane, c->w_z2 + (size_t)k * plane, plane * sizeof(float),
                                  cudaMemcpyDeviceToDevice, c->stream));
        *decision = 1;
        *J_kept = Jn;
    } else {
        *decision = 0;
        *J_kept = Jc;
    }
    return STML_OK;
}

// ------------------------------------------------------------ affine variant
int aff_P(const stml_ctx* c) { return c->d * (c->d + 1); }

stml_status ensure_affine(stml_ctx* c) {
    if (c->aff_cap >= c->n) return STML_OK;
    for (auto& kv : c->aff_graphs) cudaGraphExecDestroy(kv.second);
    c->aff_graphs.clear();
    const int P = aff_P(c);
    dfree(c->d_theta); dfree(c->d_gth); dfree(c->d_aff_part);
    if (c->h_theta) cudaFreeHost(c->h_theta);
    if (c->h_gth) cudaFreeHost(c->h_gth);
    c->h_theta = nullptr;
    c->h_gth = nullptr;
    CK(c, dalloc(&c->d_theta, (size_t)c->n * P));
    CK(c, dalloc(&c->d_gth, (size_t)c->n * P));
    CK(c, dalloc(&c->d_aff_part, (size_t)c->n * 256 * P));
    CK(c, cudaMallocHost(reinterpret_cast<void**>(&c->h_theta), sizeof(float) * (size_t)c->n * P));
    CK(c, cudaMallocHost(reinterpret_cast<void**>(&c->h_gth), sizeof(double) * (size_t)c->n * P));
    dfree(c->d_mu); dfree(c->d_Q); dfree(c->d_G); dfree(c->d_gpart);
    if (c->h_G) cudaFreeHost(c->h_G);
    c->h_G = nullptr;
    const size_t n2 = (size_t)c->n * c->n;
    CK(c, dalloc(&c->d_mu, (size_t)c->n));
    CK(c, dalloc(&c->d_Q, n2));
    CK(c, dalloc(&c->d_G, n2));
    CK(c, dalloc(&c->d_gpart, 64 * n2 + 1 + (size_t)c->n));    // Gram partials, D_NC, row sums
    CK(c, cudaMallocHost(reinterpret_cast<void**>(&c->h_G), sizeof(double)));
    c->aff_cap = c->n;
    return STML_OK;
}

AffineFrame affine_frame(const stml_ctx* c) {
    AffineFrame af{};
    double ext = 0.0;
    for (int i = 0; i < c->d; ++i) {
        const int axis = 3 - c->d + i;           // component i belongs to array axis i
        af.c[i] = (float)(0.5 * c->shape[axis]);
        ext = std::max(ext, (double)c->shape[axis]);
    }
    af.inv_rho = (float)(2.0 / ext);
    return af;
}

// Uploads theta (host doubles, nK x P) and writes its affine fields to u.
stml_status affine_fields(stml_ctx* c, int level, const double* th, int nK, float* u) {
    TRY(ensure_affine(c));
    const int P = aff_P(c);
    if (c->Sh) CK(c, cudaStreamSynchronize(c->stream));   // staging array free again
    for (long long i = 0; i < (long long)nK * P; ++i) c->h_theta[i] = (float)th[i];
    CK(c, cudaMemcpyAsync(c->d_theta, c->h_theta, sizeof(float) * (size_t)nK * P, cudaMemcpyHostToDevice,
                          c->stream));
    CK(c, launch_affine_field(c->lv[level].g, affine_frame(c), c->d_theta, nK, u, c->stream));
    return STML_OK;
}

// One evaluation on stream st (h_theta already holds theta): upload, affine
// field, objective, and with grad the gradient pass, projection and download
// of dJ/dtheta.  Returns the number of kernels launched.
cudaError_t affine_enqueue(stml_ctx* c, int level, const FrameSet& fs, bool grad, cudaStream_t st) {
    LevelBuf& L = c->lv[level];
    const int nK = fs.nK, P = aff_P(c);
    const Coef cf = make_coef(L.g, c->p, nK);
    cudaError_t e = cudaMemcpyAsync(c->d_theta, c->h_theta, sizeof(float) * (size_t)nK * P, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_affine_field(L.g, affine_frame(c), c->d_theta, nK, c->w_u, st);
    if (e == cudaSuccess)
        e = launch_objective(Stored{L.img, c->img_type}, L.g, fs, cf, c->w_u, nullptr, 0.f, nullptr, c->w_abar,
                             c->w_ubar, c->partials, c->partials_cap, &c->S->ticket[0], c->S->red, st);
    if (grad && e == cudaSuccess)
        e = launch_gradient(Stored{L.img, c->img_type}, L.g, fs, cf, c->w_u, nullptr, 0.f, c->w_abar, c->w_ubar, c->w_g,
                            c->w_dT, ST_F32, nullptr, c->partials, c->partials_cap, &c->S->ticket[4], c->S->red, st);
    if (grad && e == cudaSuccess)
        e = launch_affine_project(L.g, affine_frame(c), c->w_g, nK, c->d_aff_part, c->d_gth, st);
    if (grad && e == cudaSuccess)
        e = cudaMemcpyAsync(c->h_gth, c->d_gth, sizeof(double) * (size_t)nK * P, cudaMemcpyDeviceToHost, st);
    return e;
}

// S (spatial diffusion and temporal terms) and P of eq. (1) at the affine
// fields of theta for the sorted frames K, in closed form (FP64), and their
// gradients added to grad (nK x P, may be null).  An affine field has
// constant forward differences W_ci / rho; sums of quadratic forms over the
// grid use the moments N, sum xhat_i and sum xhat_i xhat_j of the level.
void affine_reg_terms(const stml_ctx* c, int level, const std::vector<int>& K, const double* th, double* S_out,
                      double* P_out, double* grad) {
    const LevelBuf& L = c->lv[level];
    const int d = c->d, P = aff_P(c), nK = (int)K.size();
    const AffineFrame af = affine_frame(c);
    const double h = L.g.h, hd = std::pow(h, d), rho = 1.0 / af.inv_rho;
    int m[3];
    for (int i = 0; i < d; ++i) m[i] = L.shape3[3 - d + i];
    double N = 1.0;
    for (int i = 0; i < d; ++i) N *= m[i];
    double s1[3] = {0, 0, 0}, s2[3] = {0, 0, 0}, E[3];
    for (int i = 0; i < d; ++i) {
        for (int j = 0; j < m[i]; ++j) {
            const double xh = ((j + 0.5) * h - (double)af.c[i]) / rho;
            s1[i] += xh;
            s2[i] += xh * xh;
        }
        E[i] = (m[i] - 1) * N / m[i];
    }
    double S1[3], Mm[3][3];
    for (int i = 0; i < d; ++i) {
        S1[i] = N / m[i] * s1[i];
        for (int j = 0; j < d; ++j) Mm[i][j] = i == j ? N / m[i] * s2[i] : N / ((double)m[i] * m[j]) * s1[i] * s1[j];
    }
    // Q(t) = sum_x |W xhat + b|^2 and its gradient for a parameter vector t
    auto quad = [&](const double* t, double* gq) {
        double q = 0.0;
        for (int cc = 0; cc < d; ++cc) {
            const double* w = t + cc * d;
            const double b = t[d * d + cc];
            double ws = 0.0;
            for (int i = 0; i < d; ++i) {
                double mw = 0.0;
                for (int j = 0; j < d; ++j) mw += Mm[i][j] * w[j];
                q += w[i] * mw;
                ws += w[i] * S1[i];
                if (gq) gq[cc * d + i] = 2.0 * mw + 2.0 * b * S1[i];
            }
            q += 2.0 * b * ws + N * b * b;
            if (gq) gq[d * d + cc] = 2.0 * ws + 2.0 * N * b;
        }
        return q;
    };
    const stml_params& p = c->p;
    double Sx = 0.0;
    for (int k = 0; k < nK; ++k)
        for (int cc = 0; cc < d; ++cc)
            for (int i = 0; i < d; ++i) {
                const double w = th[(size_t)k * P + cc * d + i];
                Sx += 0.5 * p.alpha * hd * E[i] * w * w / (rho * rho);
                if (grad) grad[(size_t)k * P + cc * d + i] += p.alpha * hd * E[i] * w / (rho * rho);
            }
    double St = 0.0;
    std::vector<double> dt(P), gq(P);
    if (p.alpha_t != 0.0)
        for (int k = 0; k + 1 < nK; ++k) {
            const double wk = 1.0 / ((double)(K[k + 1] - K[k]) * (K[k + 1] - K[k]));
            for (int j = 0; j < P; ++j) dt[j] = th[(size_t)(k + 1) * P + j] - th[(size_t)k * P + j];
            St += 0.5 * p.alpha_t * hd * wk * quad(dt.data(), gq.data());
            if (grad)
                for (int j = 0; j < P; ++j) {
                    grad[(size_t)(k + 1) * P + j] += 0.5 * p.alpha_t * hd * wk * gq[j];
                    grad[(size_t)k * P + j] -= 0.5 * p.alpha_t * hd * wk * gq[j];
                }
        }
    std::vector<double> mean(P, 0.0);
    for (int k = 0; k < nK; ++k)
        for (int j = 0; j < P; ++j) mean[j] += th[(size_t)k * P + j] / nK;
    const double Pv = p.lambda * hd * quad(mean.data(), gq.data());
    if (grad)
        for (int k = 0; k < nK; ++k)
            for (int j = 0; j < P; ++j) grad[(size_t)k * P + j] += p.lambda * hd / nK * gq[j];
    *S_out = Sx + St;
    *P_out = Pv;
}

// Normalised-correlation evaluation on stream st (h_theta already holds
// theta): field, warped frames and grad T, Gram matrix, D_NC and Q on the
// device, and with grad the field gradient, its projection and the download
// of dJ/dtheta (D_NC lands in d_G's last slot and is downloaded too).
cudaError_t nc_enqueue(stml_ctx* c, int level, const FrameSet& fs, bool grad, cudaStream_t st) {
    LevelBuf& L = c->lv[level];
    const int nK = fs.nK, P = aff_P(c);
    double* dD = c->d_gpart;                    // slot 0: D_NC; slots 1..nK: srow
    double* srow = c->d_gpart + 1;
    double* gpart = c->d_gpart + 1 + c->n;
    cudaError_t e = cudaMemcpyAsync(c->d_theta, c->h_theta, sizeof(float) * (size_t)nK * P, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_affine_field(L.g, affine_frame(c), c->d_theta, nK, c->w_u, st);
    if (e == cudaSuccess)
        e = launch_nc_warp(Stored{L.img, c->img_type}, L.g, fs, c->w_u, c->w_ut, c->w_dT, c->d_aff_part, c->d_mu, st);
    if (e == cudaSuccess) e = launch_nc_gram(L.g, c->w_ut, c->d_mu, nK, gpart, c->d_G, st);
    if (e == cudaSuccess) e = launch_nc_coeff(c->d_G, nK, srow, c->d_Q, dD, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_G, dD, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (grad && e == cudaSuccess) e = launch_nc_grad(L.g, c->w_ut, c->d_mu, c->d_Q, c->w_dT, nK, c->w_g, st);
    if (grad && e == cudaSuccess)
        e = launch_affine_project(L.g, affine_frame(c), c->w_g, nK, c->d_aff_part, c->d_gth, st);
    if (grad && e == cudaSuccess)
        e = cudaMemcpyAsync(c->h_gth, c->d_gth, sizeof(double) * (size_t)nK * P, cudaMemcpyDeviceToHost, st);
    return e;
}

// Normalised-correlation evaluation (params.distance = 1): D_NC and dD/dtheta
// on the device (one host wait; the second and later evaluations of a
// (level, nK, grad) replay a CUDA graph), S and P in closed form on the host.
stml_status affine_eval_nc(stml_ctx* c, int level, const std::vector<int>& K, const FrameSet& fs, const double* th,
                           double* out4, double* grad) {
    const int nK = fs.nK, P = aff_P(c);
    TRY(ensure_affine(c));
    CK(c, cudaStreamSynchronize(c->stream));
    for (long long i = 0; i < (long long)nK * P; ++i) c->h_theta[i] = (float)th[i];
    const bool g = grad != nullptr;
    const std::array<int, 3> key{level, nK, g ? 3 : 2};    // distinct from the SSD graphs
    auto it = c->prof ? c->aff_graphs.end() : c->aff_graphs.find(key);
    if (it != c->aff_graphs.end()) {
        CK(c, cudaGraphLaunch(it->second, c->stream));
        count_launches(g ? 11 : 8);
    } else {
        CK(c, nc_enqueue(c, level, fs, g, c->stream));
        if (!c->prof) {
            if (!c->cap_stream) cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            if (c->cap_stream &&
                cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                const cudaError_t e1 = nc_enqueue(c, level, fs, g, c->cap_stream);
                const cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &graph);
                if (e1 == cudaSuccess && e2 == cudaSuccess && graph &&
                    cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess)
                    c->aff_graphs[key] = exec;
                if (graph) cudaGraphDestroy(graph);
            }
            cudaGetLastError();
        }
    }
    CK(c, cudaStreamSynchronize(c->stream));
    const double D = c->h_G[0];
    double S = 0.0, Pv = 0.0;
    if (grad) std::fill(grad, grad + (size_t)nK * P, 0.0);
    affine_reg_terms(c, level, K, th, &S, &Pv, grad);
    out4[0] = D + S + Pv;
    out4[1] = D;
    out4[2] = S;
    out4[3] = Pv;
    if (!std::isfinite(out4[0])) return fail(c, STML_ENONFINITE, "objective is not finite");
    if (grad)
        for (long long i = 0; i < (long long)nK * P; ++i) grad[i] += c->h_gth[i];
    return STML_OK;
}

// J, D, S, P and (grad not null) dJ/dtheta at theta for the frames of fs.
// Without profiling, the second and later evaluations of a (level, nK, grad)
// replay a CUDA graph of the sequence.
stml_status affine_eval(stml_ctx* c, int level, const std::vector<int>& K, const FrameSet& fs, const double* th,
                        double* out4, double* grad) {
    if (c->p.distance == 1) return affine_eval_nc(c, level, K, fs, th, out4, grad);
    LevelBuf& L = c->lv[level];
    const int nK = fs.nK, P = aff_P(c);
    TRY(ensure_affine(c));
    CK(c, cudaStreamSynchronize(c->stream));   // the staging arrays are free
    for (long long i = 0; i < (long long)nK * P; ++i) c->h_theta[i] = (float)th[i];
    const bool g = grad != nullptr;
    const std::array<int, 3> key{level, nK, g ? 1 : 0};
    auto it = c->prof ? c->aff_graphs.end() : c->aff_graphs.find(key);
    if (it != c->aff_graphs.end()) {
        CK(c, cudaGraphLaunch(it->second, c->stream));
        count_launches(g ? 5 : 2);
    } else {
        const double pfK = (double)nK * L.g.N;
        const double bS = (double)store_bytes(c->img_type);
        const long pe = prof_begin(c, g ? PC_EVAL : PC_TRIAL, level);
        CK(c, affine_enqueue(c, level, fs, g, c->stream));
        prof_end(c, pe, pfK * (bS + 4.0 * L.g.d + (g ? bS + 24.0 * L.g.d : 0.0)), pfK);
        if (!c->prof) {   // capture the sequence for the next evaluations (best effort)
            if (!c->cap_stream) cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            if (c->cap_stream &&
                cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                const cudaError_t e1 = affine_enqueue(c, level, fs, g, c->cap_stream);
                const cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &graph);
                if (e1 == cudaSuccess && e2 == cudaSuccess && graph &&
                    cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess)
                    c->aff_graphs[key] = exec;
                if (graph) cudaGraphDestroy(graph);
            }
            cudaGetLastError();   // a failed capture leaves no error behind: the eager path stays
        }
    }
    TRY(read_scalars(c));
    for (int i = 0; i < 4; ++i) out4[i] = c->Sh->red[i];
    if (grad) std::memcpy(grad, c->h_gth, sizeof(double) * (size_t)nK * P);
    return std::isfinite(out4[0]) ? STML_OK : fail(c, STML_ENONFINITE, "objective is not finite");
}

double dotv(const std::vector<double>& a, const std::vector<double>& b) {
    double s = 0.0;
    for (size_t i = 0; i < a.size(); ++i) s += a[i] * b[i];
    return s;
}
double normv(const std::vector<double>& a) { return std::sqrt(dotv(a, a)); }

// GIR(K) over the affine parameters by L-BFGS (two-loop recursion), in place.
stml_status run_gir_affine(stml_ctx* c, int level, const std::vector<int>& K, double* th, stml_stats* st) {
    Range rg("affine GIR level %d |K| %d", level, (int)K.size());
    const auto t_start = std::chrono::steady_clock::now();
    const stml_params& p = c->p;
    const int nK = (int)K.size(), P = aff_P(c);
    const size_t n = (size_t)nK * P;
    FrameSet fs;
    TRY(upload_frameset(c, K, fs));
    std::vector<double> x(th, th + n), g(n), xt(n), gt(n), d(n);
    double e[4], et[4];
    TRY(affine_eval(c, level, K, fs, x.data(), e, g.data()));
    stml_stats s{};
    s.level = level;
    s.n_frames = nK;
    s.status = STML_OK;
    s.pred_learned = s.fill_learned = -1;
    const double J0 = e[0];
    s.J0 = J0;
    double J = J0, J_old = 0.0, step = 0.0;
    std::vector<std::vector<double>> S, Y;
    int it = 0;
    while (true) {
        const double gnorm = normv(g);
        if (it > 0) {
            const bool c1 = std::fabs(J_old - J) <= p.tol_J * (1.0 + std::fabs(J0));
            const bool c2 = step <= p.tol_Y * (1.0 + normv(x));
            const bool c3 = gnorm <= p.tol_G * (1.0 + std::fabs(J0));
            if (c1 && c2 && c3) break;
        }
        if (gnorm <= p.g_abs * (1.0 + std::fabs(J0)) || it >= p.max_lbfgs) break;
        bool have = false;
        if (!S.empty()) {   // two-loop recursion, H0 = gamma I from the newest pair
            std::vector<double> q = g, alpha(S.size()), rho(S.size());
            for (int i = (int)S.size() - 1; i >= 0; --i) {
                rho[i] = 1.0 / dotv(Y[i], S[i]);
                alpha[i] = rho[i] * dotv(S[i], q);
                for (size_t j = 0; j < n; ++j) q[j] -= alpha[i] * Y[i][j];
            }
            const double gamma = dotv(S.back(), Y.back()) / dotv(Y.back(), Y.back());
            for (size_t j = 0; j < n; ++j) q[j] *= gamma;
            for (size_t i = 0; i < S.size(); ++i) {
                const double beta = rho[i] * dotv(Y[i], q);
                for (size_t j = 0; j < n; ++j) q[j] += (alpha[i] - beta) * S[i][j];
            }
            for (size_t j = 0; j < n; ++j) d[j] = -q[j];
            have = dotv(g, d) < 0.0;
        }
        if (!have) {        // first step, or not a descent direction: scaled -g, memory cleared
            S.clear();
            Y.clear();
            double gmax = 0.0;
            for (double v : g) gmax = std::max(gmax, std::fabs(v));
            for (size_t j = 0; j < n; ++j) d[j] = -g[j] / gmax;
        }
        const double gTd = dotv(g, d);
        double t = 1.0;
        bool accepted = false;
        for (int trial = 0; trial < p.max_ls; ++trial) {
            ++s.ls_trials;
            for (size_t j = 0; j < n; ++j) xt[j] = x[j] + t * d[j];
            TRY(affine_eval(c, level, K, fs, xt.data(), et, gt.data()));
            if (et[0] <= J + p.armijo_c * t * gTd) {
                accepted = true;
                break;
            }
            t *= 0.5;
        }
        if (!accepted) {
            s.status = STML_ELINESEARCH;
            break;
        }
        std::vector<double> sv(n), yv(n);
        for (size_t j = 0; j < n; ++j) {
            sv[j] = xt[j] - x[j];
            yv[j] = gt[j] - g[j];
        }
        if (dotv(sv, yv) > 1e-12 * normv(sv) * normv(yv)) {
            S.push_back(sv);
            Y.push_back(yv);
            if ((int)S.size() > p.lbfgs_m) {
                S.erase(S.begin());
                Y.erase(Y.begin());
            }
        }
        step = normv(sv);
        x.swap(xt);
        g.swap(gt);
        J_old = J;
        J = et[0];
        std::memcpy(e, et, sizeof(e));
        ++it;
    }
    std::copy(x.begin(), x.end(), th);
    s.gn_iters = it;
    s.cg_iters = 0;
    s.J = e[0];
    s.D = e[1];
    s.S = e[2];
    s.P = e[3];
    s.J0_classic = s.J0;
    s.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (st) *st = s;
    return STML_OK;
}

// Linear predictor of Sec. 3 on the parameters (host): rows of `targets`
// from the rows of thK registered on K.
void aff_predict_linear(const std::vector<int>& K, const double* thK, const std::vector<int>& targets, int P,
                        double* out /* indexed by frame */) {
    for (int k : targets) {
        auto it = std::lower_bound(K.begin(), K.end(), k);
        double* o = out + (size_t)k * P;
        if (it != K.end() && *it == k) {
            std::memcpy(o, thK + (size_t)(it - K.begin()) * P, sizeof(double) * P);
            continue;
        }
        const int ir = (int)(it - K.begin()), il = ir - 1;
        const double wl = (double)(K[ir] - k) / (K[ir] - K[il]), wr = (double)(k - K[il]) / (K[ir] - K[il]);
        for (int j = 0; j < P; ++j) o[j] = wl * thK[(size_t)il * P + j] + wr * thK[(size_t)ir * P + j];
    }
}

// Least-squares predictor of eq. (2) per parameter (host, Thomas):
// zeta = omega + e, (D_K + beta L) e = D_K (eta - omega).
void aff_predict_ls(int n, const std::vector<int>& K, const double* thK, const double* omega, double beta, int P,
                    double* zeta) {
    std::vector<double> sub(n, 0.0), dia(n, 0.0), sup(n, 0.0), cp(n), dp(n), rhs(n);
    std::vector<int> pos(n, -1);
    for (size_t i = 0; i < K.size(); ++i) {
        dia[K[i]] += 1.0;
        pos[K[i]] = (int)i;
    }
    for (int k = 0; k + 1 < n; ++k) {
        dia[k] += beta;
        dia[k + 1] += beta;
        sup[k] -= beta;
        sub[k + 1] -= beta;
    }
    for (int j = 0; j < P; ++j) {
        for (int k = 0; k < n; ++k)
            rhs[k] = pos[k] >= 0 ? thK[(size_t)pos[k] * P + j] - omega[(size_t)k * P + j] : 0.0;
        cp[0] = sup[0] / dia[0];
        dp[0] = rhs[0] / dia[0];
        for (int k = 1; k < n; ++k) {
            const double den = dia[k] - sub[k] * cp[k - 1];
            cp[k] = sup[k] / den;
            dp[k] = (rhs[k] - sub[k] * dp[k - 1]) / den;
        }
        double ek = dp[n - 1];
        zeta[(size_t)(n - 1) * P + j] = omega[(size_t)(n - 1) * P + j] + ek;
        for (int k = n - 2; k >= 0; --k) {
            ek = dp[k] - cp[k] * ek;
            zeta[(size_t)k * P + j] = omega[(size_t)k * P + j] + ek;
        }
    }
}

// STML / SpML over the affine parameters; afterwards every level's fields
// are the affine fields of its result.
stml_status register_affine(stml_ctx* c, stml_mode mode, const std::function<void(const stml_stats&)>& record) {
    const int n = c->n, P = aff_P(c), L = (int)c->lv.size();
    c->theta.assign((size_t)n * P, 0.0);
    std::vector<int> all(n);
    for (int k = 0; k < n; ++k) all[k] = k;
    for (int l = 0; l < L; ++l) {
        if (mode == STML_MODE_SPML) {
            stml_stats s{};
            TRY(run_gir_affine(c, l, all, c->theta.data(), &s));
            s.tlevel = (int)c->sets.size() - 1;
            record(s);
        } else {
            std::vector<double> z = c->theta, zn((size_t)n * P);
            double dhat_prev = 0.0;
            const int Q = (int)c->sets.size();
            for (int q = 0; q < Q; ++q) {
                const std::vector<int>& K = c->sets[q];
                std::vector<double> thK(K.size() * P);
                for (size_t i = 0; i < K.size(); ++i)
                    std::memcpy(&thK[i * P], &z[(size_t)K[i] * P], sizeof(double) * P);
                stml_stats s{};
                TRY(run_gir_affine(c, l, K, thK.data(), &s));
                s.tlevel = q;
                const double dhat = s.D / (double)K.size();
                const bool stop = q > 0 && c->p.stop_rule &&
                                  std::fabs(dhat - dhat_prev) <= c->p.eps_stop * std::fabs(dhat_prev);
                s.stopped_early = stop ? 1 : 0;
                record(s);
                if (q == Q - 1 || stop) {
                    if (q == Q - 1) {
                        for (size_t i = 0; i < K.size(); ++i)
                            std::memcpy(&c->theta[(size_t)K[i] * P], &thK[i * P], sizeof(double) * P);
                    } else if (l == 0) {
                        aff_predict_linear(K, thK.data(), all, P, c->theta.data());
                    } else {
                        aff_predict_ls(n, K, thK.data(), z.data(), c->p.beta, P, c->theta.data());
                        for (size_t i = 0; i < K.size(); ++i)
                            std::memcpy(&c->theta[(size_t)K[i] * P], &thK[i * P], sizeof(double) * P);
                    }
                    break;
                }
                if (l == 0) {
                    aff_predict_linear(K, thK.data(), c->sets[q + 1], P, z.data());
                } else {
                    aff_predict_ls(n, K, thK.data(), z.data(), c->p.beta, P, zn.data());
                    z.swap(zn);
                }
                dhat_prev = dhat;
            }
        }
        TRY(affine_fields(c, l, c->theta.data(), n, c->lv[l].y));
    }
    return STML_OK;
}

// ------------------------------------------------------------------ STML steps
stml_status do_predict(stml_ctx* c, int level, int q) {
    LevelBuf& L = c->lv[level];
    const Geom gf = field_geom(c, level);
    const size_t plane = (size_t)gf.d * gf.N;      // one frame of a field
    const size_t total = (size_t)c->n * plane;
    if (q == 0) {
        if (level == 0) {
            CK(c, cudaMemsetAsync(c->w_z, 0, total * sizeof(float), c->stream));
        } else {
            const LevelBuf& C = c->lv[level - 1];
            if (L.g.nx != 2 * C.g.nx) return fail(c, STML_EINVAL, "level shapes do not halve");
            const Geom gc = field_geom(c, level - 1);
            const long pe = prof_begin(c, PC_PROLONG, level);
            CK(c, launch_prolong(C.y, c->w_z, c->n * c->d, gc, c->stream));
            prof_end(c, pe, 4.0 * c->n * c->d * (double)(gf.N + gc.N), (double)c->n * gf.N);
        }
        c->cur_level = level;
        c->last_q = -1;
        c->level_done = false;
        c->dhat_prev = 0.0;
        return STML_OK;
    }
    if (c->cur_level != level || c->last_q != q - 1 || c->level_done)
        return fail(c, STML_ESTATE, "stml_predict(level, q) needs stml_correct(level, q-1) first");
    const std::vector<int>& Kp = c->sets[q - 1];
    if (level == 0) {
        TRY(run_predict_linear(c, Kp, c->sets[q], c->w_u, c->w_z, plane));
    } else {
        TRY(run_predict_ls(c, Kp, c->w_u, c->w_z, c->w_z2, plane));
        std::swap(c->w_z, c->w_z2);
    }
    if (c->net) {
        std::vector<int> fresh;
        std::set_difference(c->sets[q].begin(), c->sets[q].end(), Kp.begin(), Kp.end(), std::back_inserter(fresh));
        double Jk = 0.0;
        TRY(learned_fill(c, level, Kp, c->w_u, fresh, c->w_z, c->sets[q], &c->pred_learned, &c->J0_classic, &Jk));
    }
    return STML_OK;
}

// The correction of temporal level q in two halves around its GIR: the
// start fields of K_q gathered into w_u, then (with the GIR's statistics)
// the stopping rule eq. (3) and the fields of the level.
stml_status correct_begin(stml_ctx* c, int level, int q) {
    if (c->cur_level != level || c->last_q != q - 1 || c->level_done)
        return fail(c, STML_ESTATE, "stml_correct(level, q) needs stml_predict(level, q) first");
    const Geom gf = field_geom(c, level);
    const size_t plane = (size_t)gf.d * gf.N;
    const std::vector<int>& K = c->sets[q];
    TRY(upload_idx(c, K));
    long pe = prof_begin(c, PC_GATHER, level);
    CK(c, launch_gather_planes(c->w_z, c->w_u, c->d_idx, (int)K.size(), plane, c->stream));
    prof_end(c, pe, 8.0 * plane * K.size(), (double)K.size() * gf.N);
    return STML_OK;
}

stml_status correct_end(stml_ctx* c, int level, int q, stml_stats s, stml_stats* st, int* finished);

stml_status do_correct(stml_ctx* c, int level, int q, stml_stats* st, int* finished) {
    TRY(correct_begin(c, level, q));
    const int Q = (int)c->sets.size();
    stml_stats s{};
    const bool last_gir = level == (int)c->lv.size() - 1 && q == Q - 1;   // the GIR over all frames
    TRY(run_gir(c, level, c->sets[q], c->w_u, &s, last_gir ? c->p.target_J : 0.0));
    return correct_end(c, level, q, s, st, finished);
}

stml_status correct_end(stml_ctx* c, int level, int q, stml_stats s, stml_stats* st, int* finished) {
    LevelBuf& L = c->lv[level];
    const Geom gf = field_geom(c, level);
    const size_t plane = (size_t)gf.d * gf.N;
    const std::vector<int>& K = c->sets[q];
    const int Q = (int)c->sets.size();
    s.tlevel = q;
    s.pred_learned = c->pred_learned;
    s.J0_classic = s.pred_learned >= 0 ? c->J0_classic : s.J0;
    s.fill_learned = -1;
    c->pred_learned = -1;
    const double dhat = s.D / (double)K.size();
    const bool stop = q > 0 && c->p.stop_rule &&
                      std::fabs(dhat - c->dhat_prev) <= c->p.eps_stop * std::fabs(c->dhat_prev);
    s.stopped_early = stop ? 1 : 0;
    c->last_q = q;
    int done = 0;
    if (q == Q - 1) {
        TRY(upload_idx(c, K));
        CK(c, launch_scatter_planes(c->w_u, L.y, c->d_idx, (int)K.size(), plane, c->stream));
        done = 1;
    } else if (stop) {
        std::vector<int> all(c->n);
        for (int k = 0; k < c->n; ++k) all[k] = k;
        if (level == 0) {
            TRY(run_predict_linear(c, K, all, c->w_u, L.y, plane));
        } else {
            TRY(run_predict_ls(c, K, c->w_u, c->w_z, L.y, plane));
            TRY(upload_idx(c, K));
            CK(c, launch_scatter_planes(c->w_u, L.y, c->d_idx, (int)K.size(), plane, c->stream));
        }
        if (c->net) {
            std::vector<int> rest;
            std::set_difference(all.begin(), all.end(), K.begin(), K.end(), std::back_inserter(rest));
            TRY(learned_fill(c, level, K, c->w_u, rest, L.y, all, &s.fill_learned, &s.J_fill_classic, &s.J_fill));
        }
        done = 1;
    }
    c->dhat_prev = dhat;
    c->level_done = done != 0;
    if (st) *st = s;
    if (finished) *finished = done;
    return STML_OK;
}

}  // namespace


// ==================================================================== batched persistent solver
struct stml_batch {
    std::vector<stml_ctx*> ctxs;
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_done = nullptr, ev_a = nullptr, ev_b = nullptr;
    std::vector<cudaEvent_t> ev_ready;    // per context
    int cap = 0;                          // sequences the buffers below hold
    BatchSeq *d_seqs = nullptr, *h_seqs = nullptr;
    BatchState *d_states = nullptr, *h_states = nullptr;
    float2* d_part = nullptr;
    BatchSync *d_sync = nullptr, *h_sync = nullptr;
    // one stage (descriptor and state upload, barrier reset, the persistent
    // kernel, state download) as a CUDA graph per (sequences, d, vec, storage,
    // CTAs per SM, tpr); the uploads copy from the pinned buffers, whose
    // contents are rewritten before every launch
    std::map<std::array<int, 6>, cudaGraphExec_t> graphs;
    // launch shapes chosen by the autotuner per (level, d, vec, storage, sequences)
    std::map<std::array<int, 5>, BatchShape> tuned;
    std::string report;                   // JSON rows of the last registration
    std::string err;
};

namespace {

stml_status bfail(stml_batch* b, stml_status s, const std::string& msg) {
    if (b) b->err = msg;
    else g_free_error = msg;
    return s;
}

#define BCK(b, call)                                                                                      \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess) return bfail((b), STML_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// Runs f(i) for i < n on up to `threads` host threads (each context is
// touched by one thread at a time; its work goes to its own stream).
template <class F>
void parallel_for(int n, F&& f) {
    const int nt = std::max(1, std::min(n, (int)std::max(1u, std::thread::hardware_concurrency())));
    std::atomic<int> next{0};
    auto worker = [&]() {
        for (int i = next.fetch_add(1); i < n; i = next.fetch_add(1)) f(i);
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
    worker();
    for (auto& th : pool) th.join();
}

bool same_solver(const stml_params& a, const stml_params& b) {
    return a.alpha == b.alpha && a.alpha_t == b.alpha_t && a.lambda == b.lambda && a.tol_J == b.tol_J &&
           a.tol_Y == b.tol_Y && a.tol_G == b.tol_G && a.g_abs == b.g_abs && a.max_gn == b.max_gn &&
           a.tol_cg == b.tol_cg && a.max_cg == b.max_cg && a.max_ls == b.max_ls && a.armijo_c == b.armijo_c &&
           a.n_levels == b.n_levels && a.n_tlevels == b.n_tlevels && a.image_dtype == b.image_dtype;
}

// The descriptor of context c's GIR over K at `level` from u0 (all nK d N floats).
BatchSeq batch_seq(stml_ctx* c, int level, const FrameSet& fs, float* u0, int vec, int tpr) {
    LevelBuf& L = c->lv[level];
    const Geom& g = L.g;
    BatchSeq b{};
    b.g = g;
    b.pi = make_pix_index(g);
    b.fs = fs;
    b.cf = make_coef(g, c->p, fs.nK);
    const long long cpf = (g.N + (long long)kThreads * vec - 1) / ((long long)kThreads * vec);
    b.cpf = FastDiv::make((unsigned)cpf);
    b.eval_tiles = (unsigned)((g.N + 32LL * vec - 1) / (32LL * vec));
    b.pcg_tiles = (unsigned)((g.N + (long long)tpr * vec - 1) / ((long long)tpr * vec));
    b.chunks = (unsigned)(cpf * fs.nK);
    b.T = L.img;
    b.u[0] = u0;
    b.u[1] = c->w_ut;
    b.grad = c->w_g;
    b.dT = c->w_dT;
    b.x = c->w_x;
    b.r = c->w_r;
    b.z = c->w_cz;
    b.q = c->w_q;
    b.p[0] = c->w_p;
    b.p[1] = c->w_p2;
    b.ms_z = c->w_m1;
    b.sv_z = c->w_m2;
    b.ms_p[0] = c->w_sp0;
    b.ms_p[1] = c->w_sp1;
    b.sv_p[0] = c->w_sp0 + g.N;
    b.sv_p[1] = c->w_sp1 + g.N;
    b.abar = c->w_abar;
    b.ubar = c->w_ubar;
    return b;
}

stml_status batch_buffers(stml_batch* b, int n) {
    if (n <= b->cap) return STML_OK;
    if (b->d_seqs) cudaFree(b->d_seqs);
    if (b->d_states) cudaFree(b->d_states);
    if (b->h_seqs) cudaFreeHost(b->h_seqs);
    if (b->h_states) cudaFreeHost(b->h_states);
    b->d_seqs = nullptr;
    b->d_states = nullptr;
    b->h_seqs = nullptr;
    b->h_states = nullptr;
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
    b->cap = 0;
    BCK(b, cudaMalloc((void**)&b->d_seqs, n * sizeof(BatchSeq)));
    BCK(b, cudaMalloc((void**)&b->d_states, n * sizeof(BatchState)));
    BCK(b, cudaMallocHost((void**)&b->h_seqs, n * sizeof(BatchSeq)));
    BCK(b, cudaMallocHost((void**)&b->h_states, n * sizeof(BatchState)));
    b->cap = n;
    return STML_OK;
}

// One stage's launches on b->stream: through a graph captured on first use
// of this (sequences, launch shape).
stml_status batch_stage_launch(stml_batch* b, int nseq, const BatchCtl& ctl, int d, int vec, int img, BatchShape sh,
                               int max_steps) {
    const std::array<int, 6> key{nseq, d, vec, img, sh.ctas_per_sm, sh.tpr};
    auto it = b->graphs.find(key);
    if (it == b->graphs.end()) {
        cudaGraph_t gph = nullptr;
        BCK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaMemcpyAsync(b->d_seqs, b->h_seqs, nseq * sizeof(BatchSeq), cudaMemcpyHostToDevice,
                                        b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->d_states, b->h_states, nseq * sizeof(BatchState), cudaMemcpyHostToDevice,
                                b->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->d_sync, 0, sizeof(BatchSync), b->stream);
        if (e == cudaSuccess)
            e = launch_batch_gir(b->d_seqs, nseq, b->d_states, ctl, d, vec, img, sh, b->d_part, b->d_sync, max_steps,
                                 b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->h_states, b->d_states, nseq * sizeof(BatchState), cudaMemcpyDeviceToHost,
                                b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->h_sync, b->d_sync, sizeof(BatchSync), cudaMemcpyDeviceToHost, b->stream);
        const cudaError_t e2 = cudaStreamEndCapture(b->stream, &gph);
        if (e == cudaSuccess) e = e2;
        cudaGraphExec_t ex = nullptr;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, gph, 0);
        if (gph) cudaGraphDestroy(gph);
        if (e != cudaSuccess) return bfail(b, STML_ECUDA, std::string("batched stage graph: ") + cudaGetErrorString(e));
        it = b->graphs.emplace(key, ex).first;
    }
    BCK(b, cudaGraphLaunch(it->second, b->stream));
    return STML_OK;
}

}  // namespace


namespace {

// STML / SpML over the sequences of a batch: per (spatial level, temporal
// level) stage the predictors and gathers of every context (on its own
// stream, several host threads), then one persistent launch for all GIRs of
// the stage, then the stopping rule eq. (3) and the fields of each context.
stml_status batch_register(stml_batch* b, stml_mode mode, stml_status* status) {
    const int n = (int)b->ctxs.size();
    stml_ctx* c0 = b->ctxs[0];
    for (int i = 0; i < n; ++i) {
        stml_ctx* c = b->ctxs[i];
        if (!c->built) return bfail(b, STML_ESTATE, "stml_batch_register: a context has no pyramid");
        if (c->device != b->device) return bfail(b, STML_EINVAL, "stml_batch_register: contexts on several devices");
        if (c->p.transform != 0) return bfail(b, STML_EINVAL, "stml_batch_register: transform 0 only");
        if (c->p.u_coarsen != 0) return bfail(b, STML_EINVAL, "stml_batch_register: u_coarsen 0 only");
        if (c->d != c0->d || c->img_type != c0->img_type || !same_solver(c->p, c0->p) ||
            c->lv.size() != c0->lv.size() || c->sets.size() != c0->sets.size())
            return bfail(b, STML_EINVAL,
                         "stml_batch_register: contexts need the same dimension, image storage, level counts and "
                         "solver parameters");
    }
    const stml_params& P = c0->p;
    const int d = c0->d, img = c0->img_type, L = (int)c0->lv.size(), Q = (int)c0->sets.size();
    int vec = 4;
    for (stml_ctx* c : b->ctxs)
        for (const LevelBuf& B : c->lv)
            if (B.g.nx % 4) vec = 1;
    const BatchCtl ctl{(float)P.tol_cg, P.max_cg, P.max_gn, P.max_ls, P.armijo_c, P.tol_J, P.tol_Y, P.tol_G, P.g_abs};
    const int max_steps = P.max_gn * (2 * P.max_cg + P.max_ls + 3) + 8;
    TRY(batch_buffers(b, n));
    for (stml_ctx* c : b->ctxs) c->last_stats.clear();
    std::vector<stml_status> st(n, STML_OK);
    std::string rep = "[";
    auto fail_ctx = [&](int i, stml_status r) {
        if (st[i] == STML_OK) st[i] = r;
    };
    for (int l = 0; l < L; ++l) {
        parallel_for(n, [&](int i) {
            if (st[i] != STML_OK) return;
            stml_ctx* c = b->ctxs[i];
            cudaSetDevice(c->device);
            stml_status r = do_predict(c, l, 0);
            if (r == STML_OK && mode == STML_MODE_SPML) {
                LevelBuf& B = c->lv[l];
                const cudaError_t e = cudaMemcpyAsync(B.y, c->w_z, (size_t)c->n * c->d * B.g.N * sizeof(float),
                                                      cudaMemcpyDeviceToDevice, c->stream);
                if (e != cudaSuccess) r = cuda_fail(c, e, "cudaMemcpyAsync");
            }
            fail_ctx(i, r);
        });
        const int stages = mode == STML_MODE_SPML ? 1 : Q;
        for (int q = 0; q < stages; ++q) {
            std::vector<int> act;
            for (int i = 0; i < n; ++i)
                if (st[i] == STML_OK && !(mode == STML_MODE_STML && b->ctxs[i]->level_done)) act.push_back(i);
            if (act.empty()) break;
            if (mode == STML_MODE_STML && q > 0) {   // z_{l,q}: the predictor from the fields of K_{q-1}
                parallel_for((int)act.size(), [&](int a) {
                    stml_ctx* c = b->ctxs[act[a]];
                    cudaSetDevice(c->device);
                    fail_ctx(act[a], do_predict(c, l, q));
                });
                std::vector<int> keep;
                for (int i : act)
                    if (st[i] == STML_OK) keep.push_back(i);
                act.swap(keep);
                if (act.empty()) break;
            }
            // the starts of the stage (re-made for every launch shape the autotuner tries)
            auto prepare = [&](const BatchShape& sh, std::vector<int>& run) {
                std::vector<int> ok(act.size(), 0);
                parallel_for((int)act.size(), [&](int a) {
                    const int i = act[a];
                    stml_ctx* c = b->ctxs[i];
                    cudaSetDevice(c->device);
                    stml_status r = STML_OK;
                    float* u0 = nullptr;
                    std::vector<int> K;
                    if (mode == STML_MODE_STML) {
                        r = correct_begin(c, l, q);
                        u0 = c->w_u;
                        K = c->sets[q];
                    } else {
                        LevelBuf& B = c->lv[l];
                        K.resize(c->n);
                        for (int k = 0; k < c->n; ++k) K[k] = k;
                        u0 = B.y;
                        const cudaError_t e = cudaMemcpyAsync(B.y, c->w_z, (size_t)c->n * c->d * B.g.N * sizeof(float),
                                                              cudaMemcpyDeviceToDevice, c->stream);
                        if (e != cudaSuccess) r = cuda_fail(c, e, "cudaMemcpyAsync");
                    }
                    FrameSet fs{};
                    if (r == STML_OK) r = upload_frameset(c, K, fs);
                    if (r == STML_OK) {
                        b->h_seqs[a] = batch_seq(c, l, fs, u0, vec, sh.tpr);
                        // the last GIR over all frames on the finest level may stop at the target objective
                        const bool last_gir = l == L - 1 && (mode == STML_MODE_SPML || q == Q - 1);
                        b->h_seqs[a].target = last_gir ? c->p.target_J : 0.0;
                        b->h_seqs[a].target_tol = c->p.target_tol;
                        const cudaError_t e = cudaEventRecord(b->ev_ready[i], c->stream);
                        if (e != cudaSuccess) r = cuda_fail(c, e, "cudaEventRecord");
                    }
                    if (r == STML_OK) ok[a] = 1;
                    else fail_ctx(i, r);
                });
                // compact the slots of the contexts that are still in the stage
                run.clear();
                int w = 0;
                for (size_t a = 0; a < act.size(); ++a) {
                    if (!ok[a]) continue;
                    b->h_seqs[w] = b->h_seqs[a];
                    BatchState z{};
                    z.phase = BPH_EVAL0;
                    z.status = STML_OK;
                    b->h_states[w] = z;
                    run.push_back(act[a]);
                    ++w;
                }
            };
            auto launch = [&](const BatchShape& sh, const std::vector<int>& run, float* ms) -> stml_status {
                if (run.empty()) return STML_OK;
                const int grid = batch_grid(d, vec, img, sh);
                if (grid < (int)run.size())
                    return bfail(b, STML_EINVAL, "stml_batch_register: " + std::to_string(run.size()) +
                                                     " sequences, the persistent grid holds " + std::to_string(grid));
                for (int i : run) BCK(b, cudaStreamWaitEvent(b->stream, b->ev_ready[i], 0));
                BCK(b, cudaEventRecord(b->ev_a, b->stream));
                TRY(batch_stage_launch(b, (int)run.size(), ctl, d, vec, img, sh, max_steps));
                BCK(b, cudaEventRecord(b->ev_b, b->stream));
                BCK(b, cudaEventRecord(b->ev_done, b->stream));
                BCK(b, cudaStreamSynchronize(b->stream));
                BCK(b, cudaEventElapsedTime(ms, b->ev_a, b->ev_b));
                if (b->h_sync->err & 1u) return bfail(b, STML_ETIMEOUT, "a grid barrier of the batched solver expired");
                if (b->h_sync->err & 6u) return bfail(b, STML_ESTATE, "the batched solver ran out of steps");
                return STML_OK;
            };
            BatchShape sh{2, 16};
            std::vector<int> run;
            const std::array<int, 5> tkey{l, d, vec, img, (int)act.size()};
            const auto tk = b->tuned.find(tkey);
            if (tk != b->tuned.end()) {
                sh = tk->second;
            } else if (P.autotune && q == 0) {
                // time one launch of this stage per candidate shape and keep the fastest
                float best = 1e30f;
                const BatchShape cands[4] = {{2, 16}, {2, 4}, {1, 16}, {1, 4}};
                std::string rows;
                for (const BatchShape& cs : cands) {
                    if (batch_grid(d, vec, img, cs) < (int)act.size()) continue;
                    prepare(cs, run);
                    float ms = 0.f;
                    TRY(launch(cs, run, &ms));
                    for (int i : run) BCK(b, cudaStreamWaitEvent(b->ctxs[i]->stream, b->ev_done, 0));
                    char row[96];
                    std::snprintf(row, sizeof(row), "%s{\"ctas_per_sm\": %d, \"tpr\": %d, \"ms\": %.4f}",
                                  rows.empty() ? "" : ", ", cs.ctas_per_sm, cs.tpr, ms);
                    rows += row;
                    if (ms < best) {
                        best = ms;
                        sh = cs;
                    }
                }
                b->tuned[tkey] = sh;
                char row[160];
                std::snprintf(row, sizeof(row), "%s{\"tuned_level\": %d, \"sequences\": %d, \"chosen\": {\"ctas_per_sm\": %d, \"tpr\": %d}, \"tried\": [",
                              rep.size() > 1 ? ", " : "", l, (int)act.size(), sh.ctas_per_sm, sh.tpr);
                rep += row + rows + "]}";
            }
            prepare(sh, run);
            float ms = 0.f;
            const stml_status lr = launch(sh, run, &ms);
            if (lr != STML_OK) {
                for (int i : run) fail_ctx(i, lr);
                break;
            }
            {
                char row[200];
                std::snprintf(row, sizeof(row),
                              "%s{\"level\": %d, \"tlevel\": %d, \"sequences\": %d, \"steps\": %u, \"ms\": %.4f, "
                              "\"ctas_per_sm\": %d, \"tpr\": %d}",
                              rep.size() > 1 ? ", " : "", l, mode == STML_MODE_STML ? q : Q - 1, (int)run.size(),
                              b->h_sync->steps, ms, sh.ctas_per_sm, sh.tpr);
                rep += row;
            }
            parallel_for((int)run.size(), [&](int a) {
                const int i = run[a];
                stml_ctx* c = b->ctxs[i];
                cudaSetDevice(c->device);
                const BatchState S = b->h_states[a];
                const BatchSeq& D = b->h_seqs[a];
                stml_status r = STML_OK;
                cudaError_t e = cudaStreamWaitEvent(c->stream, b->ev_done, 0);
                if (e == cudaSuccess && S.cur == 1)
                    e = cudaMemcpyAsync(D.u[0], D.u[1], (size_t)D.fs.nK * c->d * D.g.N * sizeof(float),
                                        cudaMemcpyDeviceToDevice, c->stream);
                if (e != cudaSuccess) r = cuda_fail(c, e, "cudaMemcpyAsync");
                stml_stats s{};
                s.level = l;
                s.n_frames = D.fs.nK;
                s.gn_iters = S.it;
                s.cg_iters = S.cg_total;
                s.ls_trials = S.ls_total;
                s.status = S.status;
                s.J0 = S.J0;
                s.J = S.J;
                s.D = S.D;
                s.S = S.S;
                s.P = S.P;
                s.seconds = ms / 1e3;
                s.pred_learned = -1;
                s.fill_learned = -1;
                if (r == STML_OK && mode == STML_MODE_STML) {
                    stml_stats out{};
                    int fin = 0;
                    r = correct_end(c, l, q, s, &out, &fin);
                    if (r == STML_OK) c->last_stats.push_back(out);
                } else if (r == STML_OK) {
                    s.tlevel = Q - 1;
                    s.J0_classic = s.J0;
                    c->last_stats.push_back(s);
                    c->level_done = true;
                }
                fail_ctx(i, r);
            });
        }
    }
    parallel_for(n, [&](int i) {
        stml_ctx* c = b->ctxs[i];
        cudaSetDevice(c->device);
        const cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) fail_ctx(i, cuda_fail(c, e, "cudaStreamSynchronize"));
    });
    rep += "]";
    b->report = rep;
    stml_status first = STML_OK;
    for (int i = 0; i < n; ++i) {
        if (status) status[i] = st[i];
        if (first == STML_OK && st[i] != STML_OK) {
            first = st[i];
            b->err = "context " + std::to_string(i) + ": " + b->ctxs[i]->err;
        }
    }
    return first;
}

void batch_free(stml_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
    if (b->d_seqs) cudaFree(b->d_seqs);
    if (b->d_states) cudaFree(b->d_states);
    if (b->d_part) cudaFree(b->d_part);
    if (b->d_sync) cudaFree(b->d_sync);
    if (b->h_seqs) cudaFreeHost(b->h_seqs);
    if (b->h_states) cudaFreeHost(b->h_states);
    if (b->h_sync) cudaFreeHost(b->h_sync);
    for (cudaEvent_t e : b->ev_ready) cudaEventDestroy(e);
    if (b->ev_done) cudaEventDestroy(b->ev_done);
    if (b->ev_a) cudaEventDestroy(b->ev_a);
    if (b->ev_b) cudaEventDestroy(b->ev_b);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // namespace

// ==================================================================== C ABI
extern "C" {

void stml_default_params(stml_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->alpha = 0.02;
    p->alpha_t = 0.0;
    p->lambda = 1.0;
    p->beta = 1e-5;
    p->eps_stop = 1e-3;
    p->stop_rule = 1;
    p->n_levels = 2;
    p->n_tlevels = 2;
    p->tol_J = 1e-3;
    p->tol_Y = 1e-2;
    p->tol_G = 5e-2;
    p->g_abs = 1e-12;
    p->max_gn = 40;
    p->tol_cg = 1e-1;
    p->max_cg = 20;
    p->max_ls = 10;
    p->armijo_c = 1e-4;
    p->image_dtype = STML_DTYPE_F32;
    p->pcg_cooperative = 1;
    p->autotune = 0;
    p->transform = 0;
    p->lbfgs_m = 5;
    p->max_lbfgs = 50;
    p->distance = 0;
    p->target_J = 0.0;
    p->target_tol = 1e-5;
}

stml_status stml_create(const stml_params* p, void* cuda_stream, stml_ctx** out) {
    if (!out) return fail(nullptr, STML_EINVAL, "out is NULL");
    *out = nullptr;
    std::string why;
    if (!valid_params(p, why)) return fail(nullptr, STML_EINVAL, why);
    stml_ctx* c = new (std::nothrow) stml_ctx();
    if (!c) return fail(nullptr, STML_ENOMEM, "host allocation failed");
    c->p = *p;
    c->stream = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = dalloc(&c->S, 1);
    if (e == cudaSuccess) e = cudaMemset(c->S, 0, sizeof(DevScalars));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&c->Sh, sizeof(DevScalars));
    if (e != cudaSuccess) {
        g_free_error = std::string("stml_create: ") + cudaGetErrorString(e);
        dfree(c->S);
        delete c;
        return STML_ECUDA;
    }
    std::memset(c->Sh, 0, sizeof(DevScalars));
    *out = c;
    return STML_OK;
}

void stml_destroy(stml_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    free_buffers(c);
    for (auto& pr : c->ev) {
        cudaEventDestroy(pr.a);
        cudaEventDestroy(pr.b);
    }
    dfree(c->S);
    if (c->Sh) cudaFreeHost(c->Sh);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
}

const char* stml_last_error(const stml_ctx* c) { return c ? c->err.c_str() : g_free_error.c_str(); }

stml_status stml_set_params(stml_ctx* c, const stml_params* p) {
    if (!c) return fail(nullptr, STML_EINVAL, "ctx is NULL");
    std::string why;
    if (!valid_params(p, why)) return fail(c, STML_EINVAL, why);
    if (c->loaded && (p->n_levels != c->p.n_levels || p->n_tlevels != c->p.n_tlevels))
        return fail(c, STML_EINVAL, "level counts cannot change after stml_load_sequence");
    if (c->loaded) {
        const int f = 1 << (p->n_levels - 1 + p->u_coarsen);
        for (int i = 3 - c->d; i < 3; ++i)
            if (c->shape[i] % f)
                return fail(c, STML_EINVAL, "the loaded shape is not a multiple of 2^(n_levels-1+u_coarsen)");
    }
    c->p = *p;
    return STML_OK;
}

// Copies the frames of a loaded layout into the finest level (rounding them
// to the storage type), clears the fields and the device scalars.
static stml_status load_frames(stml_ctx* c, const float* frames, int on_device) {
    const int L = (int)c->lv.size();
    const int n_frames = c->n, dim = c->d;
    const size_t imgN = (size_t)n_frames * c->lv[L - 1].g.N;
    CK(c, cudaMemsetAsync(c->S, 0, sizeof(DevScalars), c->stream));
    if (c->img_type == ST_F32) {
        CK(c, cudaMemcpyAsync(c->lv[L - 1].img, frames, imgN * sizeof(float),
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    } else {   // 16-bit storage: round the float frames (host frames pass through the workspace)
        const float* src = frames;
        if (!on_device) {
            CK(c, cudaMemcpyAsync(c->w_g, frames, imgN * sizeof(float), cudaMemcpyHostToDevice, c->stream));
            src = c->w_g;
        }
        CK(c, launch_to_store(src, c->lv[L - 1].img, c->img_type, (long long)imgN, c->stream));
    }
    for (int l = 0; l < L; ++l)
        CK(c, cudaMemsetAsync(c->lv[l].y, 0, (size_t)n_frames * dim * c->lv[l].g.N * sizeof(float), c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    c->loaded = true;
    c->built = false;
    return STML_OK;
}

stml_status stml_load_sequence(stml_ctx* c, const float* frames, int on_device, int n_frames, int dim,
                               const int* shape) {
    if (!c) return fail(nullptr, STML_EINVAL, "ctx is NULL");
    if (!frames || !shape || n_frames < 1 || (dim != 2 && dim != 3))
        return fail(c, STML_EINVAL, "need frames, shape, n_frames >= 1 and dim 2 or 3");
    cudaSetDevice(c->device);
    const int L = c->p.n_levels;
    const long long f = 1LL << (L - 1 + c->p.u_coarsen);
    int sh3[3] = {1, 1, 1};
    for (int i = 0; i < dim; ++i) {
        if (shape[i] < 1 || shape[i] % f)
            return fail(c, STML_EINVAL, "every axis must be a positive multiple of 2^(n_levels-1+u_coarsen)");
        if (shape[i] > 65535) return fail(c, STML_EINVAL, "an axis has more than 65535 cells");
        sh3[3 - dim + i] = shape[i];
    }
    if ((long long)sh3[0] * sh3[1] * sh3[2] > 0x7fffffffLL)
        return fail(c, STML_EINVAL, "an image has more than 2^31 - 1 cells");
    // a sequence of the same size, storage and level count reuses the buffers
    // (no device-wide synchronising free / allocation between sequences)
    const bool reuse = c->loaded && c->n == n_frames && c->d == dim && c->img_type == c->p.image_dtype &&
                       (int)c->lv.size() == L && std::memcmp(c->shape, sh3, sizeof(sh3)) == 0;
    if (reuse) return load_frames(c, frames, on_device);
    CK(c, cudaStreamSynchronize(c->stream));
    free_buffers(c);
    c->n = n_frames;
    c->d = dim;
    c->img_type = c->p.image_dtype;
    std::memcpy(c->shape, sh3, sizeof(sh3));
    c->lv.resize(L);
    for (int l = 0; l < L; ++l) {
        const int div = 1 << (L - 1 - l);
        LevelBuf& B = c->lv[l];
        B.shape3[0] = dim == 3 ? sh3[0] / div : 1;
        B.shape3[1] = sh3[1] / div;
        B.shape3[2] = sh3[2] / div;
        B.g = make_geom(B.shape3, dim, (float)div);
        if (cudaMalloc(&B.img, (size_t)n_frames * B.g.N * store_bytes(c->img_type)) != cudaSuccess ||
            dalloc(&B.y, (size_t)n_frames * dim * B.g.N) != cudaSuccess) {
            free_buffers(c);
            return fail(c, STML_ENOMEM, "device allocation of the level buffers failed");
        }
    }
    const Geom& G = c->lv[L - 1].g;
    const size_t fieldN = (size_t)n_frames * dim * G.N;
    size_t pcap = 0;
    for (int l = 0; l < L; ++l)
        pcap = std::max(pcap, std::max(eval_partials(c->lv[l].g, n_frames), gn_partials(c->lv[l].g, n_frames)));
    pcap += 1024 * kMaxRed;
    c->partials_cap = pcap;
    bool ok = true;
    float** fields[] = {&c->w_u, &c->w_g, &c->w_dT, &c->w_x, &c->w_r, &c->w_p, &c->w_q, &c->w_ut, &c->w_z, &c->w_z2,
                        &c->w_p2, &c->w_cz};
    for (float** fp : fields) ok = ok && dalloc(fp, fieldN) == cudaSuccess;
    ok = ok && dalloc(&c->w_abar, (size_t)G.N) == cudaSuccess;
    ok = ok && dalloc(&c->w_ubar, (size_t)dim * G.N) == cudaSuccess;
    ok = ok && dalloc(&c->w_m1, (size_t)G.N) == cudaSuccess;
    ok = ok && dalloc(&c->w_m2, (size_t)dim * G.N) == cudaSuccess;
    ok = ok && dalloc(&c->w_sp0, (size_t)(1 + dim) * G.N) == cudaSuccess;
    ok = ok && dalloc(&c->w_sp1, (size_t)(1 + dim) * G.N) == cudaSuccess;
    ok = ok && dalloc(&c->partials, pcap) == cudaSuccess;
    ok = ok && dalloc(&c->d_frames, n_frames) == cudaSuccess;
    ok = ok && dalloc(&c->d_wnext, n_frames) == cudaSuccess;
    ok = ok && dalloc(&c->d_idx, n_frames) == cudaSuccess;
    ok = ok && dalloc(&c->d_lsf, 3 * (size_t)n_frames) == cudaSuccess;
    ok = ok && dalloc(&c->d_kidx, n_frames) == cudaSuccess;
    ok = ok && dalloc(&c->d_taps, n_frames) == cudaSuccess;
    ok = ok && dalloc(&c->d_rho, n_frames) == cudaSuccess;
    if (!ok) {
        free_buffers(c);
        return fail(c, STML_ENOMEM, "device allocation of the solver workspace failed");
    }
    return load_frames(c, frames, on_device);
}

stml_status stml_build_pyramid(stml_ctx* c) {
    if (!c) return fail(nullptr, STML_EINVAL, "ctx is NULL");
    if (!c->loaded) return fail(c, STML_ESTATE, "no sequence loaded");
    cudaSetDevice(c->device);
    const int L = (int)c->lv.size();
    for (int l = L - 1; l > 0; --l)
        CK(c, launch_restrict(c->lv[l].img, c->lv[l - 1].img, c->img_type, c->n, c->lv[l - 1].g, c->stream));
    c->sets = make_sets(c->n, c->p.n_tlevels);
    c->built = true;
    c->cur_level = -1;
    return STML_OK;
}

stml_status stml_level_info(const stml_ctx* c, int level, int* shape3, double* h) {
    if (!c) return fail(nullptr, STML_EINVAL, "ctx is NULL");
    if (!c->loaded || level < 0 || level >= (int)c->lv.size()) return STML_EINVAL;
    if (shape3) std::memcpy(shape3, c->lv[level].shape3, 3 * sizeof(int));
    if (h) *h = c->lv[level].g.h;
    return STML_OK;
}

stml_status stml_temporal_set(const stml_ctx* c, int tlevel, int* frames, int cap, int* count) {
    if (!c) return fail(nullptr, STML_EINVAL, "ctx is NULL");
    if (!c->built || tlevel < 0 || tlevel >= (int)c->sets.size()) return STML_EINVAL;
    const std::vector<int>& K = c->sets[tlevel];
    if (count) *count = (int)K.size();
    if (frames)
        for (int i = 0; i < cap && i < (int)K.size(); ++i) frames[i] = K[i];
    return STML_OK;
}

stml_status stml_get_images(stml_ctx* c, int level, float* dst, int dst_on_device) {
    if (!c) return fail(nullptr, STML_EINVAL, "ctx is NULL");
    TRY(check_level(c, level));
    cudaSetDevice(c->device);
    const size_t cnt = (size_t)c->n * c->lv[level].g.N;
    if (c->img_type == ST_F32) {
        CK(c, cudaMemcpyAsync(dst, c->lv[level].img, cnt * sizeof(float),
                              dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    } else if (dst_on_device) {
        CK(c, launch_from_store(c->lv[level].img, c->img_type, dst, (long long)cnt, c->stream));
    } else {
        CK(c, launch_from_store(c->lv[level].img, c->img_type, c->w_g, (long long)cnt, c->stream));
        CK(c, cudaMemcpyAsync(dst, c->w_g, cnt * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    }
    CK(c, cudaStreamSynchronize(c->stream));
    return STML_OK;
}

stml_status stml_get_field(stml_ctx* c, int level, float* dst, int dst_on_device) {
    if (!c) return fail(nullptr, STML_EINVAL, "ctx is NULL");
    TRY(check_level(c, level));
    cudaSetDevice(c->device);
    const size_t cnt = (size_t)c->n * c->d * field_geom(c, level).N;
    CK(c, cudaMemcpyAsync(dst, c->lv[level].y, cnt * sizeof(float),
                          dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return STML_OK;
}

stml_status stml_set_field(stml_ctx* c, int level, const float* src, int src_on_device) {
    if (!c) return fail(nullptr, STML_EINVAL, "ctx is NULL");
    TRY(check_level(c, level));
    cudaSetDevice(c->device);
    const size_t cnt = (size_t)c->n * c->d * field_geom(c, level).N;
    CK(c, cudaMemcpyAsync(c->lv[level].y, src, cnt * sizeof(float),
                          src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return STML_OK;
}

stml_status stml_predict(stml_ctx* c, int level, int tlevel) {
    if (c && c->p.transform != 0) return fail(c, STML_EINVAL, "stml_predict serves transform 0 only");
    if (!c) return fail(nullptr, STML_EINVAL, "ctx is NULL");
    TRY(check_level(c, level));
    if (tlevel < 0 || tlevel >= (int)c->sets.size()) return fail(c, STML_EINVAL, "tlevel out of range");
    cudaSetDevice(c->device);
    return do_predict(c, level, tlevel);
}

stml_status stml_correct(stml_ctx* c, int level, int tlevel, stml_stats* stats, int* finished) {
    if (c && c->p.transform != 0) return fail(c, STML_EINVAL, "stml_correct serves transform 0 only");
    if (!c) return fail(nullptr, STML_EINVAL, "ctx is NULL");
    TRY(check_level(c, level));
    if (tlevel < 0 || tlevel >= (int)c->sets.size()) return fail(c, STML_EINVAL, "tlevel out of range");
    cudaSetDevice(c->device);
    return do_correct(c, level, tlevel, stats, finished);
}

stml_status stml_register(stml_ctx* c, stml_mode mode, stml_stats* stats, int cap, int* n_written) {
    if (!c) return fail(nullptr, STML_EINVAL, "ctx is NULL");
    if (!c->built) return fail(c, STML_ESTATE, "no pyramid: call stml_build_pyramid");
    if (mode != STML_MODE_STML && mode != STML_MODE_SPML) return fail(c, STML_EINVAL, "unknown mode");
    cudaSetDevice(c->device);
    int written = 0;
    c->last_stats.clear();
    auto record = [&](const stml_stats& s) {
        if (stats && written < cap) stats[written] = s;
        c->last_stats.push_back(s);
        ++written;
    };
    const int L = (int)c->lv.size();
    std::vector<int> all(c->n);
    for (int k = 0; k < c->n; ++k) all[k] = k;
    if (c->p.transform == 1) {
        TRY(register_affine(c, mode, record));
        CK(c, cudaStreamSynchronize(c->stream));
        if (n_written) *n_written = written;
        return STML_OK;
    }
    for (int l = 0; l < L; ++l) {
        Range rl("level %d", l);
        if (mode == STML_MODE_SPML) {
            TRY(do_predict(c, l, 0));
            LevelBuf& B = c->lv[l];
            const size_t total = (size_t)c->n * c->d * field_geom(c, l).N;
            CK(c, cudaMemcpyAsync(B.y, c->w_z, total * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
            stml_stats s{};
            TRY(run_gir(c, l, all, B.y, &s, l == L - 1 ? c->p.target_J : 0.0));
            s.tlevel = (int)c->sets.size() - 1;
            record(s);
            c->level_done = true;
        } else {
            for (int q = 0; q < (int)c->sets.size(); ++q) {
                Range rq("level %d temporal level %d", l, q);
                TRY(do_predict(c, l, q));
                stml_stats s{};
                int fin = 0;
                TRY(do_correct(c, l, q, &s, &fin));
                record(s);
                if (fin) break;
            }
        }
    }
    CK(c, cudaStreamSynchronize(c->stream));
    if (n_written) *n_written = written;
    return STML_OK;
}

stml_status stml_set_predictor_net(stml_ctx* c, stml_net* net) {
    if (!c) return fail(nullptr, STML_EINVAL, "ctx is NULL");
    c->net = net;
    c->pred_learned = -1;
    return STML_OK;
}

stml_status stml_register_batch(stml_ctx* const* ctxs, int n_ctx, stml_mode mode, int max_threads,
                                stml_status* status) {
    if (!ctxs || n_ctx < 1) return fail(nullptr, STML_EINVAL, "stml_register_batch: need contexts");
    for (int i = 0; i < n_ctx; ++i) {
        const stml_ctx* c = ctxs[i];
        if (!c) return fail(nullptr, STML_EINVAL, "stml_register_batch: a context is NULL");
        if (!c->built) return fail(nullptr, STML_ESTATE, "stml_register_batch: a context has no pyramid");
        if (c->p.pcg_cooperative)
            return fail(nullptr, STML_EINVAL, "stml_register_batch: contexts need pcg_cooperative = 0");
        for (int k = 0; k < i; ++k) {
            if (ctxs[k] == c || (c->stream && ctxs[k]->stream == c->stream))
                return fail(nullptr, STML_EINVAL, "stml_register_batch: contexts share a stream");
            if (c->net && ctxs[k]->net == c->net)
                return fail(nullptr, STML_EINVAL, "stml_register_batch: contexts share a predictor network");
        }
    }
    if (mode != STML_MODE_STML && mode != STML_MODE_SPML) return fail(nullptr, STML_EINVAL, "unknown mode");
    const int nt = std::max(1, std::min(n_ctx, max_threads > 0 ? max_threads : n_ctx));
    std::vector<stml_status> st(n_ctx, STML_OK);
    std::atomic<int> next{0};
    auto worker = [&]() {
        for (int i = next.fetch_add(1); i < n_ctx; i = next.fetch_add(1))
            st[i] = stml_register(ctxs[i], mode, nullptr, 0, nullptr);
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
    worker();
    for (auto& th : pool) th.join();
    stml_status first = STML_OK;
    for (int i = 0; i < n_ctx; ++i) {
        if (status) status[i] = st[i];
        if (first == STML_OK && st[i] != STML_OK) first = st[i];
    }
    return first;
}

stml_status stml_eval(stml_ctx* c, int level, const int* frames, int nK, const float* u, double* out,
                      float* g, float* dT) {
    if (!c) return fail(nullptr, STML_EINVAL, "ctx is NULL");
    TRY(check_level(c, level));
    TRY(check_frames(c, frames, nK));
    if (!u || !out) return fail(c, STML_EINVAL, "u and out are required");
    TRY(check_aligned(c, {u, g, dT}));
    cudaSetDevice(c->device);
    LevelBuf& L = c->lv[level];
    std::vector<int> K(frames, frames + nK);
    FrameSet fs;
    TRY(upload_frameset(c, K, fs));
    const Coef cf = make_coef(L.g, c->p, nK);
    const bool full = g || dT;
    const double pfK = (double)nK * L.g.N;
    long pe = prof_begin(c, PC_TRIAL, level);
    CK(c, launch_objective(Stored{L.img, c->img_type}, L.g, fs, cf, u, nullptr, 0.f, nullptr, c->w_abar, c->w_ubar, c->partials,
                           c->partials_cap, &c->S->ticket[0], c->S->red, c->stream));
    const double bS = (double)store_bytes(c->img_type);
    prof_end(c, pe, pfK * (bS + 4.0 * L.g.d), pfK);
    if (full) {
        pe = prof_begin(c, PC_EVAL, level);
        CK(c, launch_gradient(Stored{L.img, c->img_type}, L.g, fs, cf, u, nullptr, 0.f, c->w_abar, c->w_ubar,
                              g ? g : c->w_g, dT ? dT : c->w_dT, ST_F32, nullptr, c->partials, c->partials_cap, &c->S->ticket[4], c->S->red,
                              c->stream));
        prof_end(c, pe, pfK * (bS + 20.0 * L.g.d), pfK);
    }
    TRY(read_scalars(c));
    for (int i = 0; i < 6; ++i) out[i] = c->Sh->red[i];
    if (!full) out[4] = 0.0;
    return STML_OK;
}

stml_status stml_eval_trial(stml_ctx* c, int level, const int* frames, int nK, const float* u, const float* d,
                            double t, const float* gd, double* out) {
    if (!c) return fail(nullptr, STML_EINVAL, "ctx is NULL");
    TRY(check_level(c, level));
    TRY(check_frames(c, frames, nK));
    if (!u || !d || !out) return fail(c, STML_EINVAL, "u, d and out are required");
    TRY(check_aligned(c, {u, d, gd}));
    cudaSetDevice(c->device);
    LevelBuf& L = c->lv[level];
    std::vector<int> K(frames, frames + nK);
    FrameSet fs;
    TRY(upload_frameset(c, K, fs));
    const Coef cf = make_coef(L.g, c->p, nK);
    const double pfK = (double)nK * L.g.N;
    const double bS = (double)store_bytes(c->img_type);
    const long pe = prof_begin(c, PC_TRIAL, level);
    const ObjShapeChoice* sh = obj_choice(c, level, L.g, fs, cf, Stored{L.img, c->img_type}, u, d, (float)t, gd,
                                          gd ? 2 : 1);
    CK(c, launch_objective(Stored{L.img, c->img_type}, L.g, fs, cf, u, d, (float)t, gd, c->w_abar, c->w_ubar,
                           c->partials, c->partials_cap, &c->S->ticket[0], c->S->trial, c->stream, nullptr, sh));
    prof_end(c, pe, pfK * (bS + (gd ? 16.0 : 8.0) * L.g.d), pfK);
    TRY(read_scalars(c));
    for (int i = 0; i < 8; ++i) out[i] = c->Sh->trial[i];
    if (!gd) out[6] = out[7] = 0.0;
    out[4] = 0.0;
    return STML_OK;
}

stml_status stml_hessvec(stml_ctx* c, int level, const int* frames, int nK, const float* dT, const float* v,
                         float* Hv, double* vHv) {
    if (!c) return fail(nullptr, STML_EINVAL, "ctx is NULL");
    TRY(check_level(c, level));
    TRY(check_frames(c, frames, nK));
    if (!dT || !v || !Hv) return fail(c, STML_EINVAL, "dT, v and Hv are required");
    TRY(check_aligned(c, {dT, v, Hv}));
    cudaSetDevice(c->device);
    LevelBuf& L = c->lv[level];
    std::vector<int> K(frames, frames + nK);
    FrameSet fs;
    TRY(upload_frameset(c, K, fs));
    const Coef cf = make_coef(L.g, c->p, nK);
    TRY(hessvec_launch(c, level, L.g, fs, cf, dT, v, Hv, nullptr));
    TRY(read_scalars(c));
    if (vHv) *vHv = c->Sh->dots[4];
    return STML_OK;
}

stml_status stml_gir(stml_ctx* c, int level, const int* frames, int nK, float* u, stml_stats* stats) {
    if (!c) return fail(nullptr, STML_EINVAL, "ctx is NULL");
    TRY(check_level(c, level));
    TRY(check_frames(c, frames, nK));
    if (!u) return fail(c, STML_EINVAL, "u is required");
    TRY(check_aligned(c, {u}));
    cudaSetDevice(c->device);
    std::vector<int> K(frames, frames + nK);
    return run_gir(c, level, K, u, stats, c->p.target_J);
}

stml_status stml_eval_ugrid(stml_ctx* c, int level, const int* frames, int nK, const float* w, double* out,
                            float* g, float* dT, float* Minv) {
    if (!c) return fail(nullptr, STML_EINVAL, "ctx is NULL");
    if (c->p.u_coarsen < 1) return fail(c, STML_EINVAL, "stml_eval_ugrid needs params.u_coarsen > 0");
    TRY(check_level(c, level));
    TRY(check_frames(c, frames, nK));
    if (!w || !out) return fail(c, STML_EINVAL, "w and out are required");
    cudaSetDevice(c->device);
    std::vector<int> K(frames, frames + nK);
    UgEval E;
    TRY(ug_setup(c, level, K, E));
    const bool grad = g || dT || Minv;
    TRY(E.run(w, nullptr, 0.f, grad, out));
    const size_t Mc = (size_t)E.planes * E.gw.N, Mf = (size_t)E.planes * E.g.N;
    if (g) CK(c, cudaMemcpyAsync(g, c->ug_g, Mc * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
    if (dT) CK(c, cudaMemcpyAsync(dT, c->w_dT, Mf * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
    if (Minv) {
        TRY(E.jacobi());
        CK(c, cudaMemcpyAsync(Minv, c->ug_m, Mc * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
    }
    CK(c, cudaStreamSynchronize(c->stream));
    return STML_OK;
}

stml_status stml_hessvec_ugrid(stml_ctx* c, int level, const int* frames, int nK, const float* dT, const float* v,
                               float* Hv, double* vHv) {
    if (!c) return fail(nullptr, STML_EINVAL, "ctx is NULL");
    if (c->p.u_coarsen < 1) return fail(c, STML_EINVAL, "stml_hessvec_ugrid needs params.u_coarsen > 0");
    TRY(check_level(c, level));
    TRY(check_frames(c, frames, nK));
    if (!dT || !v || !Hv || v == Hv) return fail(c, STML_EINVAL, "dT, v and Hv (distinct from v) are required");
    cudaSetDevice(c->device);
    std::vector<int> K(frames, frames + nK);
    UgEval E;
    TRY(ug_setup(c, level, K, E));
    CK(c, cudaMemcpyAsync(c->w_dT, dT, (size_t)E.planes * E.g.N * sizeof(float), cudaMemcpyDeviceToDevice,
                          c->stream));
    double pq = 0.0;
    TRY(E.hess(v, Hv, &pq));
    if (vHv) *vHv = pq;
    return STML_OK;
}

stml_status stml_eval_affine(stml_ctx* c, int level, const int* frames, int nK, const double* theta, double* out,
                             double* grad) {
    if (!c) return fail(nullptr, STML_EINVAL, "ctx is NULL");
    TRY(check_level(c, level));
    TRY(check_frames(c, frames, nK));
    if (!theta || !out) return fail(c, STML_EINVAL, "theta and out are required");
    cudaSetDevice(c->device);
    std::vector<int> K(frames, frames + nK);
    FrameSet fs;
    TRY(upload_frameset(c, K, fs));
    return affine_eval(c, level, K, fs, theta, out, grad);
}

stml_status stml_affine_field(stml_ctx* c, int level, const int* frames, int nK, const double* theta, float* u) {
    if (!c) return fail(nullptr, STML_EINVAL, "ctx is NULL");
    TRY(check_level(c, level));
    TRY(check_frames(c, frames, nK));
    if (!theta || !u) return fail(c, STML_EINVAL, "theta and u are required");
    TRY(check_aligned(c, {u}));
    cudaSetDevice(c->device);
    TRY(affine_fields(c, level, theta, nK, u));
    CK(c, cudaStreamSynchronize(c->stream));
    return STML_OK;
}

stml_status stml_gir_affine(stml_ctx* c, int level, const int* frames, int nK, double* theta_io,
                            stml_stats* stats) {
    if (!c) return fail(nullptr, STML_EINVAL, "ctx is NULL");
    TRY(check_level(c, level));
    TRY(check_frames(c, frames, nK));
    if (!theta_io) return fail(c, STML_EINVAL, "theta_io is required");
    cudaSetDevice(c->device);
    std::vector<int> K(frames, frames + nK);
    return run_gir_affine(c, level, K, theta_io, stats);
}

stml_status stml_get_affine(const stml_ctx* c, double* theta, size_t cap) {
    if (!c) return fail(nullptr, STML_EINVAL, "ctx is NULL");
    if (c->theta.empty()) return fail(const_cast<stml_ctx*>(c), STML_ESTATE, "no affine registration yet");
    if (!theta || cap < c->theta.size()) return fail(const_cast<stml_ctx*>(c), STML_EINVAL, "theta too small");
    std::memcpy(theta, c->theta.data(), sizeof(double) * c->theta.size());
    return STML_OK;
}

stml_status stml_corr_coeff(stml_ctx* c, int level, double* rho) {
    if (!c) return fail(nullptr, STML_EINVAL, "ctx is NULL");
    TRY(check_level(c, level));
    if (!rho) return fail(c, STML_EINVAL, "rho is required");
    cudaSetDevice(c->device);
    if (c->n < 2) return STML_OK;
    CK(c, launch_corr_coeff(c->lv[level].img, c->img_type, c->n, c->lv[level].g.N, c->d_rho, c->stream));
    CK(c, cudaMemcpyAsync(rho, c->d_rho, (size_t)(c->n - 1) * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return STML_OK;
}

// ------------------------------------------------------ context-free operators
// A valid 2-D / 3-D shape whose image, and its 2x refinement, has at most
// 2^31 - 1 cells (pixel indices are 32-bit).
static bool shape_ok(int dim, const int* shape, int sh3[3]) {
    if ((dim != 2 && dim != 3) || !shape) return false;
    sh3[0] = 1;
    long long cells = 1LL << dim;
    for (int i = 0; i < dim; ++i) {
        if (shape[i] < 1 || shape[i] > 65535) return false;
        sh3[3 - dim + i] = shape[i];
        cells *= shape[i];
    }
    return cells <= 0x7fffffffLL;
}

stml_status stml_restrict(const float* fine, float* coarse, int planes, int dim, const int* fine_shape,
                          void* cuda_stream) {
    int sh3[3];
    if (!fine || !coarse || planes < 0 || !shape_ok(dim, fine_shape, sh3))
        return fail(nullptr, STML_EINVAL, "stml_restrict: bad arguments");
    for (int i = 3 - dim; i < 3; ++i) {
        if (sh3[i] % 2) return fail(nullptr, STML_EINVAL, "stml_restrict: odd axis");
        sh3[i] /= 2;
    }
    const Geom gc = make_geom(sh3, dim, 2.f);
    cudaError_t e = launch_restrict(fine, coarse, ST_F32, planes, gc, (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? STML_OK : cuda_fail(nullptr, e, "stml_restrict");
}

stml_status stml_prolong(const float* coarse, float* fine, int planes, int dim, const int* coarse_shape,
                         void* cuda_stream) {
    int sh3[3];
    if (!fine || !coarse || planes < 0 || !shape_ok(dim, coarse_shape, sh3))
        return fail(nullptr, STML_EINVAL, "stml_prolong: bad arguments");
    const Geom gc = make_geom(sh3, dim, 2.f);
    cudaError_t e = launch_prolong(coarse, fine, planes, gc, (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? STML_OK : cuda_fail(nullptr, e, "stml_prolong");
}

stml_status stml_prolong_adjoint(const float* fine, float* coarse, int planes, int dim, const int* coarse_shape,
                                 void* cuda_stream) {
    int sh3[3];
    if (!fine || !coarse || planes < 0 || !shape_ok(dim, coarse_shape, sh3))
        return fail(nullptr, STML_EINVAL, "stml_prolong_adjoint: bad arguments");
    const Geom gc = make_geom(sh3, dim, 2.f);
    cudaError_t e = launch_prolong_adjoint(fine, coarse, planes, gc, (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? STML_OK : cuda_fail(nullptr, e, "stml_prolong_adjoint");
}

static stml_status ugrid_args(const char* who, const float* a, const float* b, int planes, int dim,
                              const int* fine_shape, int s, UGrid& ug) {
    int sh3[3];
    if (!a || !b || planes < 0 || s < 1 || s > 4 || !shape_ok(dim, fine_shape, sh3))
        return fail(nullptr, STML_EINVAL, std::string(who) + ": bad arguments");
    for (int i = 3 - dim; i < 3; ++i)
        if (sh3[i] % (1 << s)) return fail(nullptr, STML_EINVAL, std::string(who) + ": an axis is not a multiple of 2^s");
    ug = make_ugrid(make_geom(sh3, dim, 1.f), s);
    return STML_OK;
}

stml_status stml_ugrid_prolong(const float* w, float* u, int planes, int dim, const int* fine_shape, int s,
                               void* cuda_stream) {
    UGrid ug;
    TRY(ugrid_args("stml_ugrid_prolong", w, u, planes, dim, fine_shape, s, ug));
    cudaError_t e = launch_ugrid_prolong(w, nullptr, 0.f, u, planes, ug, (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? STML_OK : cuda_fail(nullptr, e, "stml_ugrid_prolong");
}

stml_status stml_ugrid_adjoint(const float* u, float* w, int planes, int dim, const int* fine_shape, int s,
                               void* cuda_stream) {
    UGrid ug;
    TRY(ugrid_args("stml_ugrid_adjoint", u, w, planes, dim, fine_shape, s, ug));
    cudaError_t e = launch_ugrid_adjoint(u, w, planes, ug, (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? STML_OK : cuda_fail(nullptr, e, "stml_ugrid_adjoint");
}

static bool increasing(const int* K, int nK) {
    for (int i = 1; i < nK; ++i)
        if (K[i] <= K[i - 1]) return false;
    return true;
}

stml_status stml_predict_linear(const float* yK, const int* K, int nK, float* z, const int* targets, int nT,
                                size_t plane_elems, void* cuda_stream) {
    if (!yK || !K || !z || !targets || nK < 1 || nT < 0 || !increasing(K, nK))
        return fail(nullptr, STML_EINVAL, "stml_predict_linear: bad arguments");
    std::vector<int> Kv(K, K + nK), tv(targets, targets + nT);
    for (int t : tv)
        if (t < Kv.front() || t > Kv.back())
            return fail(nullptr, STML_EINVAL, "stml_predict_linear: target outside the span of K");
    std::vector<LinTap> taps = linear_taps(Kv, tv, false);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    LinTap* d_taps = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&d_taps, std::max<size_t>(1, taps.size()) * sizeof(LinTap), s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_taps, taps.data(), taps.size() * sizeof(LinTap), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_predict_linear(yK, z, d_taps, nT, plane_elems, s);
    if (d_taps) cudaFreeAsync(d_taps, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? STML_OK : cuda_fail(nullptr, e, "stml_predict_linear");
}

stml_status stml_predict_ls(const float* eta, const int* K, int nK, const float* omega, float* zeta, int n,
                            double beta, size_t n_comp, void* cuda_stream) {
    if (!eta || !K || !omega || !zeta || n < 1 || nK < 1 || nK > n || !(beta >= 0) || !increasing(K, nK) ||
        K[0] < 0 || K[nK - 1] >= n)
        return fail(nullptr, STML_EINVAL, "stml_predict_ls: bad arguments");
    if (omega == zeta) return fail(nullptr, STML_EINVAL, "stml_predict_ls: omega and zeta must differ");
    std::vector<int> Kv(K, K + nK), kidx;
    std::vector<float> tab;
    ls_factors(n, Kv, beta, tab, kidx);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    float* d_tab = nullptr;
    int* d_k = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&d_tab, tab.size() * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&d_k, kidx.size() * sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_tab, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_k, kidx.data(), kidx.size() * sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_predict_ls(eta, omega, zeta, d_tab, d_tab + n, d_tab + 2 * n, d_k, n, n_comp, s);
    if (d_tab) cudaFreeAsync(d_tab, s);
    if (d_k) cudaFreeAsync(d_k, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? STML_OK : cuda_fail(nullptr, e, "stml_predict_ls");
}

// ------------------------------------------------------------ profiling
stml_status stml_profile_enable(stml_ctx* c, int enable) {
    if (!c) return fail(nullptr, STML_EINVAL, "ctx is NULL");
    c->prof = enable != 0;
    c->prof_hess_only = enable == 2;
    c->ev_used = 0;
    c->pacc.clear();
    return STML_OK;
}

stml_status stml_profile_read(stml_ctx* c, long long* launches, double* ms, double* bytes, double* pixel_frames) {
    if (!c) return fail(nullptr, STML_EINVAL, "ctx is NULL");
    cudaSetDevice(c->device);
    CK(c, cudaStreamSynchronize(c->stream));
    double tot = 0.0, by = 0.0, pf = 0.0;
    long long nl = 0;
    for (size_t i = 0; i < c->ev_used; ++i) {
        if (c->ev[i].key / 64 != PC_HESS) continue;
        float m = 0.f;
        CK(c, cudaEventElapsedTime(&m, c->ev[i].a, c->ev[i].b));
        tot += m;
        ++nl;
    }
    for (const auto& kv : c->pacc)
        if (kv.first / 64 == PC_HESS) {
            by += kv.second[1];
            pf += kv.second[2];
        }
    if (launches) *launches = nl;
    if (ms) *ms = tot;
    if (bytes) *bytes = by;
    if (pixel_frames) *pixel_frames = pf;
    return STML_OK;
}

stml_status stml_profile_report(stml_ctx* c, char* buf, size_t cap, size_t* needed) {
    if (!c) return fail(nullptr, STML_EINVAL, "ctx is NULL");
    cudaSetDevice(c->device);
    CK(c, cudaStreamSynchronize(c->stream));
    std::map<int, double> ms;
    for (size_t i = 0; i < c->ev_used; ++i) {
        float m = 0.f;
        CK(c, cudaEventElapsedTime(&m, c->ev[i].a, c->ev[i].b));
        ms[c->ev[i].key] += m;
    }
    std::string out = "[";
    bool first = true;
    char line[256];
    for (const auto& kv : c->pacc) {
        const int cls = kv.first / 64, lvl = kv.first % 64;
        std::snprintf(line, sizeof(line),
                      "%s{\"kernel\": \"%s\", \"level\": %d, \"launches\": %.0f, \"ms\": %.6f, "
                      "\"bytes\": %.6g, \"pixel_frames\": %.6g}",
                      first ? "" : ", ", kProfNames[cls], lvl, kv.second[0], ms[kv.first], kv.second[1],
                      kv.second[2]);
        out += line;
        first = false;
    }
    out += "]";
    if (needed) *needed = out.size() + 1;
    if (buf && cap > 0) {
        const size_t n = std::min(cap - 1, out.size());
        std::memcpy(buf, out.data(), n);
        buf[n] = 0;
    }
    return STML_OK;
}

stml_status stml_tuning_report(const stml_ctx* c, char* buf, size_t cap, size_t* needed) {
    if (!c) return fail(nullptr, STML_EINVAL, "ctx is NULL");
    std::string out = "[";
    char line[256];
    bool first = true;
    for (const auto& kv : c->obj_tuned) {
        std::snprintf(line, sizeof(line),
                      "%s{\"what\": \"objective_shape\", \"level\": %d, \"frames\": %d, \"variant\": %d, "
                      "\"vec\": %d, \"splits\": %d}",
                      first ? "" : ", ", kv.first[0], kv.first[1], kv.first[2], kv.second.vec, kv.second.splits);
        out += line;
        first = false;
    }
    for (const auto& kv : c->coop_tuned) {
        std::snprintf(line, sizeof(line), "%s{\"what\": \"pcg_path\", \"level\": %d, \"frames\": %d, \"cooperative\": %d}",
                      first ? "" : ", ", kv.first[0], kv.first[1], kv.second);
        out += line;
        first = false;
    }
    out += "]";
    if (needed) *needed = out.size() + 1;
    if (buf && cap > 0) {
        const size_t k = std::min(cap - 1, out.size());
        std::memcpy(buf, out.data(), k);
        buf[k] = 0;
    }
    return STML_OK;
}

long long stml_launch_count(const stml_ctx* c) {
    (void)c;
    return launches_total();
}


stml_status stml_batch_create(stml_ctx* const* ctxs, int n_ctx, stml_batch** out) {
    if (!out) return fail(nullptr, STML_EINVAL, "stml_batch_create: out is NULL");
    *out = nullptr;
    if (!ctxs || n_ctx < 1) return fail(nullptr, STML_EINVAL, "stml_batch_create: need contexts");
    for (int i = 0; i < n_ctx; ++i) {
        if (!ctxs[i]) return fail(nullptr, STML_EINVAL, "stml_batch_create: a context is NULL");
        for (int k = 0; k < i; ++k)
            if (ctxs[k] == ctxs[i]) return fail(nullptr, STML_EINVAL, "stml_batch_create: a context appears twice");
        if (ctxs[i]->device != ctxs[0]->device)
            return fail(nullptr, STML_EINVAL, "stml_batch_create: contexts on several devices");
        if (ctxs[i]->net)
            for (int k = 0; k < i; ++k)
                if (ctxs[k]->net == ctxs[i]->net)
                    return fail(nullptr, STML_EINVAL, "stml_batch_create: contexts share a predictor network");
    }
    stml_batch* b = new stml_batch();
    b->ctxs.assign(ctxs, ctxs + n_ctx);
    b->device = ctxs[0]->device;
    cudaSetDevice(b->device);
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev_a);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev_b);
    b->ev_ready.assign(n_ctx, nullptr);
    for (int i = 0; i < n_ctx && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&b->ev_ready[i], cudaEventDisableTiming);
    const int sms = device_sms();
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_part, batch_partials(2 * (sms > 0 ? sms : 152)) * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_sync, sizeof(BatchSync));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_sync, sizeof(BatchSync));
    if (e != cudaSuccess) {
        const std::string msg = std::string("stml_batch_create: ") + cudaGetErrorString(e);
        batch_free(b);
        return fail(nullptr, e == cudaErrorMemoryAllocation ? STML_ENOMEM : STML_ECUDA, msg);
    }
    std::memset(b->h_sync, 0, sizeof(BatchSync));
    *out = b;
    return STML_OK;
}

stml_status stml_batch_register(stml_batch* b, stml_mode mode, stml_status* status) {
    if (!b) return fail(nullptr, STML_EINVAL, "batch is NULL");
    if (mode != STML_MODE_STML && mode != STML_MODE_SPML) return bfail(b, STML_EINVAL, "unknown mode");
    cudaSetDevice(b->device);
    return batch_register(b, mode, status);
}

stml_status stml_batch_report(const stml_batch* b, char* buf, size_t cap, size_t* needed) {
    if (!b) return fail(nullptr, STML_EINVAL, "batch is NULL");
    if (needed) *needed = b->report.size() + 1;
    if (buf && cap > 0) {
        const size_t k = std::min(cap - 1, b->report.size());
        std::memcpy(buf, b->report.data(), k);
        buf[k] = 0;
    }
    return STML_OK;
}

const char* stml_batch_last_error(const stml_batch* b) { return b ? b->err.c_str() : g_free_error.c_str(); }

void stml_batch_destroy(stml_batch* b) { batch_free(b); }

stml_status stml_check_batch_barrier(void* cuda_stream, int* expired) {
    if (!expired) return fail(nullptr, STML_EINVAL, "expired is NULL");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    BatchSync* sync = nullptr;
    int* flag = nullptr;
    cudaError_t e = cudaMalloc((void**)&sync, sizeof(BatchSync));
    if (e == cudaSuccess) e = cudaMalloc((void**)&flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, sizeof(int), st);
    if (e == cudaSuccess) e = launch_batch_barrier_probe(sync, flag, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(expired, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (sync) cudaFree(sync);
    if (flag) cudaFree(flag);
    if (e != cudaSuccess) return fail(nullptr, STML_ECUDA, std::string("stml_check_batch_barrier: ") + cudaGetErrorString(e));
    return STML_OK;
}

stml_status stml_last_stats(const stml_ctx* c, stml_stats* stats, int cap, int* n_written) {
    if (!c) return fail(nullptr, STML_EINVAL, "ctx is NULL");
    const int n = (int)c->last_stats.size();
    for (int i = 0; i < n && stats && i < cap; ++i) stats[i] = c->last_stats[i];
    if (n_written) *n_written = n;
    return STML_OK;
}

}  // extern "C"
