// Gauss-Newton Hessian product for a given v (the stml_hessvec building block):
// the per-pixel frame sums of v (tile_kernel, TILE_SUMS) followed by the
// stencil stream (apply_kernel), both in k_gn.cu.  Inside the PCG loop the
// sums come from the update pass (those of z) and the previous direction, so
// only the stencil stream runs there (launch_pcg_apply).
#include "kernels.h"

namespace stml {

cudaError_t launch_hessvec(const Geom& g, const FrameSet& fs, const Coef& cf, const float* dT,
                           const float* v, float* Hv, HessWork& w, unsigned int* ticket,
                           double* out, DevScalars* pcg, cudaStream_t s) {
    if (fs.nK <= 0) return cudaErrorInvalidValue;
    // a PCG step (pcg given) does nothing once the solve has stopped
    cudaError_t e = launch_hess_sums(g, fs, dT, v, w.mean_s, w.sum_v, s, pcg ? &pcg->cg_active : nullptr);
    if (e != cudaSuccess) return e;
    return launch_hess_apply(g, fs, cf, dT, v, w.mean_s, w.sum_v, Hv, w.partials, w.partials_cap, ticket, out, pcg, s);
}

}  // namespace stml
