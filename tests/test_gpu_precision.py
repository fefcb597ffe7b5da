"""Per-result error of the reductions on a large, near-converged level.

The objective terms, the PCG inner products and the Armijo test are reduced
in double-float arithmetic (about 44 significant bits from FP32 instructions)
with FP32 leaves and FP32 CG coefficients, not in FP64.  Near convergence the
per-pixel residuals a_k - mean_j a_j are small against the warped values, so
this is where cancellation would show.  Workload: the paper-scale sequence
(200 frames of 256 x 256) registered by STML; at the registered fields of the
finest level (13.1 M pixel-frames) J, D, S, P and <v, Hv> are compared with
FP64 sums of the FP64 oracle evaluated at the same FP32 fields."""
import numpy as np
import pytest

from _util import cuda_lib
from oracle import Params, objective
from paper_2001_06613_gb300 import synthetic

pytestmark = pytest.mark.gpu

# bounds: FP32 leaves (unit roundoff 6e-8 over ~30 operations per element)
# summed in double-float; P, the penalty of the mean field, is small near
# the registered fields and carries less relative accuracy
TOL = {"J": 1e-6, "D": 1e-6, "S": 1e-6, "P": 1e-4, "vHv": 1e-5}


def test_double_float_reductions_against_fp64_at_paper_scale():
    import torch
    S = cuda_lib()
    spec = synthetic.spec_paper_scale()
    R = synthetic.make_sequence(spec)
    n, L = R.shape[0], 4
    prm = S.stml_default_params(n_levels=L, n_tlevels=3)
    ctx = S.Context(prm)
    try:
        S.stml_load_sequence(ctx.ptr, torch.from_numpy(R).cuda())
        S.stml_build_pyramid(ctx.ptr)
        S.stml_register(ctx.ptr, S.MODE_STML)
        y = torch.empty((n, 2, 256, 256), device="cuda")
        S.stml_get_field(ctx.ptr, L - 1, y)
        frames = list(range(n))
        g = torch.empty_like(y)
        dT = torch.empty_like(y)
        out = S.stml_eval(ctx.ptr, L - 1, frames, y, g, dT)
        rng = np.random.default_rng(3)
        v = synthetic.random_field(rng, n, 2, (256, 256), amp=0.1, rough=0.2)
        Hv = torch.empty_like(y)
        vhv = S.stml_hessvec(ctx.ptr, L - 1, frames, dT, torch.from_numpy(v).cuda(), Hv)
    finally:
        ctx.close()
    op = Params(alpha=prm.alpha, lam=prm.lambda_)
    y64 = y.cpu().numpy().astype(np.float64)
    ev = objective.evaluate(R.astype(np.float64), y64, frames, 1.0, op, want_grad=False)
    got = {"J": out[0], "D": out[1], "S": out[2], "P": out[3]}
    errs = {k: abs(got[k] - ev[k]) / abs(ev[k]) for k in got}
    Hv_ref = objective.hessvec(dT.cpu().numpy().astype(np.float64), v.astype(np.float64), frames, 1.0, op)
    vhv_ref = float(np.sum(v.astype(np.float64) * Hv_ref))
    errs["vHv"] = abs(vhv - vhv_ref) / abs(vhv_ref)
    print("\nrelative error against FP64 sums at the registered paper-scale fields: " +
          ", ".join(f"{k} {e:.2e}" for k, e in errs.items()))
    for k, e in errs.items():
        assert e <= TOL[k], (k, e)
