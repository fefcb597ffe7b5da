"""Helpers shared by the test modules (tolerances, device fixtures)."""
import re
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# FP32 paths against the FP64 oracle: relative 1e-5 on scalars; arrays are
# compared elementwise against 1e-5 of the array's largest magnitude (values
# near zero have no meaningful relative error).
RTOL = 1e-5


def assert_scalar(got, ref, rtol=RTOL, what=""):
    assert abs(got - ref) <= rtol * abs(ref) + 1e-300, f"{what}: got {got!r} ref {ref!r} rel {abs(got-ref)/max(abs(ref),1e-300):.3e}"


def assert_array(got, ref, rtol=RTOL, what=""):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape, f"{what}: shape {got.shape} vs {ref.shape}"
    scale = float(np.abs(ref).max()) if ref.size else 0.0
    err = float(np.abs(got - ref).max()) if ref.size else 0.0
    assert err <= rtol * scale + 1e-30, f"{what}: max abs err {err:.3e} > {rtol:.1e} * {scale:.3e}"


def header_functions():
    import glob
    txt = "".join(open(f).read() for f in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))))
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(stml_[a-z0-9_]+)\s*\(", txt)))


def cuda_lib():
    """Build (if stale) and load the library on a CUDA machine, else skip."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_06613_gb300 import _build
    _build.build()
    import paper_2001_06613_gb300 as S
    S.load()
    return S


# Registration is an iteration whose discrete decisions (CG stops, Armijo
# acceptance, Gauss-Newton stops) compare computed values with thresholds.  A
# decision whose value sits within rounding of its threshold can go either way
# under FP32 arithmetic or another summation order, and both continuations are
# correct results of the method (several correct results: compare what is
# unique, check that the rest is valid).  A CG stopping decision counts as such
# when the oracle's own ratio ||r|| / ||g|| lies within CG_BRANCH_DELTA
# (relative) of tol_cg: FP32 residual recurrences with float CG coefficients
# drift from the FP64 ones by up to a few 1e-3 over a solve.
CG_BRANCH_DELTA = 5e-3


def gir_counts(stats):
    """Per-GIR (level, tlevel, |K|, Gauss-Newton, CG, Armijo) counts of GPU
    stats dicts or oracle LevelStats."""
    out = []
    for s in stats:
        if isinstance(s, dict):
            out.append((s["level"], s["tlevel"], s["n_frames"], s["gn_iters"], s["cg_iters"], s["ls_trials"]))
        else:
            out.append((s.level, s.tlevel, s.n_frames, s.gn_iters, s.cg_iters, s.ls_trials))
    return out


def oracle_branch(register, gpu_counts, tol_cg, max_flips=4):
    """The oracle's registration on the branch the GPU run took.

    ``register(flips)`` runs the oracle (multilevel.register with ``flips``).
    While the oracle's per-GIR counts differ from ``gpu_counts``, the first GIR
    that differs must hold a CG stopping decision of the oracle whose ratio is
    within CG_BRANCH_DELTA of tol_cg; the oracle is rerun with one such
    decision on its other branch (the oracle's own arithmetic throughout; the
    GPU contributes only which of the oracle's near-threshold decisions to
    follow the other way).  Fails when no such decision explains the
    difference.  Returns (oracle result, flips taken)."""
    flips = {}
    res = register(flips)
    for _ in range(max_flips + 1):
        got = gir_counts(res.stats)
        if got == gpu_counts:
            return res, flips
        g = next(i for i in range(min(len(got), len(gpu_counts)) + 1)
                 if i >= len(got) or i >= len(gpu_counts) or got[i] != gpu_counts[i])
        assert g < len(got), f"the GPU ran {len(gpu_counts)} GIRs, the oracle {len(got)}"
        taken = flips.get(g, set())
        cands = [(i, k) for i, rec in enumerate(res.stats[g].cg_residuals) for k, x in enumerate(rec)
                 if abs(x - tol_cg) / tol_cg < CG_BRANCH_DELTA and (i, k) not in taken]
        found = None
        for c in cands:
            trial = {k: set(v) for k, v in flips.items()}
            trial.setdefault(g, set()).add(c)
            alt = register(trial)
            if gir_counts(alt.stats)[:g + 1] == gpu_counts[:g + 1]:
                found = (trial, alt)
                break
        assert found, (f"GIR {g}: oracle counts {got[g]} vs GPU {gpu_counts[g]}; no CG decision of the "
                       f"oracle within {CG_BRANCH_DELTA} of tol_cg explains the difference")
        flips, res = found
    raise AssertionError(f"more than {max_flips} near-threshold decisions went the other way")
