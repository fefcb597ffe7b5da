"""Affine-linear / L-BFGS variant on the GPU against the FP64 oracle
(oracle/affine.py): affine fields, objective and parameter gradient, one
L-BFGS GIR, and whole STML / SpML registrations that recover a planted
affine motion."""
import numpy as np
import pytest

from _util import assert_scalar, cuda_lib
from oracle import Params, affine, grid
from oracle.multilevel import pyramid
from paper_2001_06613_gb300 import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    return cuda_lib()


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _ctx(S, R, levels, **kw):
    prm = S.stml_default_params(n_levels=levels, transform=1, **kw)
    ctx = S.Context(prm)
    S.stml_load_sequence(ctx.ptr, _dev(R))
    S.stml_build_pyramid(ctx.ptr)
    return ctx


def _op(prm, **kw):
    return Params(alpha=prm.alpha, alpha_t=prm.alpha_t, lam=prm.lambda_, beta=prm.beta, eps_stop=prm.eps_stop,
                  n_levels=prm.n_levels, n_tlevels=prm.n_tlevels, tol_J=prm.tol_J, tol_Y=prm.tol_Y,
                  tol_G=prm.tol_G, g_abs=prm.g_abs, max_ls=prm.max_ls, armijo_c=prm.armijo_c,
                  distance="nc" if prm.distance == 1 else "ssd", **kw)


FIELD_CASES = [((48, 40), 3, 1), ((48, 40), 3, 0), ((12, 16, 20), 2, 1)]


@pytest.mark.parametrize("shape,levels,level", FIELD_CASES)
def test_affine_field_parity(S, shape, levels, level):
    import torch
    R = synthetic.make_sequence(synthetic.spec_custom(4, shape, seed=21, amp=1.0))
    ctx = _ctx(S, R, levels)
    try:
        d = len(shape)
        m = tuple(int(v) for v in S.stml_level_info(ctx.ptr, level)[0][3 - d:])
        h = grid.level_h(levels, level)
        th = np.random.default_rng(22).normal(size=(3, d * (d + 1)))
        u = torch.empty((3, d) + m, device="cuda")
        S.stml_affine_field(ctx.ptr, level, [0, 2, 3], th, u)
        ref = affine.field(th, affine.coords(m, h, shape))
        assert np.abs(u.cpu().numpy() - ref).max() <= 1e-6 * np.abs(ref).max()
    finally:
        ctx.close()


EVAL_CASES = [((48, 40), 5, 2, 1, [0, 1, 2, 3, 4], {}),
              ((48, 40), 5, 2, 0, [0, 2, 4], dict(alpha_t=0.4)),
              ((12, 16, 20), 3, 2, 1, [0, 1, 2], dict(alpha=0.05))]


EVAL_CASES += [(shape, n, levels, level, frames, dict(extra, distance=1))
               for shape, n, levels, level, frames, extra in EVAL_CASES]


@pytest.mark.parametrize("shape,n,levels,level,frames,extra", EVAL_CASES)
def test_eval_affine_parity(S, shape, n, levels, level, frames, extra):
    R = synthetic.make_affine_sequence(synthetic.spec_custom(n, shape, seed=23, amp=0.0), smooth=True)
    ctx = _ctx(S, R, levels, **extra)
    try:
        d = len(shape)
        T = pyramid(R.astype(np.float64), levels)[level]
        h = grid.level_h(levels, level)
        xh = affine.coords(T.shape[1:], h, shape)
        th = 0.4 * np.random.default_rng(24).normal(size=(len(frames), d * (d + 1)))
        out, g = S.stml_eval_affine(ctx.ptr, level, frames, th)
        p = _op(ctx.params)
        ev = affine.evaluate(T[frames], th, frames, h, xh, p)
        for i, k in enumerate(("J", "D", "S", "P")):
            assert_scalar(out[i], ev[k], what=k)
        # FP32 sums of g_u * phi over the grid: error relative to the sum of magnitudes
        evu = affine.objective.evaluate(T[frames], affine.field(th, xh), frames, h, p)
        gu = evu["g"]
        if p.distance == "nc":
            hd = h ** d
            gu = affine.nc_distance(evu["a"])[1][:, None] * evu["dT"] + gu - hd * evu["r"][:, None] * evu["dT"]
        scale = affine.project(np.abs(gu), np.abs(xh))
        assert np.all(np.abs(g - ev["g"]) <= 1e-5 * scale + 1e-12), np.abs(g - ev["g"]).max()
    finally:
        ctx.close()


def test_gir_affine_parity(S):
    """One L-BFGS GIR from the identity: the FP32 evaluations let the iterates
    drift slightly from the FP64 oracle's, so the final objective and the
    parameters are compared."""
    spec = synthetic.spec_custom(5, (48, 40), seed=25, amp=0.0, noise_sd=0.0)
    R = synthetic.make_affine_sequence(spec, smooth=True)
    ctx = _ctx(S, R, 1, alpha=0.0)
    try:
        K = [0, 1, 2, 3, 4]
        th0 = np.zeros((5, 6))
        th, st = S.stml_gir_affine(ctx.ptr, 0, K, th0)
        p = _op(ctx.params)
        T = R.astype(np.float64)
        xh = affine.coords(T.shape[1:], 1.0, T.shape[1:])
        tho, sto = affine.gir(T, th0, K, 1.0, xh, p, m=ctx.params.lbfgs_m, max_it=ctx.params.max_lbfgs)
        Jg = affine.evaluate(T, th, K, 1.0, xh, p, want_grad=False)["J"]
        print(f"\nGIR: GPU {st['gn_iters']} iterations J {st['J']:.6g} (oracle J at GPU theta {Jg:.6g}); "
              f"oracle {sto.iters} iterations J {sto.J:.6g}; max |theta diff| {np.abs(th - tho).max():.3e} px")
        assert_scalar(st["J"], Jg, rtol=1e-4, what="GPU J vs oracle J at the GPU's theta")
        assert abs(Jg - sto.J) <= 2e-2 * sto.J0
        assert np.abs(th - tho).max() <= 0.05
    finally:
        ctx.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_register_recovers_planted_affine_motion(S, mode):
    import torch
    spec = synthetic.spec_custom(9, (48, 40), seed=26, amp=0.0, noise_sd=0.0)
    R = synthetic.make_affine_sequence(spec, smooth=True)
    M, s = synthetic.affine_motion(spec)
    tight = dict(tol_J=1e-9, tol_Y=1e-6, tol_G=1e-6, max_lbfgs=200)
    ctx = _ctx(S, R, 2, n_tlevels=3, alpha=0.0, **tight)
    try:
        stats = S.stml_register(ctx.ptr, mode)
        th = S.stml_get_affine(ctx.ptr, 9, 2)
        y = np.empty((9, 2, 48, 40), np.float32)
        S.stml_get_field(ctx.ptr, 1, y)
        xh = affine.coords((48, 40), 1.0, (48, 40))
        assert np.abs(y - affine.field(th, xh)).max() <= 1e-5 * np.abs(y).max()
        p = _op(ctx.params)
        tho, _ = affine.register(R.astype(np.float64), p, mode="stml" if mode == 0 else "spml", max_it=200)
    finally:
        ctx.close()
    x = grid.cell_centres((48, 40), 1.0)
    c = np.array([24.0, 20.0]).reshape(2, 1, 1)
    yy = x[None] + affine.field(th, xh)
    err = 0.0
    for k in range(1, 9):
        pred = np.tensordot(np.linalg.inv(M[k]), np.tensordot(M[0], yy[0] - c, axes=(1, 0)) +
                            (s[0] - s[k]).reshape(2, 1, 1), axes=(1, 0)) + c
        err = max(err, float(np.abs(yy[k] - pred)[:, 8:-8, 8:-8].max()))
    print(f"\nmode {mode}: {len(stats)} GIRs, L-BFGS iterations {[st['gn_iters'] for st in stats]}; "
          f"misalignment {err:.3f} px; max |theta - oracle theta| {np.abs(th - tho).max():.3e}")
    assert err < 0.05
    assert np.abs(th - tho).max() < 0.05
    del torch


def test_affine_params_are_validated(S):
    with pytest.raises(S.StmlError):
        S.Context(S.stml_default_params(transform=2))
    with pytest.raises(S.StmlError):
        S.Context(S.stml_default_params(transform=1, lbfgs_m=0))
    with pytest.raises(S.StmlError):
        S.Context(S.stml_default_params(transform=0, distance=1))   # correlation only for affine maps
    R = synthetic.make_sequence(synthetic.spec_custom(4, (16, 16), seed=27))
    ctx = _ctx(S, R, 1)
    try:
        with pytest.raises(S.StmlError):
            S.stml_predict(ctx.ptr, 0, 0)
        with pytest.raises(S.StmlError):
            S.stml_get_affine(ctx.ptr, 4, 2)           # nothing registered yet
    finally:
        ctx.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_register_nc_under_changing_contrast(S, mode):
    """Normalised-correlation distance: frames whose brightness and contrast
    change from frame to frame are aligned (the planted affine motion is
    recovered) and the parameters agree with the oracle's."""
    spec = synthetic.spec_custom(5, (48, 40), seed=7, amp=0.0, noise_sd=0.0)
    gain = [1.0, 1.3, 0.8, 1.15, 0.9]
    offset = [0.0, 0.2, -0.1, 0.05, 0.3]
    R = synthetic.make_affine_sequence(spec, smooth=True, gain=gain, offset=offset)
    M, s = synthetic.affine_motion(spec)
    tight = dict(tol_J=1e-12, tol_Y=1e-8, tol_G=1e-8, max_lbfgs=300)
    ctx = _ctx(S, R, 2, n_tlevels=2, alpha=0.0, lam=1e-3, distance=1, **tight)
    try:
        stats = S.stml_register(ctx.ptr, mode)
        th = S.stml_get_affine(ctx.ptr, 5, 2)
        p = _op(ctx.params)
    finally:
        ctx.close()
    tho, _ = affine.register(R.astype(np.float64), p, mode="stml" if mode == 0 else "spml", max_it=300)
    xh = affine.coords((48, 40), 1.0, (48, 40))
    x = grid.cell_centres((48, 40), 1.0)
    c = np.array([24.0, 20.0]).reshape(2, 1, 1)
    yy = x[None] + affine.field(th, xh)
    err = 0.0
    for k in range(1, 5):
        pred = np.tensordot(np.linalg.inv(M[k]), np.tensordot(M[0], yy[0] - c, axes=(1, 0)) +
                            (s[0] - s[k]).reshape(2, 1, 1), axes=(1, 0)) + c
        err = max(err, float(np.abs(yy[k] - pred)[:, 8:-8, 8:-8].max()))
    print(f"\nNC mode {mode}: L-BFGS iterations {[st['gn_iters'] for st in stats]}; misalignment {err:.3f} px; "
          f"max |theta - oracle theta| {np.abs(th - tho).max():.3e}")
    assert err < 0.1
    assert np.abs(th - tho).max() < 0.05
