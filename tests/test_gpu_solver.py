"""GPU parity of the Gauss-Newton registration (GIR) and of the STML / SpML
multilevel drivers against the oracle.

Registration is an iteration on a non-convex objective; FP32 device arithmetic
and FP64 oracle arithmetic follow the same algorithm but not the same
rounding, so end-to-end results are compared through the objective and the
fields (with stated tolerances) rather than bit for bit."""
import numpy as np
import pytest

from _util import assert_scalar, cuda_lib, gir_counts, oracle_branch
from oracle import Params, grid, multilevel, solver
from paper_2001_06613_gb300 import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    return cuda_lib()


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _oparams(prm, **kw):
    base = dict(alpha=prm.alpha, alpha_t=prm.alpha_t, lam=prm.lambda_, beta=prm.beta,
                eps_stop=prm.eps_stop, stop_rule=bool(prm.stop_rule), n_levels=prm.n_levels,
                n_tlevels=prm.n_tlevels, tol_J=prm.tol_J, tol_Y=prm.tol_Y, tol_G=prm.tol_G,
                max_gn=prm.max_gn, tol_cg=prm.tol_cg, max_cg=prm.max_cg, max_ls=prm.max_ls,
                armijo_c=prm.armijo_c, g_abs=prm.g_abs, target_J=prm.target_J, target_tol=prm.target_tol)
    base.update(kw)
    return Params(**base)


def _ctx(S, R, **kw):
    prm = S.stml_default_params(**kw)
    ctx = S.Context(prm)
    S.stml_load_sequence(ctx.ptr, _dev(R))
    S.stml_build_pyramid(ctx.ptr)
    return ctx


@pytest.mark.parametrize("max_gn", [1, 3])
def test_gir_matches_oracle_gauss_newton(S, max_gn):
    R = synthetic.make_sequence(synthetic.spec_custom(5, (32, 40), seed=21, amp=1.5))
    ctx = _ctx(S, R, n_levels=1, max_gn=max_gn)
    try:
        frames = [0, 1, 2, 3, 4]
        u0 = np.zeros((5, 2, 32, 40), np.float32)
        ud = _dev(u0)
        st = S.stml_gir(ctx.ptr, 0, frames, ud)
        uo, so = solver.gauss_newton(R.astype(np.float64), u0, frames, 1.0, _oparams(ctx.params))
        # the oracle's CG residual ratios stay >= 1 % away from tol_cg here,
        # so every stopping decision must be the same
        assert st["gn_iters"] == so.gn_iters
        assert st["ls_trials"] == so.ls_trials
        assert st["cg_iters"] == so.cg_iters
        assert_scalar(st["J0"], so.J0, 1e-5, "J0")
        assert_scalar(st["J"], so.J, 1e-5 * max_gn, "J after GN")
        diff = ud.cpu().numpy() - uo
        assert np.sqrt(np.mean(diff ** 2)) <= 1e-4 * max(1.0, np.sqrt(np.mean(uo ** 2)))
    finally:
        ctx.close()


def test_zero_motion_exits_at_iteration_zero(S):
    base = synthetic.make_sequence(synthetic.spec_custom(1, (32, 32), seed=3))
    R = np.repeat(base, 4, axis=0)
    ctx = _ctx(S, R, n_levels=2)
    try:
        u = _dev(np.zeros((4, 2, 32, 32)))
        st = S.stml_gir(ctx.ptr, 1, [0, 1, 2, 3], u)
        assert st["gn_iters"] == 0 and st["cg_iters"] == 0
        assert float(u.abs().max()) == 0.0
    finally:
        ctx.close()


@pytest.fixture(scope="module")
def tiny():
    spec = synthetic.spec_tiny()
    return spec, synthetic.make_sequence(spec)


def _register(S, R, mode, **kw):
    ctx = _ctx(S, R, **kw)
    try:
        stats = S.stml_register(ctx.ptr, mode)
        L = ctx.params.n_levels
        y = np.empty((R.shape[0], R.ndim - 1) + R.shape[1:], np.float32)
        S.stml_get_field(ctx.ptr, L - 1, y)
        return stats, y, ctx.params
    finally:
        ctx.close()


def _centred_rms(y, truth):
    a = y - y.mean(axis=0, keepdims=True)
    b = truth - truth.mean(axis=0, keepdims=True)
    e = (a - b)[..., 4:-4, 4:-4]
    return float(np.sqrt((e ** 2).sum(axis=1).mean()))


# End-to-end contract (per-call quantities are compared at 1e-5 elsewhere):
# final objective within 1e-4 relative, fields within 1e-3 px RMS.  Measured
# on GB300: 2-D registrations agree to 1e-8 in J and 1e-7 px, 3-D ones to 2e-6
# and 4e-5 px, with identical Gauss-Newton, CG and Armijo counts.
E2E_J, E2E_RMS = 1e-4, 1e-3


def _counts(stats, res):
    return gir_counts(stats), gir_counts(res.stats)


def _oracle(R, op, mode, stats):
    """The oracle's registration of R on the branch the GPU run took (the
    natural one unless a CG decision of the oracle sits within rounding of
    tol_cg, see _util.oracle_branch)."""
    res, _ = oracle_branch(lambda fl: multilevel.register(R.astype(np.float64), op, mode, flips=fl),
                           gir_counts(stats), op.tol_cg)
    return res


@pytest.mark.parametrize("mode,coop", [(0, 1), (1, 1), (0, 0), (1, 0)])
def test_register_tiny_matches_oracle(S, tiny, mode, coop):
    """16 frames of 64x64, 2 spatial x 2 temporal levels (STML) or spatial
    only (SpML), with the cooperative or the streaming PCG solve."""
    spec, R = tiny
    stats, y, prm = _register(S, R, mode, n_levels=2, n_tlevels=2, pcg_cooperative=coop)
    op = _oparams(prm)
    res = _oracle(R, op, "stml" if mode == 0 else "spml", stats)
    got, want = _counts(stats, res)
    assert got == want
    Jg = multilevel.final_objective(R.astype(np.float64), y.astype(np.float64), op)["J"]
    Jo = multilevel.final_objective(R.astype(np.float64), res.y, op)["J"]
    assert abs(Jg - Jo) <= E2E_J * Jo, (Jg, Jo)
    rms = float(np.sqrt(np.mean((y - res.y) ** 2)))
    assert rms <= E2E_RMS, rms
    truth = synthetic.planted_registration(spec)
    assert _centred_rms(y.astype(np.float64), truth) < 0.2


@pytest.mark.parametrize("mode", [0, 1])
def test_target_objective_lands_like_the_oracle(S, tiny, mode):
    """params.target_J: the last GIR over all frames stops where J reaches the
    target (its crossing step shortened by regula falsi); the GPU run and the
    oracle take the same steps and both end within target_tol of the target."""
    spec, R = tiny
    free, _, _ = _register(S, R, mode, n_levels=2, n_tlevels=2)
    last = free[-1]
    assert last["gn_iters"] >= 3
    target = 0.5 * (last["J0"] + last["J"])          # crossed inside the last GIR
    stats, y, prm = _register(S, R, mode, n_levels=2, n_tlevels=2, target_J=target)
    op = _oparams(prm)
    res = multilevel.register(R.astype(np.float64), op, "stml" if mode == 0 else "spml")
    got, want = _counts(stats, res)
    assert got == want
    assert stats[-1]["gn_iters"] < last["gn_iters"]
    Jg = multilevel.final_objective(R.astype(np.float64), y.astype(np.float64), op)["J"]
    Jo = multilevel.final_objective(R.astype(np.float64), res.y, op)["J"]
    assert abs(Jo - target) <= prm.target_tol * target
    assert abs(Jg - target) <= 2 * prm.target_tol * target, (Jg, target)
    assert float(np.sqrt(np.mean((y - res.y) ** 2))) <= E2E_RMS


def test_stepwise_api_equals_register(S, tiny):
    spec, R = tiny
    stats, y_reg, prm = _register(S, R, 0, n_levels=2, n_tlevels=2)
    ctx = _ctx(S, R, n_levels=2, n_tlevels=2)
    try:
        for lvl in range(2):
            for q in range(2):
                S.stml_predict(ctx.ptr, lvl, q)
                st, fin = S.stml_correct(ctx.ptr, lvl, q)
                if fin:
                    break
        y = np.empty_like(y_reg)
        S.stml_get_field(ctx.ptr, 1, y)
        assert np.array_equal(y, y_reg)     # same launches, deterministic reductions
    finally:
        ctx.close()


def test_stopping_rule_fills_from_predictor(S):
    R = synthetic.make_sequence(synthetic.spec_custom(9, (32, 32), seed=3, amp=1.0))
    stats, y, prm = _register(S, R, 0, n_levels=2, n_tlevels=3, eps_stop=10.0)
    assert [(s["level"], s["tlevel"], s["stopped_early"]) for s in stats] == \
        [(0, 0, 0), (0, 1, 1), (1, 0, 0), (1, 1, 1)]
    op = _oparams(prm)
    res = multilevel.register(R.astype(np.float64), op, "stml")
    assert np.all(np.isfinite(y))
    assert float(np.sqrt(np.mean((y - res.y) ** 2))) <= E2E_RMS


def test_single_frame_and_3d_sequence(S):
    R1 = synthetic.make_sequence(synthetic.spec_custom(1, (16, 16), seed=2))
    stats, y, _ = _register(S, R1, 0, n_levels=2, n_tlevels=2)
    assert np.all(y == 0.0)                 # one frame: the penalty pins it to Id
    spec = synthetic.spec_custom(5, (16, 16, 16), seed=4, amp=1.0)
    R3 = synthetic.make_sequence(spec)
    stats, y3, prm = _register(S, R3, 0, n_levels=2, n_tlevels=2)
    op = _oparams(prm)
    res = _oracle(R3, op, "stml", stats)
    assert gir_counts(stats) == gir_counts(res.stats)
    Jg = multilevel.final_objective(R3.astype(np.float64), y3.astype(np.float64), op)["J"]
    Jo = multilevel.final_objective(R3.astype(np.float64), res.y, op)["J"]
    assert abs(Jg - Jo) <= E2E_J * Jo, (Jg, Jo)
    assert float(np.sqrt(np.mean((y3 - res.y) ** 2))) <= E2E_RMS


def test_3d_streaming_pcg_matches_oracle(S):
    """A 3-D sequence solved with the streaming PCG passes (start, Hessian
    product, update and direction kernels in 3-D; the cooperative solve is
    switched off): the final objective agrees with the oracle's."""
    spec = synthetic.spec_custom(5, (12, 16, 20), seed=5, amp=1.0)
    R3 = synthetic.make_sequence(spec)
    stats, y3, prm = _register(S, R3, 0, n_levels=2, n_tlevels=2, pcg_cooperative=0)
    assert sum(s["cg_iters"] for s in stats) > 0
    op = _oparams(prm)
    res = _oracle(R3, op, "stml", stats)
    got, want = _counts(stats, res)
    assert got == want
    Jg = multilevel.final_objective(R3.astype(np.float64), y3.astype(np.float64), op)["J"]
    Jo = multilevel.final_objective(R3.astype(np.float64), res.y, op)["J"]
    assert abs(Jg - Jo) <= E2E_J * Jo, (Jg, Jo)
    assert float(np.sqrt(np.mean((y3 - res.y) ** 2))) <= E2E_RMS


def test_autotune_is_reproducible_and_close(S, tiny):
    """params.autotune: the tuned launch shapes and PCG path are kept for the
    context (a second registration is bit-identical) and the result stays
    within the end-to-end tolerance of the built-in choices."""
    import torch
    spec, R = tiny
    _, y_ref, prm = _register(S, R, 0, n_levels=2, n_tlevels=2)
    ctx = _ctx(S, R, n_levels=2, n_tlevels=2, autotune=1)
    try:
        ys = []
        for _ in range(2):
            S.stml_load_sequence(ctx.ptr, torch.from_numpy(R).cuda())
            S.stml_build_pyramid(ctx.ptr)
            S.stml_register(ctx.ptr, 0)
            y = np.empty_like(y_ref)
            S.stml_get_field(ctx.ptr, 1, y)
            ys.append(y)
        assert np.array_equal(ys[0], ys[1])
        table = S.stml_tuning_report(ctx.ptr)
        assert any(e["what"] == "objective_shape" for e in table)
        assert all(e["vec"] in (1, 2, 4) and 1 <= e["splits"] <= 8 for e in table if e["what"] == "objective_shape")
        op = _oparams(prm)
        J_ref = multilevel.final_objective(R.astype(np.float64), y_ref.astype(np.float64), op)["J"]
        J_tun = multilevel.final_objective(R.astype(np.float64), ys[0].astype(np.float64), op)["J"]
        assert abs(J_tun - J_ref) <= E2E_J * J_ref, (J_tun, J_ref)
        assert float(np.sqrt(np.mean((ys[0] - y_ref) ** 2))) <= E2E_RMS
    finally:
        ctx.close()


def test_coop_sync_floor_on_the_solve_grids():
    """The latency floor of a cooperative CG step is measured on grids up to
    the solve's largest (two CTAs per SM); a grid that cannot be resident is
    refused before any launch."""
    S = cuda_lib()
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for blocks in (1, 64, 2 * sms):
        us = S.stml_coop_sync_floor(blocks, 200)
        assert 0.0 < us < 1000.0
    with pytest.raises(S.StmlError) as e:
        S.stml_coop_sync_floor(1000 * sms, 10)
    assert e.value.status == -1
    assert "resident" in S.stml_last_error(None)
