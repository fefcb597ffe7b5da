"""GPU parity of the persistent batched solver (stml_batch_*).

Several sequences of uneven frame counts and sizes are registered together:
one persistent cooperative kernel per (spatial level, temporal level) stage
runs every sequence's Gauss-Newton / PCG / Armijo loop.  Each sequence's
result is compared with the FP64 oracle registering that sequence alone (the
same step counts, final objective within 1e-4, fields within 1e-3 px RMS)
and with the single-context path (stml_register)."""
import numpy as np
import pytest

from _util import cuda_lib
from oracle import Params, multilevel
from paper_2001_06613_gb300 import synthetic

pytestmark = pytest.mark.gpu

E2E_J, E2E_RMS = 1e-4, 1e-3


@pytest.fixture(scope="module")
def S():
    return cuda_lib()


def _oparams(prm):
    return Params(alpha=prm.alpha, alpha_t=prm.alpha_t, lam=prm.lambda_, beta=prm.beta, eps_stop=prm.eps_stop,
                  stop_rule=bool(prm.stop_rule), n_levels=prm.n_levels, n_tlevels=prm.n_tlevels, tol_J=prm.tol_J,
                  tol_Y=prm.tol_Y, tol_G=prm.tol_G, max_gn=prm.max_gn, tol_cg=prm.tol_cg, max_cg=prm.max_cg,
                  max_ls=prm.max_ls, armijo_c=prm.armijo_c, g_abs=prm.g_abs)


def _contexts(S, seqs, **kw):
    import torch
    prm = S.stml_default_params(**kw)
    ctxs = []
    for R in seqs:
        c = S.Context(prm)
        S.stml_load_sequence(c.ptr, torch.from_numpy(R).cuda())
        S.stml_build_pyramid(c.ptr)
        ctxs.append(c)
    return ctxs, prm


def _field(S, ctx, R):
    y = np.empty((R.shape[0], R.ndim - 1) + R.shape[1:], np.float32)
    S.stml_get_field(ctx.ptr, ctx.params.n_levels - 1, y)
    return y


def _counts_gpu(stats):
    return [(s["level"], s["tlevel"], s["n_frames"], s["gn_iters"], s["cg_iters"], s["ls_trials"]) for s in stats]


def _counts_oracle(res):
    return [(s.level, s.tlevel, s.n_frames, s.gn_iters, s.cg_iters, s.ls_trials) for s in res.stats]


def _check_against_oracle(S, ctxs, seqs, prm, mode):
    op = _oparams(prm)
    for c, R in zip(ctxs, seqs):
        y = _field(S, c, R)
        res = multilevel.register(R.astype(np.float64), op, "stml" if mode == 0 else "spml")
        assert _counts_gpu(S.stml_last_stats(c.ptr)) == _counts_oracle(res)
        Jg = multilevel.final_objective(R.astype(np.float64), y.astype(np.float64), op)["J"]
        Jo = multilevel.final_objective(R.astype(np.float64), res.y, op)["J"]
        assert abs(Jg - Jo) <= E2E_J * Jo, (R.shape, Jg, Jo)
        assert float(np.sqrt(np.mean((y - res.y) ** 2))) <= E2E_RMS


def _uneven_2d(nx_mult4=True):
    if nx_mult4:
        shapes = [(9, (32, 48), 1.2), (16, (64, 64), 1.5), (5, (48, 32), 1.0), (1, (32, 32), 1.0)]
    else:
        shapes = [(7, (30, 42), 1.2), (12, (34, 26), 1.4)]    # a level with nx % 4 != 0: scalar path
    return [synthetic.make_sequence(synthetic.spec_custom(n, sh, seed=40 + i, amp=a))
            for i, (n, sh, a) in enumerate(shapes)]


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("vec4", [True, False])
def test_batch_of_uneven_2d_sequences_matches_the_oracle(S, mode, vec4):
    seqs = _uneven_2d(vec4)
    ctxs, prm = _contexts(S, seqs, n_levels=2, n_tlevels=2)
    batch = S.Batch(ctxs)
    try:
        assert batch.register(mode) == [0] * len(seqs)
        _check_against_oracle(S, ctxs, seqs, prm, mode)
        rep = batch.report()
        assert rep and all(r["steps"] > 0 for r in rep if "steps" in r)
    finally:
        batch.close()
        for c in ctxs:
            c.close()


def test_batch_equals_single_context_registration(S):
    """The batched solver takes the decisions of stml_register: the same
    step counts and, to rounding, the same fields and objectives."""
    seqs = _uneven_2d(True)
    ctxs, prm = _contexts(S, seqs, n_levels=2, n_tlevels=2)
    batch = S.Batch(ctxs)
    try:
        batch.register(0)
        for c, R in zip(ctxs, seqs):
            y_b = _field(S, c, R)
            st_b = S.stml_last_stats(c.ptr)
            st_s = S.stml_register(c.ptr, 0)
            y_s = _field(S, c, R)
            assert _counts_gpu(st_b) == _counts_gpu(st_s)
            for a, b in zip(st_b, st_s):
                assert abs(a["J"] - b["J"]) <= 1e-5 * abs(b["J"])
            # the objective passes sum in different orders; measured 1.6e-4 px
            assert float(np.sqrt(np.mean((y_b - y_s) ** 2))) <= E2E_RMS
    finally:
        batch.close()
        for c in ctxs:
            c.close()


def test_batch_of_3d_sequences_matches_the_oracle(S):
    seqs = [synthetic.make_sequence(synthetic.spec_custom(5, (12, 16, 20), seed=45, amp=1.0)),
            synthetic.make_sequence(synthetic.spec_custom(4, (16, 16, 16), seed=46, amp=1.0))]
    ctxs, prm = _contexts(S, seqs, n_levels=2, n_tlevels=2)
    batch = S.Batch(ctxs)
    try:
        batch.register(0)
        _check_against_oracle(S, ctxs, seqs, prm, 0)
    finally:
        batch.close()
        for c in ctxs:
            c.close()


def test_batch_with_bf16_storage_equals_single_context(S):
    seqs = _uneven_2d(True)[:3]
    ctxs, prm = _contexts(S, seqs, n_levels=2, n_tlevels=2, image_dtype=2)
    batch = S.Batch(ctxs)
    try:
        batch.register(0)
        for c, R in zip(ctxs, seqs):
            y_b = _field(S, c, R)
            J_b = S.stml_last_stats(c.ptr)[-1]["J"]
            S.stml_register(c.ptr, 0)
            y_s = _field(S, c, R)
            J_s = S.stml_last_stats(c.ptr)[-1]["J"]
            assert abs(J_b - J_s) <= E2E_J * abs(J_s)
            assert float(np.sqrt(np.mean((y_b - y_s) ** 2))) <= E2E_RMS
    finally:
        batch.close()
        for c in ctxs:
            c.close()


def test_autotuned_batch_is_reproducible_and_within_tolerance(S):
    seqs = _uneven_2d(True)
    ctxs, prm = _contexts(S, seqs, n_levels=2, n_tlevels=2, autotune=1)
    batch = S.Batch(ctxs)
    try:
        batch.register(0)
        rep = batch.report()
        tuned = [r for r in rep if "tuned_level" in r]
        assert len(tuned) == 2 and all(len(r["tried"]) >= 2 for r in tuned)
        y1 = [_field(S, c, R) for c, R in zip(ctxs, seqs)]
        batch.register(0)                    # the choices are kept: no new trials
        assert not any("tuned_level" in r for r in batch.report())
        y2 = [_field(S, c, R) for c, R in zip(ctxs, seqs)]
        for a, b in zip(y1, y2):
            assert np.array_equal(a, b)
        _check_against_oracle(S, ctxs, seqs, prm, 0)
    finally:
        batch.close()
        for c in ctxs:
            c.close()


def test_batch_refuses_mixed_solver_parameters(S):
    import torch
    seqs = _uneven_2d(True)[:2]
    a = S.Context(S.stml_default_params(n_levels=2, n_tlevels=2))
    b = S.Context(S.stml_default_params(n_levels=2, n_tlevels=2, alpha=0.5))
    try:
        for c, R in zip((a, b), seqs):
            S.stml_load_sequence(c.ptr, torch.from_numpy(R).cuda())
            S.stml_build_pyramid(c.ptr)
        batch = S.Batch([a, b])
        try:
            with pytest.raises(S.StmlError) as e:
                batch.register(0)
            assert e.value.status == -1
        finally:
            batch.close()
        with pytest.raises(S.StmlError):
            S.Batch([a, a])
    finally:
        a.close()
        b.close()


def test_batch_barrier_wait_is_bounded(S):
    """A barrier that nothing completes gives up after its bound and reports
    it (the status a stalled batched solve returns as STML_ETIMEOUT); the
    device stays usable afterwards."""
    import torch
    assert S.stml_check_batch_barrier() is True
    x = torch.ones(1024, device="cuda")
    assert float(x.sum()) == 1024.0


@pytest.mark.parametrize("mode", [0, 1])
def test_batch_target_objective_lands_per_sequence(S, mode):
    """Each sequence's last GIR stops at its own target objective (the
    regula falsi landing of the single-context path, on the device)."""
    seqs = _uneven_2d(True)[:3]
    ctxs, prm = _contexts(S, seqs, n_levels=2, n_tlevels=2)
    batch = S.Batch(ctxs)
    try:
        batch.register(mode)
        targets = []
        for c in ctxs:
            last = S.stml_last_stats(c.ptr)[-1]
            targets.append(0.5 * (last["J0"] + last["J"]) if last["gn_iters"] >= 2 else 0.0)
        for c, t in zip(ctxs, targets):
            S.stml_set_params(c.ptr, S.stml_default_params(n_levels=2, n_tlevels=2, target_J=t))
        batch.register(mode)
        for c, R, t in zip(ctxs, seqs, targets):
            got = S.stml_last_stats(c.ptr)
            S.stml_set_params(c.ptr, S.stml_default_params(n_levels=2, n_tlevels=2, target_J=t))
            ref = S.stml_register(c.ptr, mode)
            assert _counts_gpu(got) == _counts_gpu(ref)
            if t > 0:
                assert abs(got[-1]["J"] - t) <= 2 * prm.target_tol * t, (got[-1]["J"], t)
    finally:
        batch.close()
        for c in ctxs:
            c.close()


def test_batch_of_one_and_a_stationary_sequence(S):
    """Degenerate batches: a single sequence (its GIRs get the whole grid),
    and a sequence of identical frames, where u = 0 is stationary and every
    GIR stops at its first evaluation with the fields exactly zero."""
    base = synthetic.make_sequence(synthetic.spec_custom(1, (32, 32), seed=3))
    still = np.repeat(base, 6, axis=0)
    one = _uneven_2d(True)[1]
    for seqs in ([one], [still, one]):
        ctxs, prm = _contexts(S, seqs, n_levels=2, n_tlevels=2)
        batch = S.Batch(ctxs)
        try:
            assert batch.register(0) == [0] * len(seqs)
            _check_against_oracle(S, ctxs, seqs, prm, 0)
            if len(seqs) == 2:
                assert all(s["gn_iters"] == 0 and s["cg_iters"] == 0 for s in S.stml_last_stats(ctxs[0].ptr))
                assert float(np.abs(_field(S, ctxs[0], still)).max()) == 0.0
        finally:
            batch.close()
            for c in ctxs:
                c.close()
