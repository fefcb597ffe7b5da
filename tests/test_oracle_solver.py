"""Pins of the oracle's solver and multilevel drivers."""
import numpy as np
import pytest

from oracle import grid, multilevel, objective, solver, Params
from paper_2001_06613_gb300 import synthetic


def _explicit_hessian(dT, frames, h, p):
    size = dT.size
    H = np.zeros((size, size))
    e = np.zeros(dT.shape)
    for i, idx in enumerate(np.ndindex(dT.shape)):
        e[idx] = 1.0
        H[:, i] = objective.hessvec(dT, e, frames, h, p).ravel()
        e[idx] = 0.0
    return H


def test_pcg_solves_the_newton_system():
    rng = np.random.default_rng(0)
    T = rng.uniform(size=(3, 5, 4))
    u = rng.uniform(-1, 1, size=(3, 2, 5, 4))
    p = Params(alpha=0.3, lam=1.0, alpha_t=0.2)
    frames = [0, 1, 3]
    ev = objective.evaluate(T, u, frames, 1.0, p)
    H = _explicit_hessian(ev["dT"], frames, 1.0, p)
    ref = np.linalg.solve(H, -ev["g"].ravel())
    Minv = 1.0 / objective.jacobi_diag(ev["dT"], frames, 1.0, p)
    x, steps, flag = solver.pcg(lambda v: objective.hessvec(ev["dT"], v, frames, 1.0, p),
                                -ev["g"], Minv, 1e-13, 500)
    assert flag == "converged"
    assert np.allclose(x.ravel(), ref, rtol=1e-8, atol=1e-10 * np.abs(ref).max())


def test_zero_motion_exits_at_iteration_zero():
    rng = np.random.default_rng(1)
    T = np.repeat(rng.uniform(size=(1, 8, 8)), 4, axis=0)
    u, st = solver.gauss_newton(T, np.zeros((4, 2, 8, 8)), [0, 1, 2, 3], 1.0, Params())
    assert st.gn_iters == 0 and st.cg_iters == 0
    assert np.all(u == 0.0)


def test_gauss_newton_decreases_objective():
    sp = synthetic.spec_tiny()
    R = synthetic.make_sequence(sp).astype(np.float64)
    T = multilevel.pyramid(R, 2)[0]
    K = grid.temporal_sets(16, 2)[0]
    _, st = solver.gauss_newton(T[K], np.zeros((len(K), 2) + T.shape[1:]), K, 2.0, Params())
    Js = [J for J, _ in st.history]
    assert all(b <= a for a, b in zip(Js[:-1], Js[1:]))
    assert Js[-1] < 0.5 * Js[0]


@pytest.fixture(scope="module")
def tiny_runs():
    sp = synthetic.spec_tiny()
    R = synthetic.make_sequence(sp).astype(np.float64)
    p = Params(n_levels=2, n_tlevels=2)
    return sp, R, p, multilevel.register(R, p, "stml"), multilevel.register(R, p, "spml")


def _centred_rms(y, truth):
    a = y - y.mean(axis=0, keepdims=True)
    b = truth - truth.mean(axis=0, keepdims=True)
    e = (a - b)[..., 4:-4, 4:-4]
    return float(np.sqrt((e ** 2).sum(axis=1).mean()))


def test_planted_motion_is_recovered(tiny_runs):
    sp, R, p, stml, spml = tiny_runs
    truth = synthetic.planted_registration(sp)
    before = _centred_rms(np.zeros_like(truth), truth)
    assert before > 0.6
    assert _centred_rms(stml.y, truth) < 0.2
    assert _centred_rms(spml.y, truth) < 0.2


def test_stml_and_spml_agree(tiny_runs):
    """Both strategies converge in proximity (Sec. 4, Table 1: relative y
    differences of a few per cent and nearly equal reductions of D)."""
    sp, R, p, stml, spml = tiny_runs
    Js = multilevel.final_objective(R, stml.y, p)["J"]
    Jp = multilevel.final_objective(R, spml.y, p)["J"]
    J0 = multilevel.final_objective(R, 0 * stml.y, p)["J"]
    assert abs(Js - Jp) <= 0.02 * Jp
    assert Js < 0.2 * J0
    rel = np.linalg.norm(stml.y - spml.y) / np.linalg.norm(spml.y)
    assert rel < 0.1
    # the STML sweep visits K_0 then K_1 on each level
    assert [(s.level, s.tlevel, s.n_frames) for s in stml.stats] == [
        (0, 0, 9), (0, 1, 16), (1, 0, 9), (1, 1, 16)]


def test_stopping_rule_fills_from_predictor():
    sp = synthetic.spec_custom(9, (32, 32), seed=3, amp=1.0)
    R = synthetic.make_sequence(sp).astype(np.float64)
    p = Params(n_levels=2, n_tlevels=3, eps_stop=10.0)       # always satisfied at q = 1
    res = multilevel.register(R, p, "stml")
    per_level = {}
    for s in res.stats:
        per_level.setdefault(s.level, []).append(s)
    for lvl, sts in per_level.items():
        assert [s.tlevel for s in sts] == [0, 1] and sts[-1].stopped_early
    assert res.y.shape == (9, 2, 32, 32)
    assert np.all(np.isfinite(res.y))


def test_corr_coeff_of_synthetic_sequence():
    R = synthetic.make_sequence(synthetic.spec_tiny())
    rho = multilevel.corr_coeff(R.astype(np.float64))
    assert rho.shape == (15,)
    assert 0.9 < rho.min() <= rho.max() < 1.0       # Table 1 reports 0.915 - 0.996
