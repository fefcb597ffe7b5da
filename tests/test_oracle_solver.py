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


# ---------------------------------------------------------------- Armijo
def _quadratic_line(a: float, g: float, scale: float):
    """f(u) = a/2 u^2 at u0 = g / a (gradient g), direction d = -scale g / a:
    phi(t) = f(u0 + t d), phi(0), phi'(0) = <g, d>."""
    u0 = g / a
    d = -scale * g / a
    return (lambda t: 0.5 * a * (u0 + t * d) ** 2), 0.5 * a * u0 * u0, g * d


@pytest.mark.parametrize("scale,c,t_expected", [
    (1.0, 1e-4, 1.0),      # the Newton step is accepted at once
    (4.0, 1e-4, 0.25),     # phi(t) - phi(0) = (g^2/a)(-4t + 8t^2): accepted iff t <= (1 - c)/2
    (4.0, 0.6, 0.125),     # a stricter c: t <= (1 - c)/2 = 0.2
    (3.0, 1e-4, 0.5),      # (g^2/a)(-3t + 4.5t^2): t <= 2(1 - c)/3
])
def test_armijo_accepts_the_largest_dyadic_step_of_the_closed_form(scale, c, t_expected):
    """For a quadratic along d the sufficient-decrease test reads
    t <= 2 (1 - c) |<g, d>| / (d^T H d); back-tracking from t = 1 by halving
    accepts the largest power of two below that bound."""
    phi, J, gTd = _quadratic_line(a=2.0, g=3.0, scale=scale)
    bound = 2.0 * (1.0 - c) * abs(gTd) / (2.0 * (scale * 3.0 / 2.0) ** 2)
    assert t_expected <= bound < 2 * t_expected
    t, trials, ok = solver.armijo(phi, J, gTd, c, 10)
    assert ok and t == t_expected
    assert trials == 1 + int(round(-np.log2(t_expected)))


def test_armijo_gives_up_after_max_ls_trials():
    phi, J, gTd = _quadratic_line(a=1.0, g=1.0, scale=16.0)     # accepted only for t <= (1 - c)/8
    t, trials, ok = solver.armijo(phi, J, gTd, 1e-4, 4)           # 1, 1/2, 1/4, 1/8 all fail
    assert not ok and trials == 4
    t, trials, ok = solver.armijo(phi, J, gTd, 1e-4, 5)
    assert ok and t == 0.0625 and trials == 5


# ---------------------------------------------------------------- PCG breakdown
def test_pcg_breakdown_on_first_step_returns_preconditioned_gradient():
    """An indefinite H with p0^T H p0 < 0 for p0 = M^-1 b: the solver returns
    M^-1 b (the preconditioned gradient step) and reports the breakdown."""
    H = np.diag([1.0, -1.0])
    b = np.array([1.0, 2.0])
    Minv = np.array([0.5, 2.0])           # p0 = (0.5, 4): p0^T H p0 = 0.25 - 16 < 0
    x, steps, flag = solver.pcg(lambda v: H @ v, b, Minv, 1e-12, 10)
    assert flag == "breakdown" and steps == 0
    assert np.array_equal(x, Minv * b)


def test_pcg_breakdown_after_one_step_keeps_the_first_iterate():
    """H = diag(2, 1, -1), b = (1, .1, .1), M = I: the first step is the exact
    line minimiser along b, x1 = (b.b / b.Hb) b; the second direction has
    negative curvature, so x1 is returned."""
    H = np.diag([2.0, 1.0, -1.0])
    b = np.array([1.0, 0.1, 0.1])
    x, steps, flag = solver.pcg(lambda v: H @ v, b, np.ones(3), 1e-12, 10)
    assert flag == "breakdown" and steps == 1
    x1 = (b @ b) / (b @ H @ b) * b
    assert np.allclose(x, x1, rtol=0, atol=1e-15)
    r1 = b - H @ x1                       # the next direction r1 + beta b has p^T H p < 0
    p1 = r1 + (r1 @ r1) / (b @ b) * b
    assert p1 @ H @ p1 < 0


# ---------------------------------------------------------------- correlation (Table 1)
def test_corr_coeff_hand_computed_and_affine_invariance():
    """Two 2x2 frames (1, 2, 3, 4) and (1, 3, 2, 4): centred (-1.5, -.5, .5, 1.5)
    and (-1.5, .5, -.5, 1.5), inner product 4, squared norms 5 and 5: rho = 0.8.
    A frame that is an increasing affine map of its predecessor has rho = 1,
    a decreasing one rho = -1; the values equal numpy's corrcoef."""
    a = np.array([[1.0, 2.0], [3.0, 4.0]])
    b = np.array([[1.0, 3.0], [2.0, 4.0]])
    assert multilevel.corr_coeff(np.stack([a, b])) == pytest.approx([0.8], abs=1e-15)
    rng = np.random.default_rng(5)
    f = rng.uniform(size=(6, 7))
    R = np.stack([f, 0.3 + 2.5 * f, 1.0 - 0.5 * (0.3 + 2.5 * f)])
    rho = multilevel.corr_coeff(R)
    assert rho == pytest.approx([1.0, -1.0], abs=1e-14)
    S = rng.uniform(size=(5, 4, 3))
    ref = [np.corrcoef(S[k].ravel(), S[k + 1].ravel())[0, 1] for k in range(4)]
    assert multilevel.corr_coeff(S) == pytest.approx(ref, abs=1e-14)


def test_gauss_newton_records_cg_steps_and_trials_per_iteration():
    sp = synthetic.spec_custom(4, (16, 16), seed=7, amp=1.0)
    R = synthetic.make_sequence(sp).astype(np.float64)
    _, st = solver.gauss_newton(R, np.zeros((4, 2, 16, 16)), [0, 1, 2, 3], 1.0, Params(max_gn=3))
    assert len(st.steps) == st.gn_iters
    assert sum(s for s, _ in st.steps) == st.cg_iters
    assert sum(t for _, t in st.steps) == st.ls_trials


# ---------------------------------------------------------------- target objective
def test_land_finds_the_crossing_of_a_quadratic():
    """phi(t) = 3 - 2t + t^2 crosses J* = 2.25 at t = 1/2 on [0, 1] (the other
    root, 3/2, lies outside the bracket)."""
    phi = lambda t: 3.0 - 2.0 * t + t * t
    t, J, evals = solver.land(phi, 3.0, 1.0, phi(1.0), 2.25, 1e-10)
    assert abs(J - 2.25) <= 1e-10 * 2.25
    assert abs(t - 0.5) <= 1e-9
    assert 1 <= evals <= 40
    # an accepted step already within the tolerance needs no evaluation
    t, J, evals = solver.land(phi, 3.0, 0.5, 2.25 * (1 + 1e-7), 2.25, 1e-6)
    assert (t, evals) == (0.5, 0)


def test_gauss_newton_stops_at_the_target_objective():
    sp = synthetic.spec_custom(4, (16, 16), seed=7, amp=1.0)
    R = synthetic.make_sequence(sp).astype(np.float64)
    K = [0, 1, 2, 3]
    u0 = np.zeros((4, 2, 16, 16))
    _, free = solver.gauss_newton(R, u0, K, 1.0, Params())
    Js = [J for J, _ in free.history]
    assert len(Js) >= 3
    target = 0.5 * (Js[1] + Js[2])            # crossed during the second step
    u, st = solver.gauss_newton(R, u0, K, 1.0, Params(target_tol=1e-7), target)
    assert st.status == "target" and st.gn_iters == 2
    assert abs(st.J - target) <= 1e-7 * target
    assert st.history[-1][0] > target          # the iterate before the shortened step
    J_check = objective.evaluate(R, u, K, 1.0, Params(), want_grad=False)["J"]
    assert J_check == pytest.approx(st.J, rel=1e-14)
    # a start at or below the target takes no step
    _, st0 = solver.gauss_newton(R, u0, K, 1.0, Params(), Js[0] * 1.01)
    assert st0.gn_iters == 0 and st0.status == "target"


def test_pcg_flip_takes_the_other_branch_of_one_stopping_decision():
    """flip=k inverts only the decision after step k + 1: a stop becomes a
    further step, a further step becomes a stop; the ratios before it are
    unchanged."""
    rng = np.random.default_rng(12)
    A = rng.normal(size=(30, 30))
    H = A @ A.T + 3.0 * np.eye(30)
    b = rng.normal(size=30)
    Minv = 1.0 / np.diag(H)
    rec = []
    x, n, flag = solver.pcg(lambda v: H @ v, b, Minv, 0.1, 50, rec)
    assert flag == "converged" and n >= 3
    rec_stop = []
    _, n1, _ = solver.pcg(lambda v: H @ v, b, Minv, 0.1, 50, rec_stop, flip=n - 1)
    assert n1 > n and rec_stop[:n] == rec
    rec_go = []
    _, n2, _ = solver.pcg(lambda v: H @ v, b, Minv, 0.1, 50, rec_go, flip=n - 2)
    assert n2 == n - 1 and rec_go == rec[:n - 1]


def test_oracle_branch_follows_only_near_threshold_decisions():
    """The test helper reruns the oracle with a near-threshold CG decision on
    its other branch when that explains the GPU's counts, and refuses
    differences that no such decision explains (3-D sequence whose oracle
    run has a CG ratio 0.14 % above tol_cg in its second GIR)."""
    import sys, os
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from _util import CG_BRANCH_DELTA, gir_counts, oracle_branch
    from oracle import multilevel
    from paper_2001_06613_gb300 import synthetic
    R3 = synthetic.make_sequence(synthetic.spec_custom(5, (16, 16, 16), seed=4, amp=1.0)).astype(np.float64)
    op = Params(n_levels=2, n_tlevels=2)
    reg = lambda fl: multilevel.register(R3, op, "stml", flips=fl)
    base = reg({})
    want = gir_counts(base.stats)
    res, flips = oracle_branch(reg, want, op.tol_cg)
    assert flips == {} and gir_counts(res.stats) == want
    rec = base.stats[1].cg_residuals
    near = [(i, k) for i, r in enumerate(rec) for k, x in enumerate(r)
            if abs(x - op.tol_cg) / op.tol_cg < CG_BRANCH_DELTA]
    assert near and abs(rec[near[0][0]][near[0][1]] / op.tol_cg - 1.0) < 2e-3
    # counts of the other branch at that decision: found again by the helper
    other = gir_counts(reg({1: {near[0]}}).stats)
    assert other != want and other[0] == want[0]
    res, flips = oracle_branch(reg, other, op.tol_cg)
    assert gir_counts(res.stats) == other and flips == {1: {near[0]}}
    # a count difference that no near-threshold decision explains is refused
    bogus = [c if i != 0 else c[:4] + (c[4] + 7,) + c[5:] for i, c in enumerate(want)]
    with pytest.raises(AssertionError):
        oracle_branch(reg, bogus, op.tol_cg)
