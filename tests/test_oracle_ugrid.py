"""Pins of the oracle's coarse displacement grid (u = P_s w, w on the image grid
coarsened by 2^s; the gradient gathers through P_s^T)."""
import numpy as np
import pytest

from oracle import Params, grid, multilevel, objective, solver, ugrid
from paper_2001_06613_gb300 import synthetic


def _problem(seed=0, K=3, shape=(16, 12), s=1, amp=1.2):
    rng = np.random.default_rng(seed)
    d = len(shape)
    T = rng.uniform(0.0, 1.0, size=(K,) + shape)
    cshape = tuple(m // 2 ** s for m in shape)
    w = rng.uniform(-amp, amp, size=(K, d) + cshape)
    frames = sorted(rng.choice(3 * K, size=K, replace=False).tolist())
    return T, w, frames


def _cells(T, w, s, h=1.0):
    """Cell index of every warped sample point (to see that a finite
    difference stays on one side of every grid line)."""
    u = ugrid.prolong(w, T.shape[1:], s)
    x = grid.cell_centres(T.shape[1:], h)
    return np.floor((x[None] + u) / h - 0.5)


def test_axis_matrix_worked_example_factor_4():
    """8 fine cells, 2 coarse cells (F = 4), worked out by hand from
    xi = (j + 1/2)/4 - 1/2 with clamping at both ends."""
    want = np.array([[1.0, 0.0], [1.0, 0.0], [0.875, 0.125], [0.625, 0.375],
                     [0.375, 0.625], [0.125, 0.875], [0.0, 1.0], [0.0, 1.0]])
    np.testing.assert_array_equal(ugrid.axis_matrix(8, 4), want)


def test_factor_two_equals_level_prolongation():
    """P_1 is the level-to-level prolongation of the grid module (written
    independently, as 2^d clamped stencils)."""
    rng = np.random.default_rng(1)
    for shape in [(5, 7), (3, 4, 5)]:
        w = rng.normal(size=shape)
        fine = tuple(2 * m for m in shape)
        np.testing.assert_allclose(ugrid.prolong(w, fine, 1), grid.prolong(w), rtol=0, atol=1e-14)
        u = rng.normal(size=fine)
        np.testing.assert_allclose(ugrid.adjoint(u, fine, 1), grid.prolong_adjoint(u), rtol=0, atol=1e-13)


@pytest.mark.parametrize("s", [1, 2, 3])
def test_prolongation_reproduces_constants_and_interior_affine(s):
    F = 2 ** s
    shape = (8 * F, 6 * F)
    cshape = (8, 6)
    np.testing.assert_allclose(ugrid.prolong(np.full(cshape, 2.5), shape, s), 2.5, rtol=0, atol=1e-14)
    # an affine function of the coarse cell centres is reproduced at every fine
    # cell centre between the first and last coarse centre (no clamping)
    xc = [(np.arange(m) + 0.5) * F for m in cshape]
    Xc = np.meshgrid(*xc, indexing="ij")
    w = 0.3 * Xc[0] - 0.7 * Xc[1] + 1.1
    u = ugrid.prolong(w, shape, s)
    xf = [np.arange(m) + 0.5 for m in shape]
    Xf = np.meshgrid(*xf, indexing="ij")
    inside = np.ones(shape, bool)
    for a in range(2):
        inside &= (Xf[a] >= xc[a][0]) & (Xf[a] <= xc[a][-1])
    exact = 0.3 * Xf[0] - 0.7 * Xf[1] + 1.1
    assert inside.sum() > 0
    np.testing.assert_allclose(u[inside], exact[inside], rtol=0, atol=1e-12)


def test_adjoints_are_transposes():
    rng = np.random.default_rng(2)
    shape, s = (12, 8, 16), 2
    cshape = tuple(m // 4 for m in shape)
    w = rng.normal(size=(2,) + cshape)
    u = rng.normal(size=(2,) + shape)
    assert float(np.sum(ugrid.prolong(w, shape, s) * u)) == pytest.approx(
        float(np.sum(w * ugrid.adjoint(u, shape, s))), rel=1e-13)
    # (P o P)^T against the explicit matrix of P built column by column
    P = np.stack([ugrid.prolong(np.eye(int(np.prod(cshape)))[i].reshape(cshape), shape, s).ravel()
                  for i in range(int(np.prod(cshape)))], axis=1)
    np.testing.assert_allclose(ugrid.adjoint_sq(u[0], shape, s).ravel(), (P * P).T @ u[0].ravel(),
                               rtol=0, atol=1e-12)


def test_no_coarsening_is_the_image_grid_model():
    rng = np.random.default_rng(3)
    T = rng.uniform(size=(4, 9, 11))
    u = rng.uniform(-1.0, 1.0, size=(4, 2, 9, 11))
    frames = [0, 2, 3, 7]
    p = Params(alpha=0.3, lam=2.0, alpha_t=0.5)
    a = ugrid.evaluate(T, u, frames, 2.0, 0, p)
    b = objective.evaluate(T, u, frames, 2.0, p)
    for k in ("J", "D", "S", "P"):
        assert a[k] == pytest.approx(b[k], rel=1e-14)
    np.testing.assert_allclose(a["g"], b["g"], rtol=0, atol=1e-13 * np.abs(b["g"]).max())
    v = rng.normal(size=u.shape)
    np.testing.assert_allclose(ugrid.hessvec(a["dT"], v, frames, 2.0, 0, p),
                               objective.hessvec(b["dT"], v, frames, 2.0, p), rtol=0, atol=1e-12)
    np.testing.assert_allclose(ugrid.jacobi_diag(a["dT"], frames, 2.0, 0, p),
                               objective.jacobi_diag(b["dT"], frames, 2.0, p), rtol=1e-14)


@pytest.mark.parametrize("s,h", [(1, 1.0), (2, 2.0)])
@pytest.mark.parametrize("terms", [dict(alpha=0.0, lam=0.0), dict(alpha=0.4, lam=2.0, alpha_t=0.3)])
def test_gradient_matches_central_differences(s, h, terms):
    T, w, frames = _problem(seed=4, s=s)
    p = Params(**terms)
    ev = ugrid.evaluate(T, w, frames, h, s, p)
    rng = np.random.default_rng(5)
    v = rng.uniform(-1, 1, size=w.shape)
    eps = 1e-6
    # the difference must not carry a sample point across a grid line
    assert np.array_equal(_cells(T, w + eps * v, s, h), _cells(T, w - eps * v, s, h))
    Jp = ugrid.evaluate(T, w + eps * v, frames, h, s, p, want_grad=False)["J"]
    Jm = ugrid.evaluate(T, w - eps * v, frames, h, s, p, want_grad=False)["J"]
    fd = (Jp - Jm) / (2 * eps)
    assert float(np.sum(ev["g"] * v)) == pytest.approx(fd, rel=1e-6, abs=1e-9 * (1 + abs(ev["J"])))


def test_hessian_is_symmetric_and_the_jacobian_gram_plus_quadratic_terms():
    s, h = 1, 1.0
    T, w, frames = _problem(seed=6, s=s)
    p = Params(alpha=0.5, lam=1.5, alpha_t=0.2)
    ev = ugrid.evaluate(T, w, frames, h, s, p)
    rng = np.random.default_rng(7)
    a = rng.normal(size=w.shape)
    b = rng.normal(size=w.shape)
    Ha = ugrid.hessvec(ev["dT"], a, frames, h, s, p)
    Hb = ugrid.hessvec(ev["dT"], b, frames, h, s, p)
    assert float(np.sum(a * Hb)) == pytest.approx(float(np.sum(Ha * b)), rel=1e-12)
    eps = 1e-6
    assert np.array_equal(_cells(T, w + eps * a, s, h), _cells(T, w - eps * a, s, h))
    # residual derivative by central differences of the residual r(P w)
    p0 = p.with_(alpha=0.0, alpha_t=0.0, lam=0.0)
    rp = ugrid.evaluate(T, w + eps * a, frames, h, s, p0, want_grad=False)
    rm = ugrid.evaluate(T, w - eps * a, frames, h, s, p0, want_grad=False)
    ra = (objective.residual(objective.evaluate(T, rp["u"], frames, h, p0)["a"])
          - objective.residual(objective.evaluate(T, rm["u"], frames, h, p0)["a"])) / (2 * eps)
    # S and P are quadratic in w: their second derivative along a is
    # (S + P)(2a) - 2 (S + P)(a) + (S + P)(0) = (S + P)(2a) - 2 (S + P)(a)
    q = lambda z: (lambda e: e["S"] + e["P"])(ugrid.evaluate(T, z, frames, h, s, p, want_grad=False))
    second = q(2 * a) - 2 * q(a) + q(0 * a)
    hd = h ** 2
    assert float(np.sum(a * Ha)) == pytest.approx(hd * float(np.sum(ra * ra)) + second, rel=1e-6)


def test_jacobi_diagonal_is_the_hessian_diagonal():
    """Probe the Hessian with every unit vector of a small problem."""
    s, h = 1, 1.0
    T, w, frames = _problem(seed=8, K=2, shape=(8, 6), s=s)
    p = Params(alpha=0.3, lam=0.8, alpha_t=0.4)
    ev = ugrid.evaluate(T, w, frames, h, s, p)
    diag = ugrid.jacobi_diag(ev["dT"], frames, h, s, p)
    probe = np.empty(w.size)
    for i in range(w.size):
        e = np.zeros(w.size)
        e[i] = 1.0
        probe[i] = ugrid.hessvec(ev["dT"], e.reshape(w.shape), frames, h, s, p).ravel()[i]
    np.testing.assert_allclose(diag.ravel(), probe, rtol=1e-12, atol=1e-14)


def test_identical_frames_zero_motion_is_stationary():
    rng = np.random.default_rng(9)
    T = np.repeat(rng.uniform(size=(1, 16, 16)), 4, axis=0)
    w = np.zeros((4, 2, 8, 8))
    ev = ugrid.evaluate(T, w, list(range(4)), 1.0, 1, Params(alpha=0.3, lam=2.0))
    assert ev["J"] < 1e-28 and np.max(np.abs(ev["g"])) < 1e-14
    u, st = solver.gauss_newton(T, w, list(range(4)), 1.0, Params(),
                                model=ugrid.Model(T, list(range(4)), 1.0, 1, Params()))
    assert st.gn_iters == 0 and np.all(u == 0.0)


def test_registration_recovers_planted_motion_on_a_coarse_grid():
    """Groupwise registration of a smooth planted motion with the unknowns on
    the image grid coarsened by 2 (STML, 2 x 2 levels): the prolonged fields,
    centred over the frames, match the centred inverse of the planted motion
    in the interior, as with the unknowns on the image grid."""
    spec = synthetic.spec_custom(6, (32, 32), seed=11, amp=1.5)
    R = synthetic.make_sequence(spec).astype(np.float64)
    truth = synthetic.planted_registration(spec)
    p = Params(n_levels=2, n_tlevels=2, u_coarsen=1)
    res = multilevel.register(R, p, "stml")
    assert res.y.shape == (6, 2, 16, 16)
    u = ugrid.prolong(res.y, (32, 32), 1)
    c = lambda f: f - f.mean(axis=0, keepdims=True)
    err = c(u) - c(truth)
    inner = lambda f: float(np.sqrt(np.mean(f[:, :, 4:-4, 4:-4] ** 2)))
    rms, rms0 = inner(err), inner(c(truth))
    # the same registration with the unknowns on the image grid
    img = multilevel.register(R, p.with_(u_coarsen=0), "stml")
    rms_img = inner(c(img.y) - c(truth))
    assert rms < 0.25 and rms < 0.5 * rms0 and rms < 1.2 * rms_img, (rms, rms0, rms_img)
    fo = multilevel.final_objective(R, res.y, p)
    assert fo["J"] == pytest.approx(res.stats[-1].J, rel=1e-12)
