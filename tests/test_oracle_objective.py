"""Pins of the oracle's objective layer (eq. 1, S and P of Sec. 2, GN Hessian)."""
import numpy as np
import pytest

from oracle import grid, objective, Params


def _problem(seed=0, K=4, shape=(10, 12), h=1.0, amp=1.5, away=0.02):
    """Random images and a displacement whose sample points sit >= ``away``
    (in cell units) from every grid line, so finite differences see no kink."""
    rng = np.random.default_rng(seed)
    d = len(shape)
    T = rng.uniform(0.0, 1.0, size=(K,) + shape)
    u = rng.uniform(-amp, amp, size=(K, d) + shape) * h
    x = grid.cell_centres(shape, h)
    xi = (x[None] + u) / h - 0.5
    frac = xi - np.floor(xi)
    u = np.where(frac < away, u + 2 * away * h, u)
    u = np.where(frac > 1 - away, u - 2 * away * h, u)
    frames = sorted(rng.choice(3 * K, size=K, replace=False).tolist())
    return T, u, frames


def test_distance_pairwise_equals_mean_form():
    rng = np.random.default_rng(3)
    a = rng.normal(size=(6, 5, 7))
    assert objective.distance_pairwise(a, 0.25) == pytest.approx(
        objective.distance_to_mean(a, 0.25), rel=1e-13)


def test_identical_frames_zero_motion_is_stationary():
    rng = np.random.default_rng(4)
    T = np.repeat(rng.uniform(size=(1, 9, 11)), 5, axis=0)
    u = np.zeros((5, 2, 9, 11))
    ev = objective.evaluate(T, u, list(range(5)), 1.0, Params(alpha=0.3, lam=2.0, alpha_t=0.5))
    # the frame mean of equal numbers is exact up to one rounding of the sum
    assert ev["J"] < 1e-28 and ev["S"] == 0.0 and ev["P"] == 0.0
    assert np.max(np.abs(ev["g"])) < 1e-14


@pytest.mark.parametrize("terms", [dict(alpha=0.0, lam=0.0), dict(alpha=0.7, lam=0.0),
                                   dict(alpha=0.0, lam=3.0), dict(alpha=0.2, lam=1.0, alpha_t=0.4)])
@pytest.mark.parametrize("shape,h", [((10, 12), 1.0), ((6, 5, 4), 2.0)])
def test_gradient_matches_central_differences(terms, shape, h):
    T, u, frames = _problem(shape=shape, h=h)
    p = Params(**terms)
    ev = objective.evaluate(T, u, frames, h, p)
    rng = np.random.default_rng(5)
    w = rng.uniform(-1, 1, size=u.shape)
    eps = 1e-6
    Jp = objective.evaluate(T, u + eps * w, frames, h, p, want_grad=False)["J"]
    Jm = objective.evaluate(T, u - eps * w, frames, h, p, want_grad=False)["J"]
    fd = (Jp - Jm) / (2 * eps)
    an = float(np.sum(ev["g"] * w))
    assert an == pytest.approx(fd, rel=1e-6, abs=1e-9 * (1 + abs(ev["J"])))


def test_gauss_newton_product_is_jacobian_gram():
    """<w, H_D v> = hd <J_r w, J_r v>, with J_r v the derivative of the residual."""
    T, u, frames = _problem(seed=6)
    h, hd = 1.0, 1.0
    p = Params(alpha=0.0, lam=0.0)
    ev = objective.evaluate(T, u, frames, h, p)
    rng = np.random.default_rng(7)
    v = rng.normal(size=u.shape)
    w = rng.normal(size=u.shape)
    eps = 1e-6

    def jr(z):
        rp = objective.evaluate(T, u + eps * z, frames, h, p, want_grad=False)["r"]
        rm = objective.evaluate(T, u - eps * z, frames, h, p, want_grad=False)["r"]
        return (rp - rm) / (2 * eps)

    lhs = float(np.sum(w * objective.hessvec(ev["dT"], v, frames, h, p)))
    rhs = hd * float(np.sum(jr(w) * jr(v)))
    assert lhs == pytest.approx(rhs, rel=1e-6)


def test_quadratic_terms_hessian_equals_gradient_difference():
    """S and P are quadratic: their Hessian times v is grad(S+P)(v) - grad(S+P)(0)."""
    T, u, frames = _problem(seed=8, shape=(6, 7, 5), h=2.0)
    p = Params(alpha=0.6, lam=1.7, alpha_t=0.3)
    flat = np.zeros_like(T)                       # images without structure: D is constant
    dT = np.zeros_like(u)
    rng = np.random.default_rng(9)
    v = rng.normal(size=u.shape)
    g_v = objective.evaluate(flat, v, frames, 2.0, p)["g"]
    g_0 = objective.evaluate(flat, 0 * v, frames, 2.0, p)["g"]
    assert np.allclose(objective.hessvec(dT, v, frames, 2.0, p), g_v - g_0, atol=1e-12)


def test_hessian_symmetric_psd_and_single_frame_null():
    T, u, frames = _problem(seed=10)
    p = Params(alpha=0.3, lam=2.0, alpha_t=0.2)
    dT = objective.evaluate(T, u, frames, 1.0, p)["dT"]
    rng = np.random.default_rng(11)
    v, w = rng.normal(size=u.shape), rng.normal(size=u.shape)
    Hv = objective.hessvec(dT, v, frames, 1.0, p)
    Hw = objective.hessvec(dT, w, frames, 1.0, p)
    assert float(np.sum(w * Hv)) == pytest.approx(float(np.sum(Hw * v)), rel=1e-13)
    assert float(np.sum(v * Hv)) > 0
    # one frame, no regulariser, no penalty: the residual is identically zero
    H1 = objective.hessvec(dT[:1], v[:1], frames[:1], 1.0, Params(alpha=0.0, lam=0.0))
    assert np.all(np.abs(H1) < 1e-15)


def test_jacobi_diagonal_is_hessian_diagonal():
    T, u, frames = _problem(seed=12, K=3, shape=(4, 5))
    p = Params(alpha=0.4, lam=1.3, alpha_t=0.7)
    dT = objective.evaluate(T, u, frames, 1.0, p)["dT"]
    diag = objective.jacobi_diag(dT, frames, 1.0, p)
    e = np.zeros(u.shape)
    got = np.zeros(u.shape)
    for idx in np.ndindex(u.shape):
        e[idx] = 1.0
        got[idx] = objective.hessvec(dT, e, frames, 1.0, p)[idx]
        e[idx] = 0.0
    assert np.allclose(diag, got, rtol=1e-13, atol=1e-15)


def test_regulariser_null_space_and_linear_field():
    shape, h = (7, 9), 2.0
    p = Params(alpha=0.8, lam=0.0)
    u = np.zeros((2, 2) + shape)
    u[:, 0] = 1.5
    u[:, 1] = -0.5
    flat = np.zeros((2,) + shape)
    ev = objective.evaluate(flat, u, [0, 1], h, p)
    assert ev["S"] == 0.0
    assert np.all(objective.diffusion_operator(u[0, 0], h) == 0.0)
    # u_1 = c * x_1: every interior edge along axis 1 has difference c
    c = 0.3
    x = grid.cell_centres(shape, h)
    u = np.zeros((1, 2) + shape)
    u[0, 1] = c * x[1]
    Sx = objective.evaluate(flat[:1], u, [0], h, p)["Sx"]
    edges = shape[0] * (shape[1] - 1)
    assert Sx == pytest.approx(0.5 * p.alpha * h ** 2 * c * c * edges, rel=1e-13)


def test_temporal_term_closed_forms():
    shape = (5, 6)
    p = Params(alpha=0.0, lam=0.0, alpha_t=1.3)
    frames = [0, 2, 3, 7]
    flat = np.zeros((4,) + shape)
    u = np.ones((4, 2) + shape) * 0.7
    assert objective.evaluate(flat, u, frames, 1.0, p)["St"] == 0.0
    # linear in time: u_k = k c -> each pair contributes (dk c)^2 / dk^2 = c^2 per component
    c = np.array([0.2, -0.4])
    u = np.stack([k * c[:, None, None] * np.ones((2,) + shape) for k in frames])
    St = objective.evaluate(flat, u, frames, 1.0, p)["St"]
    assert St == pytest.approx(0.5 * 1.3 * 3 * np.prod(shape) * float(c @ c), rel=1e-13)


def test_penalty_closed_forms():
    shape, h = (4, 6), 2.0
    p = Params(alpha=0.0, lam=2.5)
    flat = np.zeros((3,) + shape)
    rng = np.random.default_rng(13)
    u = rng.normal(size=(3, 2) + shape)
    u -= u.mean(axis=0, keepdims=True)
    assert objective.evaluate(flat, u, [0, 1, 2], h, p)["P"] == pytest.approx(0.0, abs=1e-25)
    t = np.array([0.3, -1.1])
    u = np.broadcast_to(t[None, :, None, None], (3, 2) + shape).copy()
    P = objective.evaluate(flat, u, [0, 1, 2], h, p)["P"]
    assert P == pytest.approx(2.5 * h ** 2 * np.prod(shape) * float(t @ t), rel=1e-13)
