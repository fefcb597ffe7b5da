"""Pins of the oracle's temporal predictors (Sec. 3 linear rule, eq. 2)."""
import numpy as np
import pytest

from oracle import grid, predictor


def test_linear_predictor_midpoint_rule():
    K = [0, 4, 8]
    yK = np.array([[1.0], [3.0], [-1.0]])
    z = predictor.predict_linear(yK, K, [0, 2, 4, 6, 8])
    assert np.allclose(z[:, 0], [1.0, 2.0, 3.0, 1.0, -1.0])   # 0.5/0.5 at midpoints


@pytest.mark.parametrize("n,Q", [(17, 4), (16, 2), (200, 3)])
def test_linear_predictor_reproduces_temporally_linear_fields(n, Q):
    rng = np.random.default_rng(0)
    a, b = rng.normal(size=(2, 3, 5)), rng.normal(size=(2, 3, 5))
    truth = np.stack([a + b * k for k in range(n)])
    sets = grid.temporal_sets(n, Q)
    for q in range(Q - 1):
        K, nxt = sets[q], sets[q + 1]
        z = predictor.predict_linear(truth[K], K, nxt)
        assert np.allclose(z, truth[nxt], atol=1e-12)


def _ls_objective(zeta, eta, omega, K, beta):
    """Eq. (2) written term by term (n-1 consecutive differences)."""
    n = omega.shape[0]
    fit = sum((zeta[k] - eta[i]) ** 2 for i, k in enumerate(K))
    smooth = sum(((zeta[k + 1] - zeta[k]) - (omega[k + 1] - omega[k])) ** 2 for k in range(n - 1))
    return fit + beta * smooth


@pytest.mark.parametrize("beta", [1e-5, 0.3, 7.0])
def test_ls_predictor_minimises_eq2(beta):
    """First-order condition of eq. (2), by central differences of the sum itself."""
    rng = np.random.default_rng(1)
    n, K = 13, [0, 3, 4, 9, 12]
    eta, omega = rng.normal(size=len(K)), rng.normal(size=n)
    zeta = predictor.predict_ls(eta, omega, K, beta)
    eps = 1e-6
    for k in range(n):
        e = np.zeros(n)
        e[k] = eps
        gk = (_ls_objective(zeta + e, eta, omega, K, beta)
              - _ls_objective(zeta - e, eta, omega, K, beta)) / (2 * eps)
        assert abs(gk) < 1e-7
    # and it is a minimum: random perturbations increase the objective
    f0 = _ls_objective(zeta, eta, omega, K, beta)
    for _ in range(20):
        assert _ls_objective(zeta + 1e-3 * rng.normal(size=n), eta, omega, K, beta) > f0


def test_thomas_equals_dense_solve():
    rng = np.random.default_rng(2)
    n, K = 40, grid.temporal_sets(40, 3)[0]
    eta, omega = rng.normal(size=(len(K), 2, 6)), rng.normal(size=(n, 2, 6))
    for beta in (1e-5, 1.0, 1e3):
        zt = predictor.predict_ls(eta, omega, K, beta, "thomas")
        zd = predictor.predict_ls(eta, omega, K, beta, "dense")
        assert np.allclose(zt, zd, rtol=1e-12, atol=1e-12 * np.abs(zd).max())


def test_ls_constant_offset_is_exact_for_any_beta():
    rng = np.random.default_rng(3)
    n, K = 21, [0, 5, 10, 15, 20]
    omega = rng.normal(size=(n, 4))
    c = rng.normal(size=4)
    eta = omega[K] + c
    for beta in (1e-5, 1.0, 1e4):
        assert np.allclose(predictor.predict_ls(eta, omega, K, beta), omega + c, atol=1e-11)
    # eta = omega on K -> zeta = omega
    assert np.allclose(predictor.predict_ls(omega[K], omega, K, 0.5), omega, atol=1e-13)


def test_ls_limits_in_beta():
    rng = np.random.default_rng(4)
    n, K = 17, [0, 4, 8, 12, 16]
    omega = rng.normal(size=n)
    eta = rng.normal(size=len(K))
    # beta -> 0: zeta - omega interpolates (eta - omega) linearly between K frames
    z0 = predictor.predict_ls(eta, omega, K, 1e-10)
    lin = np.interp(np.arange(n), K, eta - omega[K])
    assert np.allclose(z0 - omega, lin, atol=1e-6)
    # beta -> infinity: the correction becomes the constant mean over K of (eta - omega)
    zi = predictor.predict_ls(eta, omega, K, 1e10)
    assert np.allclose(zi - omega, np.mean(eta - omega[K]), atol=1e-6)


def test_ls_single_frame_and_full_set():
    omega = np.array([[1.0], [2.0], [4.0]])
    # K = all frames and tiny beta: zeta ~ eta
    eta = np.array([[0.0], [5.0], [1.0]])
    z = predictor.predict_ls(eta, omega, [0, 1, 2], 1e-12)
    assert np.allclose(z, eta, atol=1e-9)
    z1 = predictor.predict_ls(np.array([[3.0]]), np.array([[2.0]]), [0], 0.1)
    assert np.allclose(z1, [[3.0]])
