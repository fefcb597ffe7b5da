"""Affine-linear registration by L-BFGS: the setting of the paper's experiments.

TEST INFRASTRUCTURE ONLY (like the rest of this package).

Sec. 4 registers the frames by affine-linear transformations, and Sec. 2
minimises eq. (1) with FAIR's L-BFGS.  Readings (the paper names both and
leaves their details to FAIR):

* Parametrisation.  Frame k's transformation is y_k(x) = x + u_k(x) with
  ``u_k(x) = W_k (x - c) / rho + b_k``: x a cell centre in finest-level pixel
  units ((j + 1/2) h on level l), c the centre of the domain, rho half of its
  largest extent, W_k a d x d matrix and b_k a d-vector (both in pixels, so
  the map's matrix is A_k = I + W_k / rho).  theta_k = (W_k row by row, b_k):
  d (d + 1) parameters, the same on every spatial level (prolongation is the
  identity).  The scaling by rho gives all parameters pixel units, which is
  what L-BFGS's scaled-identity initial Hessian needs.
* Objective.  The same J = D + S + P as the non-parametric path (eq. 1,
  Sec. 2) evaluated at the affine fields, so its gradient is the projection
  ``dJ/dtheta_k = sum_x Phi(x)^T (dJ/du_k)(x)`` with Phi(x) = [xhat^T, 1] for
  each component.
* Distance.  Sec. 2 names a correlation-based measure, the SVD-based SqN
  distance of its reference [Kai2019], whose definition is not in the paper.
  Reading (p.distance = "nc"): with a_k = T_k o y_k, centred a_k - mean(a_k),
  normalised m_k and rho_ij = <m_i, m_j>,
  ``D_NC = 1/2 sum_{i, j in K} (1 - rho_ij^2) = 1/2 (|K|^2 - ||M^T M||_F^2)``,
  i.e. one half of |K|^2 minus the fourth power of the Schatten-4 norm of the
  matrix M of normalised frames (sum of sigma^4 of its singular values): it
  vanishes when all frames agree up to per-frame brightness and contrast.
  S and P stay as in eq. (1).
* L-BFGS (Nocedal & Wright, Algorithm 7.4 two-loop recursion with
  H0 = gamma I, gamma = s^T y / y^T y of the newest pair; memory m; a pair
  with s^T y <= 1e-12 |s| |y| is not stored).  The first step (and any step
  after a direction that is not a descent direction, which also clears the
  memory) is -g scaled to move no parameter by more than one pixel.  Armijo
  back-tracking t = 1, 1/2, ... (c = armijo_c, max_ls trials) and the FAIR
  stopping tests of the Gauss-Newton solver in theta-space (tol_J, tol_Y on
  |t d| against 1 + |theta|, tol_G, g_abs, at most max_it iterations).
* Multilevel.  STML and SpML as in multilevel.py with theta in place of the
  fields: no prolongation, linear predictor on the coarsest level, eq. (2)
  (per parameter) on finer ones, stopping rule eq. (3).
"""
from __future__ import annotations

from dataclasses import dataclass, field as dc_field
from typing import Callable, List, Sequence

import numpy as np

from . import grid, objective, predictor
from .params import Params


def n_params(d: int) -> int:
    return d * (d + 1)


def coords(shape: Sequence[int], h: float, fine: Sequence[int]) -> np.ndarray:
    """xhat = (x - c) / rho at the cell centres x of a level of ``shape`` and
    cell width h; c and rho from the finest shape ``fine``."""
    d = len(shape)
    x = grid.cell_centres(shape, h)
    c = np.asarray(fine, dtype=np.float64).reshape((d,) + (1,) * d) / 2.0
    rho = max(fine) / 2.0
    return (x - c) / rho


def field(theta: np.ndarray, xhat: np.ndarray) -> np.ndarray:
    """u_k = W_k xhat + b_k for theta (K, d(d+1)): (K, d, *m)."""
    d = xhat.shape[0]
    theta = np.asarray(theta, dtype=np.float64)
    K = theta.shape[0]
    out = np.empty((K, d) + xhat.shape[1:])
    for k in range(K):
        W = theta[k, :d * d].reshape(d, d)
        b = theta[k, d * d:]
        for c in range(d):
            out[k, c] = b[c] + sum(W[c, i] * xhat[i] for i in range(d))
    return out


def project(v: np.ndarray, xhat: np.ndarray) -> np.ndarray:
    """Adjoint of :func:`field`: (K, d(d+1)) with entries sum_x v_{k,c}(x) xhat_i(x)
    (the W part) and sum_x v_{k,c}(x) (the b part)."""
    d = xhat.shape[0]
    K = v.shape[0]
    out = np.empty((K, n_params(d)))
    for k in range(K):
        for c in range(d):
            for i in range(d):
                out[k, c * d + i] = float(np.sum(v[k, c] * xhat[i]))
            out[k, d * d + c] = float(np.sum(v[k, c]))
    return out


def nc_distance(a: np.ndarray):
    """D_NC of the warped frames a (K, *m) and dD_NC/da (same shape).

    With c = mean-free a, n_k = |c_k|, m_k = c_k / n_k, rho = M M^T:
    dD/dm_i = -2 sum_j rho_ij m_j, and through the centring and normalisation
    dD/da_i = -(2 / n_i) (sum_j rho_ij m_j - m_i sum_j rho_ij^2)."""
    K = a.shape[0]
    A = a.reshape(K, -1)
    C = A - A.mean(axis=1, keepdims=True)
    n = np.linalg.norm(C, axis=1)
    M = C / n[:, None]
    R = M @ M.T
    D = 0.5 * (K * K - float(np.sum(R * R)))
    s = np.sum(R * R, axis=1)
    G = -(2.0 / n[:, None]) * (R @ M - M * s[:, None])
    return D, G.reshape(a.shape)


def evaluate(T: np.ndarray, theta: np.ndarray, frames: Sequence[int], h: float, xhat: np.ndarray,
             p: Params, want_grad: bool = True) -> dict:
    """J, D, S, P at the affine fields of theta and dJ/dtheta (key "g")."""
    u = field(theta, xhat)
    ev = objective.evaluate(T, u, frames, h, p, want_grad=want_grad)
    if p.distance == "nc":
        D, Ga = nc_distance(ev["a"])
        out = dict(J=D + ev["S"] + ev["P"], D=D, S=ev["S"], P=ev["P"])
        if want_grad:
            hd = h ** u.shape[1]
            g_reg = ev["g"] - hd * ev["r"][:, None] * ev["dT"]      # S and P terms of dJ/du
            out["g"] = project(Ga[:, None] * ev["dT"] + g_reg, xhat)
        return out
    out = {k: ev[k] for k in ("J", "D", "S", "P")}
    if want_grad:
        out["g"] = project(ev["g"], xhat)
    return out


# ---------------------------------------------------------------------------
# L-BFGS
# ---------------------------------------------------------------------------
@dataclass
class LbfgsStats:
    J: float = 0.0
    J0: float = 0.0
    iters: int = 0
    evals: int = 0
    ls_trials: int = 0
    status: str = "ok"
    extra: dict = dc_field(default_factory=dict)


def two_loop(g: np.ndarray, S: List[np.ndarray], Y: List[np.ndarray]) -> np.ndarray:
    """H g by the two-loop recursion over the stored pairs (oldest first)."""
    q = g.copy()
    alphas = []
    for s, y in reversed(list(zip(S, Y))):
        rho = 1.0 / float(y @ s)
        a = rho * float(s @ q)
        alphas.append((a, rho))
        q -= a * y
    s, y = S[-1], Y[-1]
    r = (float(s @ y) / float(y @ y)) * q
    for (s, y), (a, rho) in zip(zip(S, Y), reversed(alphas)):
        bta = rho * float(y @ r)
        r += (a - bta) * s
    return r


def lbfgs(fun: Callable, x0: np.ndarray, p: Params, m: int = 5, max_it: int = 50):
    """Minimise fun(x) -> (J, g, extra) from x0 (flat); returns (x, LbfgsStats)."""
    x = np.array(x0, dtype=np.float64).ravel()
    J, g, extra = fun(x)
    st = LbfgsStats(J0=J, evals=1)
    J0 = J
    S: List[np.ndarray] = []
    Y: List[np.ndarray] = []
    J_old = None
    step = None
    it = 0
    while True:
        gnorm = float(np.linalg.norm(g))
        if it > 0:
            c1 = abs(J_old - J) <= p.tol_J * (1.0 + abs(J0))
            c2 = step <= p.tol_Y * (1.0 + float(np.linalg.norm(x)))
            c3 = gnorm <= p.tol_G * (1.0 + abs(J0))
            if c1 and c2 and c3:
                break
        if gnorm <= p.g_abs * (1.0 + abs(J0)) or it >= max_it:
            break
        d = -two_loop(g, S, Y) if S else None
        if d is None or not float(g @ d) < 0.0:
            S, Y = [], []
            d = -g / float(np.abs(g).max())
        gTd = float(g @ d)
        t = 1.0
        accepted = False
        for _ in range(p.max_ls):
            st.ls_trials += 1
            Jt, gt, et = fun(x + t * d)
            st.evals += 1
            if Jt <= J + p.armijo_c * t * gTd:
                accepted = True
                break
            t *= 0.5
        if not accepted:
            st.status = "line-search"
            break
        s = t * d
        y = gt - g
        if float(s @ y) > 1e-12 * float(np.linalg.norm(s) * np.linalg.norm(y)):
            S.append(s)
            Y.append(y)
            if len(S) > m:
                S.pop(0)
                Y.pop(0)
        x = x + s
        step = float(np.linalg.norm(s))
        J_old = J
        J, g, extra = Jt, gt, et
        it += 1
    st.J, st.iters, st.extra = J, it, extra
    return x, st


def gir(T: np.ndarray, theta0: np.ndarray, frames: Sequence[int], h: float, xhat: np.ndarray, p: Params,
        m: int = 5, max_it: int = 50):
    """GIR(K) over the affine parameters of the frames in K, from theta0 (K, P)."""
    K, P = np.asarray(theta0).shape

    def fun(x):
        ev = evaluate(T, x.reshape(K, P), frames, h, xhat, p)
        return ev["J"], ev["g"].ravel(), ev

    x, st = lbfgs(fun, np.asarray(theta0, dtype=np.float64).ravel(), p, m, max_it)
    return x.reshape(K, P), st


# ---------------------------------------------------------------------------
# multilevel drivers
# ---------------------------------------------------------------------------
@dataclass
class LevelStats:
    level: int
    tlevel: int
    n_frames: int
    iters: int
    J: float
    D: float
    stopped_early: bool = False


def register(R: np.ndarray, p: Params, mode: str = "stml", m: int = 5, max_it: int = 50):
    """Affine STML / SpML: theta (n, d(d+1)) of all frames and per-GIR stats."""
    from .multilevel import pyramid
    n = R.shape[0]
    d = R.ndim - 1
    L = p.n_levels
    pyr = pyramid(R, L)
    sets = grid.temporal_sets(n, p.n_tlevels)
    allK = list(range(n))
    fine = R.shape[1:]
    theta_all = np.zeros((n, n_params(d)))
    stats: List[LevelStats] = []
    for ell in range(L):
        T = pyr[ell]
        h = grid.level_h(L, ell)
        xh = coords(T.shape[1:], h, fine)
        if mode == "spml":
            theta_all, st = gir(T, theta_all, allK, h, xh, p, m, max_it)
            stats.append(LevelStats(ell, len(sets) - 1, n, st.iters, st.J, st.extra["D"]))
            continue
        z = theta_all.copy()
        dhat_prev = None
        for q, K in enumerate(sets):
            tK, st = gir(T[K], z[K], K, h, xh, p, m, max_it)
            dhat = st.extra["D"] / len(K)
            stop = q > 0 and p.stop_rule and abs(dhat - dhat_prev) <= p.eps_stop * abs(dhat_prev)
            stats.append(LevelStats(ell, q, len(K), st.iters, st.J, st.extra["D"], stop))
            if q == len(sets) - 1:
                theta_all = tK
                break
            if stop:
                if ell == 0:
                    theta_all = predictor.predict_linear(tK, K, allK)
                else:
                    theta_all = predictor.predict_ls(tK, z, K, p.beta)
                    theta_all[list(K)] = tK
                break
            if ell == 0:
                nxt = sets[q + 1]
                z[nxt] = predictor.predict_linear(tK, K, nxt)
            else:
                z = predictor.predict_ls(tK, z, K, p.beta)
            dhat_prev = dhat
    return theta_all, stats
