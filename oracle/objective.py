"""Groupwise objective of eq. (1), its gradient and Gauss-Newton Hessian product.

Readings (the paper names the terms but leaves their discretisation to FAIR):

* Distance (eq. 1): the pairwise sum over all ordered pairs (i, j) of K with
  ``D(a, b) = hd/(4|K|) ||a - b||^2`` (sum of squared differences on the grid,
  ``hd`` = cell volume).  This equals ``hd/2 sum_k ||a_k - mean_j a_j||^2``;
  :func:`distance_pairwise` spells out the double sum and
  :func:`distance_to_mean` the residual form used everywhere else.
* Regulariser S (Sec. 2): diffusion, ``alpha/2 hd sum_k sum_c sum_i ||d_i u_{k,c}||^2``
  with forward differences ``d_i`` between neighbouring cell centres (interior
  edges only), plus an optional temporal first difference
  ``alpha_t/2 hd sum ||u_k' - u_k||^2 / (k' - k)^2`` over consecutive frames of K.
* Penalty P (Sec. 2, displayed formula after eq. 1):
  ``lambda hd ||(1/|K|) sum_j u_j||^2`` (``y_j - Id = u_j``).

Arrays: images ``T`` (|K|, *m); fields ``u`` (|K|, d, *m); ``frames`` the
sorted frame numbers of K (only the temporal term uses them).
"""
from __future__ import annotations

from typing import Dict, Sequence

import numpy as np

from . import grid
from .params import Params


# ---------------------------------------------------------------------------
# distance
# ---------------------------------------------------------------------------
def distance_pairwise(a: np.ndarray, hd: float) -> float:
    """Eq. (1) distance term as the literal double sum over i, j in K."""
    K = a.shape[0]
    tot = 0.0
    for i in range(K):
        for j in range(K):
            tot += hd / (4.0 * K) * float(np.sum((a[i] - a[j]) ** 2))
    return tot


def residual(a: np.ndarray) -> np.ndarray:
    """r_k = a_k - mean_j a_j (per pixel)."""
    return a - a.mean(axis=0, keepdims=True)


def distance_to_mean(a: np.ndarray, hd: float) -> float:
    return 0.5 * hd * float(np.sum(residual(a) ** 2))


# ---------------------------------------------------------------------------
# spatial diffusion regulariser
# ---------------------------------------------------------------------------
def forward_diff(w: np.ndarray, axis: int, h: float) -> np.ndarray:
    """(w[j+1] - w[j]) / h along ``axis`` (interior edges only)."""
    return np.diff(w, axis=axis) / h


def forward_diff_T(e: np.ndarray, axis: int, h: float) -> np.ndarray:
    """Transpose of :func:`forward_diff`: out[j] = (e[j-1] - e[j]) / h with
    the missing edge terms at both ends dropped."""
    shape = list(e.shape)
    shape[axis] += 1
    out = np.zeros(shape)
    lo = [slice(None)] * e.ndim
    hi = [slice(None)] * e.ndim
    lo[axis] = slice(0, -1)
    hi[axis] = slice(1, None)
    out[tuple(lo)] -= e / h
    out[tuple(hi)] += e / h
    return out


def diffusion_energy(w: np.ndarray, h: float) -> float:
    """sum_i ||d_i w||^2 for one scalar plane."""
    return float(sum(np.sum(forward_diff(w, ax, h) ** 2) for ax in range(w.ndim)))


def diffusion_operator(w: np.ndarray, h: float) -> np.ndarray:
    """B^T B w = sum_i d_i^T d_i w (negative Laplacian, homogeneous Neumann)."""
    out = np.zeros_like(w)
    for ax in range(w.ndim):
        out += forward_diff_T(forward_diff(w, ax, h), ax, h)
    return out


def diffusion_diag(shape: Sequence[int], h: float) -> np.ndarray:
    """Diagonal of B^T B: (number of neighbours inside the grid) / h^2."""
    out = np.zeros(tuple(shape))
    for ax, s in enumerate(shape):
        cnt = np.full(s, 2.0)
        cnt[0] -= 1.0
        cnt[-1] -= 1.0
        if s == 1:
            cnt[:] = 0.0
        sh = [1] * len(shape)
        sh[ax] = s
        out += cnt.reshape(sh)
    return out / (h * h)


# ---------------------------------------------------------------------------
# temporal first difference over consecutive frames of K
# ---------------------------------------------------------------------------
def temporal_pairs(frames: Sequence[int]):
    return [(i, i + 1, 1.0 / float(frames[i + 1] - frames[i]) ** 2)
            for i in range(len(frames) - 1)]


def temporal_energy(u: np.ndarray, frames: Sequence[int]) -> float:
    return float(sum(w * np.sum((u[j] - u[i]) ** 2) for i, j, w in temporal_pairs(frames)))


def temporal_operator(v: np.ndarray, frames: Sequence[int]) -> np.ndarray:
    """Gradient of temporal_energy/2: sum over neighbours of w (v_k - v_k')."""
    out = np.zeros_like(v)
    for i, j, w in temporal_pairs(frames):
        out[i] += w * (v[i] - v[j])
        out[j] += w * (v[j] - v[i])
    return out


def temporal_diag(frames: Sequence[int]) -> np.ndarray:
    out = np.zeros(len(frames))
    for i, j, w in temporal_pairs(frames):
        out[i] += w
        out[j] += w
    return out


# ---------------------------------------------------------------------------
# objective, gradient, Hessian product
# ---------------------------------------------------------------------------
def evaluate(T: np.ndarray, u: np.ndarray, frames: Sequence[int], h: float, p: Params,
             want_grad: bool = True) -> Dict:
    """J = D + S + P at u, and (optionally) its gradient and grad T o y.

    Gradient w.r.t. u_k (per pixel and component):
    ``hd r_k grad T_k(y_k) + alpha hd B^T B u_k + alpha_t hd (temporal) + 2 lambda hd ubar/|K|``.
    """
    K, d = u.shape[0], u.shape[1]
    hd = h ** d
    a = np.empty_like(T)
    dT = np.empty_like(u)
    for k in range(K):
        a[k], dT[k] = grid.warp(T[k], u[k], h)
    r = residual(a)
    D = 0.5 * hd * float(np.sum(r * r))
    Sx = 0.5 * p.alpha * hd * sum(diffusion_energy(u[k, c], h) for k in range(K) for c in range(d))
    St = 0.5 * p.alpha_t * hd * temporal_energy(u, frames)
    ubar = u.mean(axis=0)
    P = p.lam * hd * float(np.sum(ubar * ubar))
    out = dict(J=D + Sx + St + P, D=D, S=Sx + St, Sx=Sx, St=St, P=P, a=a, r=r, dT=dT)
    if want_grad:
        g = hd * r[:, None] * dT
        for k in range(K):
            for c in range(d):
                g[k, c] += p.alpha * hd * diffusion_operator(u[k, c], h)
        if p.alpha_t:
            g += p.alpha_t * hd * temporal_operator(u, frames)
        g += (2.0 * p.lam * hd / K) * ubar[None]
        out["g"] = g
    return out


def hessvec(dT: np.ndarray, v: np.ndarray, frames: Sequence[int], h: float, p: Params) -> np.ndarray:
    """Gauss-Newton Hessian times v (J^T J v + alpha B^T B v + ...).

    ``(Hv)_k = hd grad T_k (s_k - sbar) + alpha hd B^T B v_k + alpha_t hd (L_t v)_k
    + (2 lambda hd / |K|^2) sum_j v_j`` with ``s_k = grad T_k . v_k``; the first
    term is J^T J v for the residual r = (I - 11^T/|K|) a, whose Jacobian is
    (I - 11^T/|K|) diag(grad T_k).
    """
    K, d = v.shape[0], v.shape[1]
    hd = h ** d
    s = np.sum(dT * v, axis=1)                      # (K, *m)
    Hv = hd * dT * (s - s.mean(axis=0, keepdims=True))[:, None]
    for k in range(K):
        for c in range(d):
            Hv[k, c] += p.alpha * hd * diffusion_operator(v[k, c], h)
    if p.alpha_t:
        Hv += p.alpha_t * hd * temporal_operator(v, frames)
    Hv += (2.0 * p.lam * hd / K ** 2) * v.sum(axis=0)[None]
    return Hv


def jacobi_diag(dT: np.ndarray, frames: Sequence[int], h: float, p: Params) -> np.ndarray:
    """Diagonal of the Hessian used by :func:`hessvec` (Jacobi preconditioner)."""
    K, d = dT.shape[0], dT.shape[1]
    hd = h ** d
    diag = hd * (1.0 - 1.0 / K) * dT * dT
    diag += p.alpha * hd * diffusion_diag(dT.shape[2:], h)[None, None]
    if p.alpha_t:
        diag += p.alpha_t * hd * temporal_diag(frames).reshape((K, 1) + (1,) * (dT.ndim - 2))
    diag += 2.0 * p.lam * hd / K ** 2
    return diag
