"""Temporal predictors of the spatio-temporal multilevel strategy (Sec. 3).

* :func:`predict_linear` -- coarsest spatial level: injection of the fields
  registered on K_q and linear interpolation in time for the frames in between
  (Sec. 3, the 0.5/0.5 rule between left(k) and right(k)).  For a frame that is
  not midway between its neighbours (the appended last frame makes such gaps)
  the weights are the linear-interpolation weights ((r-k), (k-l)) / (r-l),
  which reduce to 0.5/0.5 at midpoints.
* :func:`predict_ls` -- finer spatial levels: eq. (2), for every pixel and
  displacement component independently,
  ``min_zeta sum_{k in K_q} (zeta_k - eta_k)^2
       + beta sum_{k=0}^{n-2} [(zeta_{k+1} - zeta_k) - (omega_{k+1} - omega_k)]^2``.
  (The printed upper limit n-1 with zeta_{k+1} would reach past the last of n
  frames; the sum runs over the n-1 consecutive differences.)  Writing
  ``e = zeta - omega`` the normal equations are ``(D_K + beta L) e = D_K (eta - omega)``
  with ``D_K`` the 0/1 indicator of K_q on the diagonal and ``L`` the n-by-n
  second-difference matrix tridiag(-1, [1, 2, ..., 2, 1], -1): a tridiagonal
  system solved by Thomas' algorithm (Sec. 3, O(n)) or, to check it, densely.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np


def predict_linear(yK: np.ndarray, K: Sequence[int], targets: Sequence[int]) -> np.ndarray:
    """Fields at ``targets`` from fields ``yK`` (|K|, ...) registered on frames K."""
    K = list(K)
    out = np.empty((len(targets),) + yK.shape[1:])
    for t, k in enumerate(targets):
        if k in K:
            out[t] = yK[K.index(k)]
            continue
        left = max(z for z in K if z < k)
        right = min(z for z in K if z > k)
        wl = (right - k) / (right - left)
        wr = (k - left) / (right - left)
        out[t] = wl * yK[K.index(left)] + wr * yK[K.index(right)]
    return out


def ls_system(n: int, K: Sequence[int], beta: float):
    """Tridiagonal (sub, diag, super) of D_K + beta L, each of length n."""
    diag = np.zeros(n)
    for k in K:
        diag[k] += 1.0
    sub = np.zeros(n)
    sup = np.zeros(n)
    for k in range(n - 1):              # one term per consecutive difference
        diag[k] += beta
        diag[k + 1] += beta
        sup[k] -= beta
        sub[k + 1] -= beta
    return sub, diag, sup


def thomas(sub: np.ndarray, diag: np.ndarray, sup: np.ndarray, rhs: np.ndarray) -> np.ndarray:
    """Solve the tridiagonal system for every column of rhs (n, ...) at once.

    Forward elimination without pivoting, then back substitution; safe here
    because D_K + beta L is symmetric positive definite and weakly diagonally
    dominant.
    """
    n = diag.shape[0]
    cp = np.zeros(n)
    dp = np.zeros_like(rhs)
    cp[0] = sup[0] / diag[0]
    dp[0] = rhs[0] / diag[0]
    for k in range(1, n):
        den = diag[k] - sub[k] * cp[k - 1]
        cp[k] = sup[k] / den
        dp[k] = (rhs[k] - sub[k] * dp[k - 1]) / den
    x = np.zeros_like(rhs)
    x[n - 1] = dp[n - 1]
    for k in range(n - 2, -1, -1):
        x[k] = dp[k] - cp[k] * x[k + 1]
    return x


def ls_rhs(eta: np.ndarray, omega: np.ndarray, K: Sequence[int]) -> np.ndarray:
    rhs = np.zeros_like(omega)
    for i, k in enumerate(K):
        rhs[k] = eta[i] - omega[k]
    return rhs


def predict_ls(eta: np.ndarray, omega: np.ndarray, K: Sequence[int], beta: float,
               method: str = "thomas") -> np.ndarray:
    """Minimiser zeta (n, ...) of eq. (2) for eta (|K|, ...) and omega (n, ...)."""
    n = omega.shape[0]
    sub, diag, sup = ls_system(n, K, beta)
    rhs = ls_rhs(eta, omega, K)
    if method == "thomas":
        e = thomas(sub, diag, sup, rhs)
    elif method == "dense":
        A = np.diag(diag) + np.diag(sub[1:], -1) + np.diag(sup[:-1], 1)
        e = np.linalg.solve(A, rhs.reshape(n, -1)).reshape(rhs.shape)
    else:
        raise ValueError(method)
    return omega + e
