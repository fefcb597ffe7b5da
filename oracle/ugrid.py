"""Displacements on a grid coarser than the images (the optional m_u = m / 2^s).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper leaves the discretisation of the transformation to FAIR (Sec. 2:
"any other meaningful registration strategy").  In the default reading the
unknown field of every frame lives on the image grid of its level.  This
module is the reading in which the unknowns w_k live on the grid of cell
width F h, F = 2^s (s >= 1), and the field that warps the image is its
prolongation onto the image grid:

    u_k = P_s w_k,  P_s = cell-centred multilinear interpolation from the
    F-times coarser grid, clamp-to-edge (per axis: fine cell j has its centre
    at coarse index coordinate xi = (j + 1/2)/F - 1/2 and takes
    (1 - f) w[clamp(i0)] + f w[clamp(i0 + 1)], i0 = floor(xi), f = xi - i0).

For F = 2 this is the level-to-level prolongation of :mod:`grid`.

Objective over the frames of K (eq. (1) with S and P of Sec. 2):

    J(w) = D(P_s w) + S_w(w) + P_w(w)

* D is the distance of eq. (1) evaluated with the fields u = P_s w on the
  image grid (cell width h, cell volume hd = h^d), as in :mod:`objective`;
* S_w and P_w are the regulariser and penalty of :mod:`objective` evaluated
  on the grid of w itself (cell width h_w = F h, cell volume hd_w = h_w^d):
  the same continuous energies, discretised where the unknowns live.

Gradient:  g = P_s^T (hd r_k grad T_k) + alpha hd_w B^T B w_k
               + alpha_t hd_w (L_t w)_k + 2 lambda hd_w wbar / |K|.
Gauss-Newton Hessian:  H v = P_s^T H_D (P_s v) + alpha hd_w B^T B v + ...,
with H_D the distance part of the image-grid Hessian.  Because H_D couples
only values at the same pixel, diag(P_s^T H_D P_s) = (P_s o P_s)^T diag(H_D)
exactly (o: element-wise product), which gives the Jacobi preconditioner.

P_s is a tensor product of one matrix per axis, so P_s^T and (P_s o P_s)^T
are tensor products of the transposed and squared axis matrices.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np

from . import objective
from .params import Params


def axis_matrix(m_fine: int, F: int) -> np.ndarray:
    """(m_fine, m_fine // F) matrix of the interpolation along one axis."""
    mc = m_fine // F
    A = np.zeros((m_fine, mc))
    for j in range(m_fine):
        xi = (j + 0.5) / F - 0.5
        i0 = int(np.floor(xi))
        f = xi - i0
        A[j, min(max(i0, 0), mc - 1)] += 1.0 - f
        A[j, min(max(i0 + 1, 0), mc - 1)] += f
    return A


def _apply(mats: Sequence[np.ndarray], x: np.ndarray) -> np.ndarray:
    """Apply mats[a] along the a-th of the last len(mats) axes of x."""
    nd = len(mats)
    out = x
    for a, A in enumerate(mats):
        ax = out.ndim - nd + a
        out = np.moveaxis(np.tensordot(A, out, axes=([1], [ax])), 0, ax)
    return out


def prolong(w: np.ndarray, fine_shape: Sequence[int], s: int) -> np.ndarray:
    """u = P_s w over the trailing spatial axes of w (any leading axes)."""
    F = 2 ** s
    return _apply([axis_matrix(m, F) for m in fine_shape], w)


def adjoint(u: np.ndarray, fine_shape: Sequence[int], s: int) -> np.ndarray:
    """P_s^T u: every coarse value gathers the fine values it was blended into."""
    F = 2 ** s
    return _apply([axis_matrix(m, F).T for m in fine_shape], u)


def adjoint_sq(u: np.ndarray, fine_shape: Sequence[int], s: int) -> np.ndarray:
    """(P_s o P_s)^T u (squared interpolation weights)."""
    F = 2 ** s
    return _apply([(axis_matrix(m, F) ** 2).T for m in fine_shape], u)


def _data_params(p: Params) -> Params:
    """The image-grid objective with only its distance term."""
    return p.with_(alpha=0.0, alpha_t=0.0, lam=0.0)


def evaluate(T: np.ndarray, w: np.ndarray, frames: Sequence[int], h: float, s: int, p: Params,
             want_grad: bool = True) -> dict:
    """J, D, S, P at the coarse fields w (|K|, d, *m/F) for images T (|K|, *m).

    The returned ``dT`` is grad T at the warped positions on the image grid
    (what :func:`hessvec` and :func:`jacobi_diag` need)."""
    K, d = w.shape[0], w.shape[1]
    m = T.shape[1:]
    hw = h * 2 ** s
    hdw = hw ** d
    u = prolong(w, m, s)
    ev = objective.evaluate(T, u, frames, h, _data_params(p), want_grad=want_grad)
    Sx = 0.5 * p.alpha * hdw * sum(objective.diffusion_energy(w[k, c], hw) for k in range(K) for c in range(d))
    St = 0.5 * p.alpha_t * hdw * objective.temporal_energy(w, frames)
    wbar = w.mean(axis=0)
    P = p.lam * hdw * float(np.sum(wbar * wbar))
    out = dict(J=ev["D"] + Sx + St + P, D=ev["D"], S=Sx + St, Sx=Sx, St=St, P=P, dT=ev["dT"], u=u)
    if want_grad:
        g = adjoint(ev["g"], m, s)
        for k in range(K):
            for c in range(d):
                g[k, c] += p.alpha * hdw * objective.diffusion_operator(w[k, c], hw)
        if p.alpha_t:
            g += p.alpha_t * hdw * objective.temporal_operator(w, frames)
        g += (2.0 * p.lam * hdw / K) * wbar[None]
        out["g"] = g
    return out


def hessvec(dT: np.ndarray, v: np.ndarray, frames: Sequence[int], h: float, s: int, p: Params) -> np.ndarray:
    """Gauss-Newton Hessian of :func:`evaluate` times v (coarse fields)."""
    K, d = v.shape[0], v.shape[1]
    m = dT.shape[2:]
    hw = h * 2 ** s
    hdw = hw ** d
    Hv = adjoint(objective.hessvec(dT, prolong(v, m, s), frames, h, _data_params(p)), m, s)
    for k in range(K):
        for c in range(d):
            Hv[k, c] += p.alpha * hdw * objective.diffusion_operator(v[k, c], hw)
    if p.alpha_t:
        Hv += p.alpha_t * hdw * objective.temporal_operator(v, frames)
    Hv += (2.0 * p.lam * hdw / K ** 2) * v.sum(axis=0)[None]
    return Hv


def jacobi_diag(dT: np.ndarray, frames: Sequence[int], h: float, s: int, p: Params) -> np.ndarray:
    """Diagonal of the Hessian of :func:`hessvec`: (P_s o P_s)^T of the image-grid
    distance diagonal plus the regulariser and penalty diagonal on the coarse grid."""
    K, d = dT.shape[0], dT.shape[1]
    m = dT.shape[2:]
    hd = h ** d
    hw = h * 2 ** s
    hdw = hw ** d
    cshape = tuple(x // 2 ** s for x in m)
    diag = adjoint_sq(hd * (1.0 - 1.0 / K) * dT * dT, m, s)
    diag += p.alpha * hdw * objective.diffusion_diag(cshape, hw)[None, None]
    if p.alpha_t:
        diag += p.alpha_t * hdw * objective.temporal_diag(frames).reshape((K, 1) + (1,) * len(m))
    diag += 2.0 * p.lam * hdw / K ** 2
    return diag


class Model:
    """The coarse-grid objective of one frame subset, in the form the
    Gauss-Newton loop of :mod:`solver` takes (``model=``)."""

    def __init__(self, T: np.ndarray, frames: Sequence[int], h: float, s: int, p: Params):
        self.T, self.frames, self.h, self.s, self.p = T, list(frames), h, s, p

    def evaluate(self, w: np.ndarray, want_grad: bool = True) -> dict:
        return evaluate(self.T, w, self.frames, self.h, self.s, self.p, want_grad)

    def hessvec(self, dT: np.ndarray, v: np.ndarray) -> np.ndarray:
        return hessvec(dT, v, self.frames, self.h, self.s, self.p)

    def jacobi(self, dT: np.ndarray) -> np.ndarray:
        return jacobi_diag(dT, self.frames, self.h, self.s, self.p)
