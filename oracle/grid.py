"""Grids, linear interpolation, spatial transfer operators, temporal tree.

Conventions (readings of the paper, which builds on FAIR's grids without
restating them):

* A grid of ``m`` cells per axis at cell width ``h`` (finest-pixel units) has
  cell centres ``x_j = (j + 1/2) h``; level ``l`` of ``L`` spatial levels has
  ``h = 2**(L-1-l)`` (Sec. 3: "spatial discretization levels").
* Displacements ``u`` live at the same cell centres, ``y = x + u`` in physical
  units, so no rescaling happens between levels.
* Frames are numbered 0..n-1.
"""
from __future__ import annotations

import itertools
from typing import List, Sequence, Tuple

import numpy as np


# ---------------------------------------------------------------------------
# temporal binary tree (Sec. 3, Fig. 1)
# ---------------------------------------------------------------------------
def temporal_sets(n: int, n_tlevels: int) -> List[List[int]]:
    """Frame subsets K_0 ... K_T of the temporal binary tree (Sec. 3, Fig. 1).

    K_T holds every frame, K_{T-1} every second one, K_{T-2} every fourth and
    so on; K_q therefore takes frames at stride ``2**(T-q)``.  The first and
    the last frame always belong to every set (for n = 2**p + 1 the last frame
    lies on the stride; otherwise it is appended, the adaptation "to any number
    of images" that Sec. 3 leaves open).
    """
    if n < 1 or n_tlevels < 1:
        raise ValueError("need n >= 1 and at least one temporal level")
    T = n_tlevels - 1
    sets = []
    for q in range(n_tlevels):
        stride = 2 ** (T - q)
        K = list(range(0, n, stride))
        if K[-1] != n - 1:
            K.append(n - 1)
        sets.append(K)
    return sets


# ---------------------------------------------------------------------------
# cell-centred grids
# ---------------------------------------------------------------------------
def level_shape(finest: Sequence[int], n_levels: int, level: int) -> Tuple[int, ...]:
    f = 2 ** (n_levels - 1 - level)
    for s in finest:
        if s % f:
            raise ValueError("grid size must be divisible by 2**(levels-1)")
    return tuple(s // f for s in finest)


def level_h(n_levels: int, level: int) -> float:
    return float(2 ** (n_levels - 1 - level))


def cell_centres(shape: Sequence[int], h: float) -> np.ndarray:
    axes = [(np.arange(s, dtype=np.float64) + 0.5) * h for s in shape]
    return np.stack(np.meshgrid(*axes, indexing="ij"), axis=0)


# ---------------------------------------------------------------------------
# linear interpolation with zero extension (image model of eq. 1: R_i o y_i)
# ---------------------------------------------------------------------------
def interpolate(T: np.ndarray, h: float, pos: np.ndarray):
    """Multilinear interpolant of the cell-centred image ``T`` and its gradient.

    ``pos`` has shape (d, *S) in physical units.  With ``xi = pos/h - 1/2`` the
    point falls in the cell spanned by ``i0 = floor(xi)`` and ``i0 + 1`` along
    every axis; the value is the multilinear blend of those 2**d samples, where
    a sample outside the grid counts as 0 (zero extension).  The gradient is the
    exact derivative of that blend on the cell [i0, i0 + 1]: at an integer
    ``xi`` this is the one-sided derivative towards ``i0 + 1``.
    Returns ``(value (*S), gradient (d, *S))``.
    """
    d = T.ndim
    m = T.shape
    xi = pos / h - 0.5
    i0 = np.floor(xi).astype(np.int64)
    f = xi - i0
    val = np.zeros(pos.shape[1:])
    grad = np.zeros(pos.shape)
    for corner in itertools.product((0, 1), repeat=d):
        idx = [i0[c] + corner[c] for c in range(d)]
        inside = np.ones(pos.shape[1:], dtype=bool)
        for c in range(d):
            inside &= (idx[c] >= 0) & (idx[c] < m[c])
        safe = tuple(np.clip(idx[c], 0, m[c] - 1) for c in range(d))
        sample = np.where(inside, T[safe], 0.0)
        w = [f[c] if corner[c] else 1.0 - f[c] for c in range(d)]
        weight = np.ones(pos.shape[1:])
        for c in range(d):
            weight = weight * w[c]
        val += weight * sample
        for c in range(d):
            dw = np.full(pos.shape[1:], (1.0 if corner[c] else -1.0) / h)
            for c2 in range(d):
                if c2 != c:
                    dw = dw * w[c2]
            grad[c] += dw * sample
    return val, grad


def warp(T: np.ndarray, u: np.ndarray, h: float):
    """Transformed image a = T(x + u(x)) at the cell centres, and grad T there."""
    x = cell_centres(T.shape, h)
    return interpolate(T, h, x + u)


# ---------------------------------------------------------------------------
# spatial transfer operators (Sec. 3; Sec. 4: smoothing only in space)
# ---------------------------------------------------------------------------
def restrict(T: np.ndarray) -> np.ndarray:
    """Coarse image = mean over each block of 2**d fine cells (per frame if 3+ dims given)."""
    d = T.ndim
    out = np.zeros(tuple(s // 2 for s in T.shape))
    for corner in itertools.product((0, 1), repeat=d):
        sl = tuple(slice(corner[c], None, 2) for c in range(d))
        out += T[sl]
    return out / (2 ** d)


def _prolong_stencil(shape_c: Sequence[int]):
    """For each fine cell: the 2**d coarse indices (clamped) and weights.

    Fine cell j (width h/2) has its centre at coarse index coordinate
    xi = j/2 - 1/4; the value there is the multilinear blend of the coarse
    centres floor(xi) and floor(xi)+1, an index beyond the grid replaced by the
    nearest edge cell (clamp-to-edge).
    """
    d = len(shape_c)
    shape_f = tuple(2 * s for s in shape_c)
    jj = np.stack(np.meshgrid(*[np.arange(s) for s in shape_f], indexing="ij"), axis=0)
    xi = jj / 2.0 - 0.25
    i0 = np.floor(xi).astype(np.int64)
    f = xi - i0
    entries = []
    for corner in itertools.product((0, 1), repeat=d):
        idx = tuple(np.clip(i0[c] + corner[c], 0, shape_c[c] - 1) for c in range(d))
        w = np.ones(shape_f)
        for c in range(d):
            w = w * (f[c] if corner[c] else 1.0 - f[c])
        entries.append((idx, w))
    return entries


def prolong(uc: np.ndarray) -> np.ndarray:
    """Cell-centred multilinear prolongation P of one scalar field, clamp-to-edge."""
    out = np.zeros(tuple(2 * s for s in uc.shape))
    for idx, w in _prolong_stencil(uc.shape):
        out += w * uc[idx]
    return out


def prolong_adjoint(wf: np.ndarray) -> np.ndarray:
    """Transpose P^T of :func:`prolong`: every fine value is scattered back to the
    coarse cells it was blended from, with the same weights."""
    shape_c = tuple(s // 2 for s in wf.shape)
    out = np.zeros(shape_c)
    for idx, w in _prolong_stencil(shape_c):
        np.add.at(out, idx, w * wf)
    return out


def prolong_fields(u: np.ndarray) -> np.ndarray:
    """Apply :func:`prolong` to every (frame, component) plane of (n, d, *m)."""
    n, d = u.shape[:2]
    return np.stack([np.stack([prolong(u[k, c]) for c in range(d)]) for k in range(n)])


def restrict_frames(T: np.ndarray) -> np.ndarray:
    return np.stack([restrict(t) for t in T])
