"""Spatio-temporal multilevel (STML) and spatial-only multilevel (SpML) drivers.

STML (Sec. 3): for every spatial level l from coarse to fine, a
predictor-corrector sweep over the temporal sets K_0 ... K_T:

* start values: Id (u = 0) on the coarsest level; otherwise the prolongated
  fields of all frames from level l-1 (z_{l,0} = P y_{l-1,T,all});
* correct: y_{l,q} = GIR(l, K_q) from z_{l,q} restricted to K_q;
* stop (eq. 3): for q > 0, if the per-frame distance D(y_{l,q})/|K_q| changed
  by at most eps relative to D(y_{l,q-1})/|K_{q-1}| the frames outside K_q are
  filled by the predictor and the level ends (the absolute D of eq. (3) sums
  over different numbers of frames; comparing per-frame values relative to
  the previous one is this implementation's reading of the rule);
* predict: z_{l,q+1} by :func:`predictor.predict_linear` on the coarsest level
  and by :func:`predictor.predict_ls` (eq. 2, eta = y_{l,q}, omega = z_{l,q})
  on the others;
* after q = T every frame has been registered: y_{l,all} = y_{l,T}.

SpML: one GIR over all frames per level, started from the prolongated result
of the previous level (Id on the coarsest).

With ``p.u_coarsen = s > 0`` the fields of every level live on its image grid
coarsened by 2^s per axis (:mod:`ugrid`); the drivers are unchanged (the
level-to-level prolongation and the predictors act on those grids, which
halve from level to level like the images).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np

from . import grid, objective, predictor, solver, ugrid
from .params import Params


def pyramid(R: np.ndarray, n_levels: int) -> List[np.ndarray]:
    """Images of all frames at every spatial level; index 0 is the coarsest."""
    levels = [np.asarray(R, dtype=np.float64)]
    for _ in range(n_levels - 1):
        levels.append(grid.restrict_frames(levels[-1]))
    return levels[::-1]


@dataclass
class LevelStats:
    level: int
    tlevel: int
    n_frames: int
    gn_iters: int
    cg_iters: int
    ls_trials: int
    J: float
    D: float
    S: float
    P: float
    stopped_early: bool = False
    cg_margin: float = float("inf")    # see solver.GirStats.cg_margin
    cg_residuals: list = field(default_factory=list)   # ||r|| / ||g|| after each CG step, per solve


@dataclass
class Result:
    y: np.ndarray                        # finest-level fields of all frames (n, d, *m)
    stats: List[LevelStats] = field(default_factory=list)
    fields: List[np.ndarray] = field(default_factory=list)   # y_{l,all} per level


def _fill(ell: int, yK, K, z_all, beta):
    n = z_all.shape[0]
    if ell == 0:
        out = predictor.predict_linear(yK, K, list(range(n)))
    else:
        out = predictor.predict_ls(yK, z_all, K, beta)
        out[list(K)] = yK
    return out


def _model(T, K, h, p: Params):
    """The objective of a GIR: None (image-grid fields) or the coarse-grid model."""
    return ugrid.Model(T, K, h, p.u_coarsen, p) if p.u_coarsen else None


def register(R: np.ndarray, p: Params, mode: str = "stml", flips=None) -> Result:
    """``flips``: {GIR index: set of (solve, k)} -- CG stopping decisions that
    take their other branch (:func:`solver.gauss_newton`); GIRs are numbered
    in the order they run."""
    n = R.shape[0]
    d = R.ndim - 1
    L = p.n_levels
    pyr = pyramid(R, L)
    sets = grid.temporal_sets(n, p.n_tlevels)
    allK = list(range(n))
    res = Result(y=None)
    y_prev = None
    for ell in range(L):
        T = pyr[ell]
        h = grid.level_h(L, ell)
        m = tuple(x // 2 ** p.u_coarsen for x in T.shape[1:])   # grid of the fields
        z_all = np.zeros((n, d) + m) if ell == 0 else grid.prolong_fields(y_prev)
        target = p.target_J if ell == L - 1 else 0.0     # the last GIR over all frames
        if mode == "spml":
            y_all, st = solver.gauss_newton(T, z_all, allK, h, p, target, _model(T, allK, h, p),
                                            (flips or {}).get(len(res.stats)))
            res.stats.append(LevelStats(ell, p.n_tlevels - 1, n, st.gn_iters, st.cg_iters,
                                        st.ls_trials, st.J, st.D, st.S, st.P,
                                        cg_margin=st.cg_margin(p.tol_cg), cg_residuals=st.cg_residuals))
        elif mode == "stml":
            y_all = None
            dhat_prev = None
            for q, K in enumerate(sets):
                yK, st = solver.gauss_newton(T[K], z_all[K], K, h, p,
                                             target if q == len(sets) - 1 else 0.0, _model(T[K], K, h, p),
                                             (flips or {}).get(len(res.stats)))
                dhat = st.D / len(K)
                stop = (q > 0 and p.stop_rule and
                        abs(dhat - dhat_prev) <= p.eps_stop * abs(dhat_prev))
                res.stats.append(LevelStats(ell, q, len(K), st.gn_iters, st.cg_iters,
                                            st.ls_trials, st.J, st.D, st.S, st.P, stop,
                                            cg_margin=st.cg_margin(p.tol_cg), cg_residuals=st.cg_residuals))
                if q == len(sets) - 1:
                    y_all = yK
                    break
                if stop:
                    y_all = _fill(ell, yK, K, z_all, p.beta)
                    break
                if ell == 0:
                    nxt = sets[q + 1]
                    z_all[nxt] = predictor.predict_linear(yK, K, nxt)
                else:
                    z_all = predictor.predict_ls(yK, z_all, K, p.beta)
                dhat_prev = dhat
        else:
            raise ValueError(mode)
        res.fields.append(y_all)
        y_prev = y_all
    res.y = y_prev
    return res


def final_objective(R: np.ndarray, y: np.ndarray, p: Params) -> dict:
    """J, D, S, P over all frames on the finest level at fields y."""
    n = R.shape[0]
    if p.u_coarsen:
        ev = ugrid.evaluate(np.asarray(R, dtype=np.float64), y, list(range(n)), 1.0, p.u_coarsen, p,
                            want_grad=False)
        return {k: ev[k] for k in ("J", "D", "S", "P")}
    ev = objective.evaluate(np.asarray(R, dtype=np.float64), y, list(range(n)), 1.0, p,
                            want_grad=False)
    return {k: ev[k] for k in ("J", "D", "S", "P")}


def corr_coeff(R: np.ndarray) -> np.ndarray:
    """Correlation coefficient of consecutive frames (Sec. 4, Table 1 column 3)."""
    out = []
    for k in range(R.shape[0] - 1):
        a = R[k].ravel() - R[k].mean()
        b = R[k + 1].ravel() - R[k + 1].mean()
        out.append(float(a @ b / np.sqrt((a @ a) * (b @ b))))
    return np.array(out)
