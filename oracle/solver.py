"""Gauss-Newton / PCG / Armijo: the registration scheme GIR on a frame subset.

The paper registers with FAIR's L-BFGS (Sec. 2) and allows "any numerical
optimization scheme".  This oracle (like the library) uses a matrix-free
Gauss-Newton method on the displacement fields of all frames in K:

1. evaluate J and its gradient g at u;
2. stop (the three FAIR-style tests below) or continue;
3. solve H d = -g approximately by Jacobi-preconditioned conjugate gradients
   started at 0 (stop when ||r|| <= tol_cg ||g|| or after max_cg steps; if a
   search direction has p^T H p <= 0 the iterate so far is returned, or the
   preconditioned gradient step when that happens on the first step);
4. Armijo back-tracking on t in {1, 1/2, 1/4, ...}:
   accept the first t with J(u + t d) <= J(u) + c t g^T d (at most max_ls trials);
5. u <- u + t d, go to 1.

Stopping after iteration i >= 1 when all of
|J_old - J| <= tol_J (1 + |J0|), ||t d|| <= tol_Y (1 + ||u||),
||g|| <= tol_G (1 + |J0|) hold, or at once when ||g|| <= g_abs (1 + |J0|),
or when max_gn iterations were taken.

Target objective (a measurement device, not part of the paper's method: it
makes registrations that follow different paths end at the same objective):
with a target J* > 0 the loop stops as soon as an accepted step reaches
J <= J*, after shortening that step so that J(u + t d) = J* within
target_tol J* (Illinois regula falsi on t between 0 and the accepted step);
a start with J0 <= J* takes no step.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, Sequence

import numpy as np

from . import objective
from .params import Params


def pcg(apply_H: Callable[[np.ndarray], np.ndarray], b: np.ndarray, Minv: np.ndarray,
        tol: float, maxit: int, record: list | None = None, flip: int | None = None):
    """Jacobi-preconditioned CG for H x = b from x = 0; returns (x, steps, flag).

    With ``record`` given, ||r|| / ||b|| after every step is appended to it
    (the quantity the stopping test compares with ``tol``).  ``flip`` = k
    inverts the stopping decision taken after step k + 1 (the other branch of
    a decision whose ratio sits within rounding of ``tol``: several results
    of the method are then correct, and a test may compare with either)."""
    x = np.zeros_like(b)
    bnorm = float(np.sqrt(np.sum(b * b)))
    if bnorm == 0.0:
        return x, 0, "zero-rhs"
    r = b.copy()
    z = Minv * r
    p = z.copy()
    rho = float(np.sum(r * z))
    steps = 0
    flag = "maxit"
    while steps < maxit:
        q = apply_H(p)
        pq = float(np.sum(p * q))
        if pq <= 0.0:
            if steps == 0:
                x = z.copy()
            flag = "breakdown"
            break
        alpha = rho / pq
        x += alpha * p
        r -= alpha * q
        steps += 1
        if record is not None:
            record.append(float(np.sqrt(np.sum(r * r))) / bnorm)
        stop = float(np.sqrt(np.sum(r * r))) <= tol * bnorm
        if flip is not None and steps - 1 == flip:
            stop = not stop
        if stop:
            flag = "converged"
            break
        z = Minv * r
        rho_new = float(np.sum(r * z))
        beta = rho_new / rho
        rho = rho_new
        p = z + beta * p
    return x, steps, flag


def armijo(phi: Callable[[float], float], J: float, gTd: float, c: float, max_ls: int):
    """Back-tracking line search with the sufficient-decrease test of Armijo.

    phi(t) is the objective at u + t d, J = phi(0) and gTd the directional
    derivative <g, d> < 0.  Trial k takes t = 2^-k and accepts when
    phi(t) <= J + c t gTd; at most max_ls trials.  Returns (t, trials, accepted);
    on failure t is the last step tried.
    """
    t = 1.0
    for k in range(max_ls):
        if phi(t) <= J + c * t * gTd:
            return t, k + 1, True
        if k + 1 < max_ls:
            t *= 0.5
    return t, max_ls, False


def land(phi: Callable[[float], float], J_start: float, t_acc: float, J_acc: float, target: float,
         tol: float, max_it: int = 40):
    """Step length t in (0, t_acc] with |phi(t) - target| <= tol * target.

    phi(0) = J_start > target >= J_acc = phi(t_acc).  Regula falsi with the
    Illinois modification (the retained end's function value is halved when
    the same end is kept twice in a row).  Returns (t, phi(t), evaluations);
    after max_it evaluations the point of smallest |phi - target| seen."""
    a, fa = 0.0, J_start - target
    b, fb = t_acc, J_acc - target
    best = (abs(fb), b, J_acc)
    if abs(fb) <= tol * target:
        return b, J_acc, 0
    side = 0
    for i in range(max_it):
        t = (a * fb - b * fa) / (fb - fa)
        Jt = phi(t)
        ft = Jt - target
        if abs(ft) < best[0]:
            best = (abs(ft), t, Jt)
        if abs(ft) <= tol * target:
            return t, Jt, i + 1
        if ft > 0.0:
            a, fa = t, ft
            if side == 1:
                fb *= 0.5
            side = 1
        else:
            b, fb = t, ft
            if side == -1:
                fa *= 0.5
            side = -1
    return best[1], best[2], max_it


@dataclass
class GirStats:
    J: float = 0.0
    D: float = 0.0
    S: float = 0.0
    P: float = 0.0
    J0: float = 0.0
    gn_iters: int = 0
    cg_iters: int = 0
    ls_trials: int = 0
    status: str = "ok"
    landing_evals: int = 0                          # objective evaluations of the target landing
    history: list = field(default_factory=list)    # (J, ||g||) at every iterate
    steps: list = field(default_factory=list)      # (CG steps, Armijo trials) of every GN step
    cg_residuals: list = field(default_factory=list)   # ||r|| / ||g|| after each CG step, per solve

    def cg_margin(self, tol: float) -> float:
        """Smallest relative distance |ratio - tol| / tol of any CG stopping
        decision of this GIR from its threshold (inf without CG steps): how
        far the solve is from a decision that FP32 rounding could flip."""
        r = [abs(x - tol) / tol for rec in self.cg_residuals for x in rec]
        return min(r) if r else float("inf")


class ImageGridModel:
    """Eq. (1) with S and P over the fields of the frames in K on the image
    grid of the level (the default reading): what the Gauss-Newton loop
    evaluates.  Another discretisation of the unknowns provides the same three
    methods (``evaluate``, ``hessvec``, ``jacobi``)."""

    def __init__(self, T: np.ndarray, frames: Sequence[int], h: float, p: Params):
        self.T, self.frames, self.h, self.p = T, frames, h, p

    def evaluate(self, u: np.ndarray, want_grad: bool = True) -> dict:
        return objective.evaluate(self.T, u, self.frames, self.h, self.p, want_grad=want_grad)

    def hessvec(self, dT: np.ndarray, v: np.ndarray) -> np.ndarray:
        return objective.hessvec(dT, v, self.frames, self.h, self.p)

    def jacobi(self, dT: np.ndarray) -> np.ndarray:
        return objective.jacobi_diag(dT, self.frames, self.h, self.p)


def gauss_newton(T: np.ndarray, u0: np.ndarray, frames: Sequence[int], h: float, p: Params,
                 target: float = 0.0, model=None, flips=None):
    """GIR(K): minimise eq. (1) over the fields of the frames in K, from u0
    (with target > 0: until J reaches the target objective, see above).
    ``model`` replaces the image-grid objective (:class:`ImageGridModel`).
    ``flips``: set of (solve, k) -- the CG stopping decision after step k + 1
    of the solve-th PCG solve of this GIR takes its other branch (see
    :func:`pcg`)."""
    mdl = model if model is not None else ImageGridModel(T, frames, h, p)
    u = np.array(u0, dtype=np.float64, copy=True)
    ev = mdl.evaluate(u)
    J0 = ev["J"]
    st = GirStats(J0=J0)
    J, g = ev["J"], ev["g"]
    J_old = None
    step_norm = None
    it = 0
    if target > 0.0 and J0 <= target:
        st.status = "target"
        st.J, st.D, st.S, st.P = ev["J"], ev["D"], ev["S"], ev["P"]
        return u, st
    while True:
        gnorm = float(np.sqrt(np.sum(g * g)))
        st.history.append((J, gnorm))
        if it > 0:
            c1 = abs(J_old - J) <= p.tol_J * (1.0 + abs(J0))
            c2 = step_norm <= p.tol_Y * (1.0 + float(np.sqrt(np.sum(u * u))))
            c3 = gnorm <= p.tol_G * (1.0 + abs(J0))
            if c1 and c2 and c3:
                break
        if gnorm <= p.g_abs * (1.0 + abs(J0)) or it >= p.max_gn:
            break
        Minv = 1.0 / mdl.jacobi(ev["dT"])
        dT = ev["dT"]
        rec = []
        solve = len(st.cg_residuals)
        fk = [k for (si, k) in (flips or ()) if si == solve]
        d, steps, _ = pcg(lambda v: mdl.hessvec(dT, v), -g, Minv,
                          p.tol_cg, p.max_cg, rec, fk[0] if fk else None)
        st.cg_residuals.append(rec)
        st.cg_iters += steps
        gTd = float(np.sum(g * d))
        if not gTd < 0.0:
            st.status = "no-descent"
            break
        t, trials, accepted = armijo(
            lambda s: mdl.evaluate(u + s * d, want_grad=False)["J"],
            J, gTd, p.armijo_c, p.max_ls)
        st.ls_trials += trials
        st.steps.append((steps, trials))
        if not accepted:
            st.status = "line-search"
            break
        if target > 0.0:
            Jt = mdl.evaluate(u + t * d, want_grad=False)["J"]
            if Jt <= target:
                t, _, st.landing_evals = land(
                    lambda s: mdl.evaluate(u + s * d, want_grad=False)["J"],
                    J, t, Jt, target, p.target_tol)
                u = u + t * d
                ev = mdl.evaluate(u)
                it += 1
                st.status = "target"
                break
        u = u + t * d
        step_norm = t * float(np.sqrt(np.sum(d * d)))
        J_old = J
        ev = mdl.evaluate(u)
        J, g = ev["J"], ev["g"]
        it += 1
    st.J, st.D, st.S, st.P = ev["J"], ev["D"], ev["S"], ev["P"]
    st.gn_iters = it
    return u, st
