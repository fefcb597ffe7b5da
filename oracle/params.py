"""Parameters of the oracle (its own copy; nothing is shared with the CUDA path)."""
from __future__ import annotations

from dataclasses import dataclass, replace


@dataclass
class Params:
    # objective (Sec. 2): regulariser weights, penalty weight
    alpha: float = 0.02        # spatial diffusion weight
    alpha_t: float = 0.0       # temporal first-difference weight (the paper uses none)
    lam: float = 1.0           # lambda of the mean-transform penalty P
    # predictor (eq. 2) and temporal stopping rule (eq. 3)
    beta: float = 1e-5
    eps_stop: float = 1e-3
    stop_rule: bool = True
    # multilevel structure
    n_levels: int = 2          # spatial levels
    n_tlevels: int = 2         # temporal levels Q (q = 0..Q-1)
    # Gauss-Newton / PCG / Armijo
    tol_J: float = 1e-3
    tol_Y: float = 1e-2
    tol_G: float = 5e-2
    max_gn: int = 40           # a safeguard: the GIRs end on the stopping tests below it
    tol_cg: float = 1e-1
    max_cg: int = 20
    max_ls: int = 10
    armijo_c: float = 1e-4
    g_abs: float = 1e-12       # ||g|| below g_abs (1 + |J0|) counts as stationary
    # target objective of the last GIR over all frames on the finest level
    # (0: none): it stops where J first reaches target_J, within target_tol
    target_J: float = 0.0
    target_tol: float = 1e-5
    # distance of the affine variant: "ssd" (eq. 1 as in the non-parametric
    # path) or "nc" (normalised-correlation reading of the SqN distance, Sec. 2)
    distance: str = "ssd"
    # displacement grid: the unknowns of every level live on its image grid
    # coarsened by 2^u_coarsen per axis and are prolonged onto the image grid
    # (0: the image grid itself); see :mod:`ugrid`
    u_coarsen: int = 0

    def with_(self, **kw) -> "Params":
        return replace(self, **kw)
