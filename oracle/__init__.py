"""FP64 CPU oracle for spatio-temporal multilevel (STML) registration.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
restatement of the method that the CUDA library is checked against.  Only the
test-suite, the smoke check in ``__graft_entry__`` and the CPU-baseline leg of
``bench.py`` may import it; the library itself never does, and it shares no
code with the CUDA path (the seeded input generator lives in its own module).

Layout of the oracle:

* ``grid``       -- cell-centred grids, linear interpolation with zero
                    extension, spatial restriction/prolongation (and the
                    prolongation's transpose), the temporal binary tree (Fig. 1).
* ``objective``  -- groupwise distance (eq. 1 with the sum-of-squares reading),
                    diffusion regulariser, mean-transform penalty (Sec. 2),
                    gradient, Gauss-Newton Hessian product, Jacobi diagonal.
* ``solver``     -- PCG, Armijo back-tracking and the Gauss-Newton loop that
                    stands in for the paper's GIR (Sec. 2).
* ``predictor``  -- the coarse-level linear predictor (Sec. 3) and the
                    least-squares predictor of eq. (2), by Thomas' algorithm and
                    by a dense solve.
* ``ugrid``      -- displacements on a grid 2^s times coarser than the images:
                    the prolongation P_s, its transpose (the gradient's
                    adjoint gather) and the objective, Hessian product and
                    Jacobi diagonal of the unknowns on that grid.
* ``multilevel`` -- image pyramid, STML predictor-corrector driver with the
                    stopping rule of eq. (3), and the spatial-only (SpML) driver.
* ``affine``     -- affine-linear transformations per frame (Sec. 4) solved by
                    L-BFGS (Sec. 2): parametrisation, projected gradient,
                    two-loop recursion, and the STML/SpML drivers over the
                    parameters.
* ``net``        -- the learned temporal predictor: a convolutional
                    encoder-decoder proposing a skipped frame's field from its
                    two registered neighbours and three images (in place of
                    the predictors of Sec. 3 where the objective says it is
                    better), its MSE loss, gradient and Adam update, with an
                    optional BF16 rounding of the convolution operands.

Every function works in float64 on numpy arrays.  Where the paper is silent the
oracle follows one stated reading, documented on the function.
"""
from .params import Params  # noqa: F401
from . import grid, objective, solver, predictor, multilevel, net, affine, ugrid  # noqa: F401
