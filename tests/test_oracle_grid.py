"""Pins of the oracle's grid layer: temporal tree, interpolation, transfer operators."""
import json
import os

import numpy as np
import pytest

from oracle import grid

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------- temporal tree
def test_temporal_tree_fig1():
    g = json.load(open(os.path.join(GOLDEN, "temporal_tree.json")))["fig1_n17"]
    sets = grid.temporal_sets(g["n"], 4)
    one_based = [[k + 1 for k in K] for K in sets]
    assert one_based[0] == g["K0"]
    assert one_based[1] == g["K1"]
    assert one_based[-1] == g["KT"]


def test_temporal_tree_sec4_sizes():
    g = json.load(open(os.path.join(GOLDEN, "temporal_tree.json")))["sec4_n129"]
    sets = grid.temporal_sets(g["n"], 4)
    assert [len(K) for K in sets] == [g["K0_size"], g["K1_size"], 65, g["KT_size"]]


def test_temporal_tree_nested_and_uneven():
    sets = grid.temporal_sets(200, 3)
    assert [len(K) for K in sets] == [51, 101, 200]
    for a, b in zip(sets[:-1], sets[1:]):
        assert set(a) <= set(b)
    assert sets[0][-2:] == [196, 199]
    assert grid.temporal_sets(1, 3) == [[0], [0], [0]]
    assert grid.temporal_sets(2, 3) == [[0, 1]] * 3


# --------------------------------------------------------------- interpolation
def _affine_image(shape, h, a, b):
    x = grid.cell_centres(shape, h)
    return np.tensordot(a, x, axes=(0, 0)) + b


@pytest.mark.parametrize("shape,h", [((9, 13), 1.0), ((6, 5), 2.0), ((4, 5, 6), 1.0)])
def test_interpolation_exact_on_affine_images(shape, h):
    rng = np.random.default_rng(0)
    d = len(shape)
    a = rng.normal(size=d)
    T = _affine_image(shape, h, a, 0.3)
    # random points inside the hull of the cell centres
    lo = 0.5 * h
    hi = (np.asarray(shape) - 0.5) * h
    pts = np.stack([rng.uniform(lo, hi[c], size=500) for c in range(d)])
    val, gr = grid.interpolate(T, h, pts)
    assert np.allclose(val, np.tensordot(a, pts, axes=(0, 0)) + 0.3, rtol=0, atol=1e-12)
    for c in range(d):
        assert np.allclose(gr[c], a[c], rtol=0, atol=1e-12)


def test_interpolation_at_grid_points_returns_samples():
    rng = np.random.default_rng(1)
    T = rng.normal(size=(7, 8))
    x = grid.cell_centres(T.shape, 2.0)
    val, _ = grid.interpolate(T, 2.0, x)
    assert np.array_equal(val, T)


def test_interpolation_zero_extension_hand_cases():
    T = np.array([[1.0, 2.0, 4.0]])          # one row of 3 cells, h = 1
    # centres at 0.5, 1.5, 2.5 along axis 1; axis 0 at its centre 0.5
    def at(x1):
        v, g = grid.interpolate(T, 1.0, np.array([[0.5], [x1]]))
        return v[0], g[1][0]
    v, g = at(0.0)          # half a cell left of the first centre: blend of 0 and 1
    assert v == pytest.approx(0.5) and g == pytest.approx(1.0)
    v, g = at(-0.5)         # xi = -1: the sample at i0 = -1 is 0; the derivative is T[0] - 0
    assert v == pytest.approx(0.0) and g == pytest.approx(1.0)
    v, g = at(-0.6)
    assert v == 0.0 and g == 0.0
    v, g = at(3.0)          # half a cell right of the last centre
    assert v == pytest.approx(2.0) and g == pytest.approx(-4.0)
    v, g = at(1.5)          # integer xi: the cell to the right is used for the derivative
    assert v == pytest.approx(2.0) and g == pytest.approx(2.0)
    # and the other axis sees zero outside too: the row above is empty
    v, _ = grid.interpolate(T, 1.0, np.array([[0.0], [1.5]]))
    assert v[0] == pytest.approx(1.0)


# --------------------------------------------------------------- transfer ops
def test_restriction_preserves_constant_and_affine():
    shape_f, h_f = (8, 12), 1.0
    a = np.array([0.7, -1.3])
    Tf = _affine_image(shape_f, h_f, a, 2.0)
    Tc = grid.restrict(Tf)
    assert np.allclose(Tc, _affine_image((4, 6), 2.0, a, 2.0), atol=1e-12)
    assert np.allclose(grid.restrict(np.full((4, 4, 4), 3.0)), 3.0)


def test_prolongation_1d_worked_example():
    uc = np.array([[1.0, 5.0]])            # 1 x 2 coarse cells -> 2 x 4 fine cells
    uf = grid.prolong(uc)
    row = np.array([1.0, 0.75 * 1 + 0.25 * 5, 0.25 * 1 + 0.75 * 5, 5.0])
    assert np.allclose(uf, np.stack([row, row]))


def test_prolongation_constant_and_affine_interior():
    a = np.array([0.4, -0.9, 0.2])
    uc = _affine_image((4, 5, 6), 2.0, a, 1.0)
    uf = grid.prolong(uc)
    ref = _affine_image((8, 10, 12), 1.0, a, 1.0)
    inner = (slice(1, -1),) * 3
    assert np.allclose(uf[inner], ref[inner], atol=1e-12)
    assert np.allclose(grid.prolong(np.full((3, 3), -2.0)), -2.0)


@pytest.mark.parametrize("shape", [(5, 7), (3, 4, 2), (1, 6)])
def test_prolongation_adjoint(shape):
    rng = np.random.default_rng(2)
    u = rng.normal(size=shape)
    w = rng.normal(size=tuple(2 * s for s in shape))
    lhs = float(np.sum(grid.prolong(u) * w))
    rhs = float(np.sum(u * grid.prolong_adjoint(w)))
    assert lhs == pytest.approx(rhs, rel=1e-13, abs=1e-13)
