"""GPU parity of the transfer operators and temporal predictors (C ABI vs oracle)."""
import numpy as np
import pytest

from _util import assert_array, cuda_lib
from oracle import grid, predictor

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    return cuda_lib()


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("shape", [(38, 54), (2, 2), (64, 64), (8, 12, 10), (2, 6, 4)])
def test_restrict(S, shape):
    import torch
    rng = np.random.default_rng(0)
    planes = 3
    f = rng.normal(size=(planes,) + shape).astype(np.float32)
    out = torch.empty((planes,) + tuple(s // 2 for s in shape), device="cuda")
    S.stml_restrict(_dev(f), out, planes, shape)
    ref = np.stack([grid.restrict(x.astype(np.float64)) for x in f])
    assert_array(out.cpu().numpy(), ref, 1e-6, "restrict")


@pytest.mark.parametrize("cshape", [(19, 27), (1, 6), (32, 32), (4, 5, 6), (1, 1, 3)])
def test_prolong_and_adjoint(S, cshape):
    import torch
    rng = np.random.default_rng(1)
    planes = 4
    fshape = tuple(2 * s for s in cshape)
    c = rng.normal(size=(planes,) + cshape).astype(np.float32)
    w = rng.normal(size=(planes,) + fshape).astype(np.float32)
    pf = torch.empty((planes,) + fshape, device="cuda")
    S.stml_prolong(_dev(c), pf, planes, cshape)
    assert_array(pf.cpu().numpy(), np.stack([grid.prolong(x.astype(np.float64)) for x in c]), 1e-6, "P")
    pa = torch.empty((planes,) + cshape, device="cuda")
    S.stml_prolong_adjoint(_dev(w), pa, planes, cshape)
    assert_array(pa.cpu().numpy(), np.stack([grid.prolong_adjoint(x.astype(np.float64)) for x in w]), 1e-6, "P^T")
    lhs = float(np.sum(pf.cpu().numpy().astype(np.float64) * w))
    rhs = float(np.sum(c.astype(np.float64) * pa.cpu().numpy()))
    assert abs(lhs - rhs) <= 1e-5 * (abs(lhs) + 1.0)


@pytest.mark.parametrize("n,Q", [(200, 3), (17, 4), (16, 2), (5, 3)])
def test_predict_linear(S, n, Q):
    import torch
    rng = np.random.default_rng(2)
    plane = 1003                       # ragged, not a multiple of 4
    sets = grid.temporal_sets(n, Q)
    for q in range(Q - 1):
        K, nxt = sets[q], sets[q + 1]
        y = rng.normal(size=(len(K), plane)).astype(np.float32)
        z = torch.empty((len(nxt), plane), device="cuda")
        S.stml_predict_linear(_dev(y), K, z, nxt, plane)
        ref = predictor.predict_linear(y.astype(np.float64), K, nxt)
        assert_array(z.cpu().numpy(), ref, 1e-6, f"linear q={q}")
        # frames of K are injected exactly
        got = z.cpu().numpy()
        for i, k in enumerate(K):
            assert np.array_equal(got[nxt.index(k)], y[i])


def test_predict_linear_reproduces_linear_fields(S):
    import torch
    n, Q = 33, 3
    a = np.linspace(-1, 1, 64, dtype=np.float32)
    b = np.float32(0.25)
    truth = np.stack([a + b * k for k in range(n)]).astype(np.float32)
    sets = grid.temporal_sets(n, Q)
    K, nxt = sets[0], sets[1]
    z = torch.empty((len(nxt), 64), device="cuda")
    S.stml_predict_linear(_dev(truth[K]), K, z, nxt, 64)
    assert_array(z.cpu().numpy(), truth[nxt], 1e-6, "linear exact")


@pytest.mark.parametrize("n,Q,q", [(200, 3, 0), (200, 3, 1), (17, 4, 0), (129, 4, 1), (1, 1, 0), (2, 2, 0)])
@pytest.mark.parametrize("beta", [1e-5, 1.0])
def test_predict_ls(S, n, Q, q, beta):
    import torch
    rng = np.random.default_rng(3)
    K = grid.temporal_sets(n, Q)[q]
    ncomp = 2 * 517 + 1
    omega = rng.normal(size=(n, ncomp)).astype(np.float32) * 2
    eta = (omega[K] + rng.normal(size=(len(K), ncomp)) * 0.3).astype(np.float32)
    zeta = torch.empty((n, ncomp), device="cuda")
    S.stml_predict_ls(_dev(eta), K, _dev(omega), zeta, n, beta, ncomp)
    ref = predictor.predict_ls(eta.astype(np.float64), omega.astype(np.float64), K, beta)
    assert_array(zeta.cpu().numpy(), ref, 1e-5, "eq. (2)")


def test_predict_ls_constant_offset_exact(S):
    import torch
    n, K = 40, grid.temporal_sets(40, 3)[0]
    rng = np.random.default_rng(4)
    omega = rng.normal(size=(n, 256)).astype(np.float32)
    c = rng.normal(size=256).astype(np.float32)
    eta = (omega[K] + c).astype(np.float32)
    zeta = torch.empty((n, 256), device="cuda")
    S.stml_predict_ls(_dev(eta), K, _dev(omega), zeta, n, 1e-5, 256)
    assert_array(zeta.cpu().numpy(), omega.astype(np.float64) + c, 2e-6, "offset")


def test_context_free_ops_reject_bad_arguments(S):
    import torch
    x = torch.zeros(16, device="cuda")
    with pytest.raises(S.StmlError):
        S.stml_predict_ls(x, [3, 1], x, torch.zeros(16, device="cuda"), 4, 1.0, 4)
    with pytest.raises(S.StmlError):
        S.stml_restrict(x, x, 1, (3, 4))
