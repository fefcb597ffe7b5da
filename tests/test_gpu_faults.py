"""Failure detection without a GPU fault: non-finite data, an Armijo failure
and a bounded device wait that runs out each end in a status the host reads,
and the context stays usable."""
import numpy as np
import pytest

from _util import cuda_lib
from paper_2001_06613_gb300 import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    return cuda_lib()


def _run(S, R, **kw):
    import torch
    ctx = S.Context(S.stml_default_params(n_levels=2, n_tlevels=2, **kw))
    try:
        S.stml_load_sequence(ctx.ptr, torch.from_numpy(R).cuda())
        S.stml_build_pyramid(ctx.ptr)
        stats = S.stml_register(ctx.ptr, 0)
        # the context stays usable: a second registration of clean data works
        S.stml_load_sequence(ctx.ptr, torch.from_numpy(synthetic.make_sequence(synthetic.spec_tiny(seed=9))).cuda())
        S.stml_build_pyramid(ctx.ptr)
        again = S.stml_register(ctx.ptr, 0)
    finally:
        ctx.close()
    return stats, again


def test_nan_in_the_data_is_reported_not_a_crash(S):
    R = synthetic.make_sequence(synthetic.spec_tiny(seed=8))
    R[5, 30, 30] = np.nan
    stats, again = _run(S, R)
    assert any(s["status"] == -4 for s in stats), [s["status"] for s in stats]     # STML_ENONFINITE
    assert all(s["status"] == 0 for s in again)


def test_armijo_failure_ends_the_gir_with_a_status(S):
    """With c = 0.99 and a single trial the full Gauss-Newton step cannot pass
    (it decreases J by about half of the linear prediction)."""
    R = synthetic.make_sequence(synthetic.spec_tiny(seed=10))
    stats, again = _run(S, R, max_ls=1, armijo_c=0.99)
    assert any(s["status"] == -6 for s in stats), [s["status"] for s in stats]     # STML_ELINESEARCH
    assert all(np.isfinite(s["J"]) for s in stats)


def test_a_device_wait_that_nothing_completes_gives_up(S):
    import torch
    assert S.stml_check_bounded_wait() is True
    torch.cuda.synchronize()                      # the context is still usable
    assert float(torch.ones(4, device="cuda").sum()) == 4.0
