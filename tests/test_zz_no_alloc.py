"""The allocation-free Hessian product (stml_hessvec_noalloc) against the
context entry point (stml_hessvec).

Some callers cannot allocate device memory -- they run inside a framework that
owns all device memory through its own pool, or may only touch the buffers
they are given.  stml_hessvec_noalloc lets them compute the Gauss-Newton
Hessian product with their own input and output buffers and the library's
static scratch array.  Two calls in a row must agree with stml_hessvec (the
second call also checks that the shared scratch left by the first is reset).
This file is collected last on purpose."""
import numpy as np
import pytest

from _util import assert_array, assert_scalar, cuda_lib
from paper_2001_06613_gb300 import synthetic

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("shape,n,frames,extra", [
    ((48, 40), 9, [0, 2, 3, 5, 8], {}),
    ((74, 106), 6, [0, 1, 2, 3, 4, 5], dict(alpha_t=0.3, lambda_=2.0)),
    ((12, 16, 20), 5, [0, 1, 3, 4], {}),
])
def test_noalloc_hessvec_matches_context_entry_point(shape, n, frames, extra):
    import torch
    S = cuda_lib()
    R = synthetic.make_sequence(synthetic.spec_custom(n, shape, seed=31))
    prm = S.stml_default_params(n_levels=1, **extra)
    ctx = S.Context(prm)
    try:
        S.stml_load_sequence(ctx.ptr, _dev(R))
        S.stml_build_pyramid(ctx.ptr)
        rng = np.random.default_rng(12)
        for call in range(2):
            dT = rng.normal(size=(len(frames), len(shape)) + shape).astype(np.float32)
            v = synthetic.random_field(rng, len(frames), len(shape), shape, amp=1.0, rough=0.5)
            ref = torch.empty_like(_dev(v))
            vhv_ref = S.stml_hessvec(ctx.ptr, 0, frames, _dev(dT), _dev(v), ref)
            out = torch.full_like(ref, float("nan"))
            vhv = S.stml_hessvec_noalloc(_dev(dT), _dev(v), out, shape, 1.0, frames, prm)
            torch.cuda.synchronize()
            assert_array(out.cpu().numpy(), ref.cpu().numpy(), what=f"Hv call {call}")
            assert_scalar(vhv, vhv_ref, what=f"<v,Hv> call {call}")
    finally:
        ctx.close()


def test_noalloc_rejects_problems_beyond_the_static_scratch():
    import torch
    S = cuda_lib()
    prm = S.stml_default_params()
    x = torch.zeros(8, device="cuda")
    with pytest.raises(S.StmlError) as e:
        S.stml_hessvec_noalloc(x, x, x, (2048, 2048), 1.0, [0, 1], prm)
    assert e.value.status == -1
    assert "scratch" in S.stml_last_error(None)
