"""Batched registration of several sequences of uneven length and size
(stml_register_batch): results equal stml_register on each context alone, and
contexts that may launch cooperative solves are refused before any work."""
import numpy as np
import pytest

from _util import cuda_lib
from paper_2001_06613_gb300 import synthetic

pytestmark = pytest.mark.gpu

SEQS = [(6, (32, 32), 41), (9, (48, 40), 42), (16, (64, 64), 43), (12, (40, 48), 44), (20, (32, 48), 45)]


@pytest.fixture(scope="module")
def S():
    return cuda_lib()


def _make(S, n, shape, seed, stream=None, **kw):
    import torch
    R = synthetic.make_sequence(synthetic.spec_custom(n, shape, seed=seed, amp=1.5))
    prm = S.stml_default_params(n_levels=2, n_tlevels=2, pcg_cooperative=0, **kw)
    ctx = S.Context(prm, stream)
    S.stml_load_sequence(ctx.ptr, torch.from_numpy(R).cuda())
    S.stml_build_pyramid(ctx.ptr)
    return ctx


def _field(S, ctx, n, shape):
    y = np.empty((n, len(shape)) + shape, np.float32)
    S.stml_get_field(ctx.ptr, 1, y)
    return y


@pytest.mark.parametrize("mode", [0, 1])
def test_batch_equals_sequential(S, mode):
    import torch
    ref = []
    for n, shape, seed in SEQS:
        ctx = _make(S, n, shape, seed)
        try:
            S.stml_register(ctx.ptr, mode)
            ref.append(_field(S, ctx, n, shape))
        finally:
            ctx.close()
    streams = [torch.cuda.Stream() for _ in SEQS]
    ctxs = [_make(S, n, shape, seed, st.cuda_stream) for (n, shape, seed), st in zip(SEQS, streams)]
    try:
        status = S.stml_register_batch(ctxs, mode, max_threads=3)
        assert status == [0] * len(SEQS)
        for (n, shape, _), ctx, y in zip(SEQS, ctxs, ref):
            assert np.array_equal(_field(S, ctx, n, shape), y)
    finally:
        for c in ctxs:
            c.close()


def test_batch_refuses_cooperative_contexts(S):
    import torch
    streams = [torch.cuda.Stream() for _ in range(2)]
    a = _make(S, 6, (32, 32), 46, streams[0].cuda_stream)
    b = _make(S, 6, (32, 32), 47, streams[1].cuda_stream, )
    try:
        S.stml_set_params(b.ptr, S.stml_default_params(n_levels=2, n_tlevels=2, pcg_cooperative=1))
        with pytest.raises(S.StmlError) as e:
            S.stml_register_batch([a, b], 0)
        assert e.value.status == -1
        with pytest.raises(S.StmlError):
            S.stml_register_batch([a, a], 0)   # the same context (and stream) twice
    finally:
        a.close()
        b.close()
