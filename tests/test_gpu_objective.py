"""GPU parity of the objective, gradient, warped-image derivatives and the
Gauss-Newton Hessian product (C ABI vs oracle), including the full
200 x 256 x 256 finest level of the paper-scale workload."""
import numpy as np
import pytest

from _util import assert_array, assert_scalar, cuda_lib
from oracle import Params, grid, multilevel, objective
from paper_2001_06613_gb300 import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    return cuda_lib()


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _ctx(S, R, levels, **kw):
    prm = S.stml_default_params(n_levels=levels, **kw)
    ctx = S.Context(prm)
    S.stml_load_sequence(ctx.ptr, _dev(R))
    S.stml_build_pyramid(ctx.ptr)
    return ctx


def _oracle_params(prm):
    return Params(alpha=prm.alpha, alpha_t=prm.alpha_t, lam=prm.lambda_, beta=prm.beta)


CASES = [
    # shape, n, levels, level, frames, extra params
    ((48, 40), 9, 2, 1, list(range(9)), {}),
    ((48, 40), 9, 2, 0, [0, 4, 8], {}),
    ((48, 40), 9, 2, 1, [3], {}),
    ((74, 106), 7, 2, 0, [0, 2, 3, 6], dict(alpha_t=0.3)),        # level 0 is 37 x 53
    ((64, 64), 16, 2, 1, list(range(16)), dict(alpha=0.5, lambda_=3.0)),
    ((12, 16, 20), 5, 2, 1, [0, 1, 3, 4], {}),                   # 3-D
    ((12, 16, 20), 5, 2, 0, [0, 2, 4], dict(alpha_t=0.2)),
]


@pytest.mark.parametrize("shape,n,levels,level,frames,extra", CASES)
def test_eval_parity(S, shape, n, levels, level, frames, extra):
    import torch
    spec = synthetic.spec_custom(n, shape, seed=5, amp=1.5)
    R = synthetic.make_sequence(spec)
    ctx = _ctx(S, R, levels, **extra)
    try:
        T = multilevel.pyramid(R.astype(np.float64), levels)[level]
        h = grid.level_h(levels, level)
        m = T.shape[1:]
        rng = np.random.default_rng(7)
        u = synthetic.random_field(rng, len(frames), len(m), m, amp=1.2 * h, rough=0.3 * h)
        g = torch.empty((len(frames), len(m)) + m, device="cuda")
        dT = torch.empty_like(g)
        out = S.stml_eval(ctx.ptr, level, frames, _dev(u), g, dT)
        ev = objective.evaluate(T[frames], u.astype(np.float64), frames, h, _oracle_params(ctx.params))
        for i, k in enumerate(("J", "D", "S", "P")):
            assert_scalar(out[i], ev[k], what=k)
        assert_scalar(out[4], float(np.sum(ev["g"] ** 2)), what="|g|^2")
        assert_scalar(out[5], float(np.sum(u.astype(np.float64) ** 2)), what="|u|^2")
        assert_array(dT.cpu().numpy(), ev["dT"], what="grad T")
        assert_array(g.cpu().numpy(), ev["g"], what="gradient")
        obj = S.stml_eval(ctx.ptr, level, frames, _dev(u))
        assert_scalar(obj[0], ev["J"], what="objective-only J")
        assert obj[4] == 0.0
    finally:
        ctx.close()


@pytest.mark.parametrize("with_gd", [True, False])
@pytest.mark.parametrize("shape,n,levels,level,frames,extra", CASES)
def test_eval_trial_parity(S, shape, n, levels, level, frames, extra, with_gd):
    """Armijo trial objective at u + t d in the solver's launch (no array formed),
    with and without <g, d> and |d|^2."""
    spec = synthetic.spec_custom(n, shape, seed=11, amp=1.5)
    R = synthetic.make_sequence(spec)
    ctx = _ctx(S, R, levels, **extra)
    try:
        T = multilevel.pyramid(R.astype(np.float64), levels)[level]
        h = grid.level_h(levels, level)
        m = T.shape[1:]
        rng = np.random.default_rng(12)
        u = synthetic.random_field(rng, len(frames), len(m), m, amp=1.0 * h, rough=0.3 * h)
        d = synthetic.random_field(rng, len(frames), len(m), m, amp=0.5 * h, rough=0.3 * h)
        gd = rng.normal(size=u.shape).astype(np.float32)
        t = 0.5
        out = S.stml_eval_trial(ctx.ptr, level, frames, _dev(u), _dev(d), t, _dev(gd) if with_gd else None)
        ut = u.astype(np.float64) + t * d.astype(np.float64)
        ev = objective.evaluate(T[frames], ut, frames, h, _oracle_params(ctx.params))
        for i, k in enumerate(("J", "D", "S", "P")):
            assert_scalar(out[i], ev[k], what=f"trial {k}")
        assert_scalar(out[5], float(np.sum(ut ** 2)), what="|u + t d|^2")
        if with_gd:
            assert_scalar(out[6], float(np.sum(gd.astype(np.float64) * d)), what="<g, d>")
            assert_scalar(out[7], float(np.sum(d.astype(np.float64) ** 2)), what="|d|^2")
        else:
            assert out[6] == 0.0 and out[7] == 0.0
    finally:
        ctx.close()


@pytest.mark.parametrize("shape,n,levels,level,frames,extra", CASES)
def test_hessvec_parity(S, shape, n, levels, level, frames, extra):
    import torch
    spec = synthetic.spec_custom(n, shape, seed=6, amp=1.0)
    R = synthetic.make_sequence(spec)
    ctx = _ctx(S, R, levels, **extra)
    try:
        h = grid.level_h(levels, level)
        m = grid.level_shape(shape, levels, level)
        rng = np.random.default_rng(8)
        dT = rng.normal(size=(len(frames), len(m)) + m).astype(np.float32)
        v = synthetic.random_field(rng, len(frames), len(m), m, amp=1.0, rough=0.5)
        Hv = torch.empty_like(_dev(v))
        vhv = S.stml_hessvec(ctx.ptr, level, frames, _dev(dT), _dev(v), Hv)
        ref = objective.hessvec(dT.astype(np.float64), v.astype(np.float64), frames, h,
                                _oracle_params(ctx.params))
        assert_array(Hv.cpu().numpy(), ref, what="Hv")
        assert_scalar(vhv, float(np.sum(v.astype(np.float64) * ref)), what="<v,Hv>")
    finally:
        ctx.close()


def test_pyramid_and_correlation(S):
    spec = synthetic.spec_custom(6, (40, 24, 16), seed=9)
    R = synthetic.make_sequence(spec)
    ctx = _ctx(S, R, 3)
    try:
        pyr = multilevel.pyramid(R.astype(np.float64), 3)
        for lvl in range(3):
            out = np.empty((6,) + pyr[lvl].shape[1:], np.float32)
            S.stml_get_images(ctx.ptr, lvl, out)
            assert_array(out, pyr[lvl], 1e-6, f"level {lvl}")
            assert S.stml_level_info(ctx.ptr, lvl)[1] == grid.level_h(3, lvl)
        rho = S.stml_corr_coeff(ctx.ptr, 2, 6)
        assert_array(rho, multilevel.corr_coeff(R.astype(np.float64)), 1e-6, "rho")
        assert S.stml_temporal_set(ctx.ptr, 0) == grid.temporal_sets(6, 2)[0]
    finally:
        ctx.close()


@pytest.fixture(scope="module")
def paper_scale():
    spec = synthetic.spec_paper_scale()
    return synthetic.make_sequence(spec)


def test_full_size_finest_level(S, paper_scale):
    """All 200 frames of 256 x 256 at the finest of 4 levels, element by element,
    in the launch configuration the registration uses on that level."""
    import torch
    R = paper_scale
    ctx = _ctx(S, R, 4)
    try:
        frames = list(range(200))
        rng = np.random.default_rng(10)
        u = synthetic.random_field(rng, 200, 2, (256, 256), amp=3.0, rough=0.2, modes=2)
        g = torch.empty((200, 2, 256, 256), device="cuda")
        dT = torch.empty_like(g)
        out = S.stml_eval(ctx.ptr, 3, frames, _dev(u), g, dT)
        p = _oracle_params(ctx.params)
        ev = objective.evaluate(R.astype(np.float64), u.astype(np.float64), frames, 1.0, p)
        for i, k in enumerate(("J", "D", "S", "P")):
            assert_scalar(out[i], ev[k], what=k)
        assert_array(g.cpu().numpy(), ev["g"], what="gradient")
        assert_array(dT.cpu().numpy(), ev["dT"], what="grad T")
        v = synthetic.random_field(rng, 200, 2, (256, 256), amp=1.0, rough=0.5, modes=2)
        Hv = torch.empty_like(g)
        S.stml_hessvec(ctx.ptr, 3, frames, dT, _dev(v), Hv)
        ref = objective.hessvec(dT.cpu().numpy().astype(np.float64), v.astype(np.float64), frames, 1.0, p)
        assert_array(Hv.cpu().numpy(), ref, what="Hv")
    finally:
        ctx.close()


def test_bad_frames_are_rejected(S):
    import torch
    R = synthetic.make_sequence(synthetic.spec_custom(4, (16, 16), seed=1))
    ctx = _ctx(S, R, 1)
    try:
        u = torch.zeros((2, 2, 16, 16), device="cuda")
        with pytest.raises(S.StmlError) as e:
            S.stml_eval(ctx.ptr, 0, [2, 1], u)
        assert e.value.status == -1
        with pytest.raises(S.StmlError):
            S.stml_eval(ctx.ptr, 0, [0, 4], u)
        with pytest.raises(S.StmlError):
            S.stml_eval(ctx.ptr, 3, [0, 1], u)
        with pytest.raises(S.StmlError) as e:
            S.stml_predict(ctx.ptr, 0, 1)          # q = 1 before q = 0
        assert e.value.status == -8
    finally:
        ctx.close()


def test_many_frames_use_the_two_pass_path(S):
    """1000 frames exceed the shared memory of the single-pass cluster kernels
    (their staged per-frame terms); the two-pass kernels take over."""
    import torch
    n, shape = 1000, (8, 64)
    R = synthetic.make_sequence(synthetic.spec_custom(n, shape, seed=17, amp=1.0))
    ctx = _ctx(S, R, 1)
    try:
        frames = list(range(n))
        rng = np.random.default_rng(18)
        u = synthetic.random_field(rng, n, 2, shape, amp=0.8, rough=0.2, modes=1)
        g = torch.empty((n, 2) + shape, device="cuda")
        dT = torch.empty_like(g)
        out = S.stml_eval(ctx.ptr, 0, frames, _dev(u), g, dT)
        p = _oracle_params(ctx.params)
        ev = objective.evaluate(R.astype(np.float64), u.astype(np.float64), frames, 1.0, p)
        assert_scalar(out[0], ev["J"], what="J")
        assert_array(g.cpu().numpy(), ev["g"], what="gradient")
        v = synthetic.random_field(rng, n, 2, shape, amp=1.0, rough=0.5, modes=1)
        Hv = torch.empty_like(g)
        vhv = S.stml_hessvec(ctx.ptr, 0, frames, dT, _dev(v), Hv)
        ref = objective.hessvec(dT.cpu().numpy().astype(np.float64), v.astype(np.float64), frames, 1.0, p)
        assert_array(Hv.cpu().numpy(), ref, what="Hv")
        assert_scalar(vhv, float(np.sum(v.astype(np.float64) * ref)), what="<v,Hv>")
    finally:
        ctx.close()


def test_misaligned_device_arrays_are_rejected(S):
    import torch
    R = synthetic.make_sequence(synthetic.spec_custom(3, (16, 16), seed=1))
    ctx = _ctx(S, R, 1)
    try:
        buf = torch.zeros(3 * 2 * 16 * 16 + 1, device="cuda")
        u = buf[1:]                                   # 4-byte offset
        with pytest.raises(S.StmlError) as e:
            S.stml_eval(ctx.ptr, 0, [0, 1, 2], u)
        assert e.value.status == -1 and "aligned" in S.stml_last_error(ctx.ptr)
    finally:
        ctx.close()
