"""Mixed precision (16-bit storage of the images and of grad T; FP32
arithmetic): stored values, per-call parity against the oracle on the stored
inputs, and the error of each result against the FP64 oracle on the original
float frames."""
import numpy as np
import pytest

from _util import assert_array, assert_scalar, cuda_lib
from oracle import Params, grid, multilevel, objective
from paper_2001_06613_gb300 import synthetic

pytestmark = pytest.mark.gpu

DTYPES = [(1, "f16"), (2, "bf16")]


@pytest.fixture(scope="module")
def S():
    return cuda_lib()


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def quantize(x, dtype):
    """float32 -> 16-bit storage, round to nearest even, back to float32."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    if dtype == 1:
        return x.astype(np.float16).astype(np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def ulp(x, dtype):
    """Spacing of the 16-bit storage format at |x| (normal range)."""
    bits = 11 if dtype == 1 else 8
    _, e = np.frexp(np.abs(np.asarray(x, dtype=np.float64)))
    return np.maximum(np.ldexp(1.0, e - bits), 2.0 ** -24 if dtype == 1 else 2.0 ** -126)


def _ctx(S, R, levels, dtype, **kw):
    prm = S.stml_default_params(n_levels=levels, image_dtype=dtype, **kw)
    ctx = S.Context(prm)
    S.stml_load_sequence(ctx.ptr, _dev(R))
    S.stml_build_pyramid(ctx.ptr)
    return ctx


def _oparams(prm):
    return Params(alpha=prm.alpha, alpha_t=prm.alpha_t, lam=prm.lambda_, beta=prm.beta)


def _images(S, ctx, level, n, d):
    shape3 = tuple(S.stml_level_info(ctx.ptr, level)[0])
    out = np.empty((n,) + (shape3[1:] if d == 2 else shape3), np.float32)
    S.stml_get_images(ctx.ptr, level, out)
    return out


@pytest.mark.parametrize("dtype,name", DTYPES)
def test_stored_images_round_to_nearest_even(S, dtype, name):
    R = synthetic.make_sequence(synthetic.spec_custom(6, (48, 40), seed=31, amp=1.5))
    ctx = _ctx(S, R, 3, dtype)
    try:
        fine = _images(S, ctx, 2, 6, 2)
        assert np.array_equal(fine, quantize(R, dtype)), f"{name}: finest level is not the rounded input"
        # coarser levels: FP32 block mean of stored values, rounded; within
        # one unit in the last place of the exact mean of the level above
        above = fine.astype(np.float64)
        for lvl in (1, 0):
            got = _images(S, ctx, lvl, 6, 2).astype(np.float64)
            exact = multilevel.pyramid(above, 2)[0]
            assert np.all(np.abs(got - exact) <= ulp(exact, dtype)), f"{name}: level {lvl}"
            assert np.array_equal(quantize(got, dtype), got.astype(np.float32))
            above = got
    finally:
        ctx.close()


CASES = [
    ((48, 40), 9, 2, 1, list(range(9)), {}),
    ((48, 40), 9, 2, 0, [0, 4, 8], dict(alpha_t=0.3)),
    ((12, 16, 20), 5, 2, 1, [0, 1, 3, 4], {}),
]


@pytest.mark.parametrize("dtype,name", DTYPES)
@pytest.mark.parametrize("shape,n,levels,level,frames,extra", CASES)
def test_eval_parity_on_stored_images(S, dtype, name, shape, n, levels, level, frames, extra):
    """The objective, gradient and grad T from 16-bit images equal the oracle's
    on the same (stored) images at the FP32 tolerance."""
    import torch
    R = synthetic.make_sequence(synthetic.spec_custom(n, shape, seed=32, amp=1.5))
    ctx = _ctx(S, R, levels, dtype, **extra)
    try:
        T = _images(S, ctx, level, n, len(shape)).astype(np.float64)
        h = grid.level_h(levels, level)
        m = T.shape[1:]
        rng = np.random.default_rng(33)
        u = synthetic.random_field(rng, len(frames), len(m), m, amp=1.2 * h, rough=0.3 * h)
        g = torch.empty((len(frames), len(m)) + m, device="cuda")
        dT = torch.empty_like(g)
        out = S.stml_eval(ctx.ptr, level, frames, _dev(u), g, dT)
        ev = objective.evaluate(T[frames], u.astype(np.float64), frames, h, _oparams(ctx.params))
        for i, k in enumerate(("J", "D", "S", "P")):
            assert_scalar(out[i], ev[k], what=f"{name} {k}")
        assert_array(dT.cpu().numpy(), ev["dT"], what=f"{name} grad T")
        assert_array(g.cpu().numpy(), ev["g"], what=f"{name} gradient")
    finally:
        ctx.close()


@pytest.mark.parametrize("dtype,name", DTYPES)
def test_error_against_fp64_oracle_on_float_frames(S, dtype, name):
    """Error of each result of the 16-bit path against the FP64 oracle on the
    original float frames: J and |g| at the finest level, the Hessian product
    with grad T rounded to the storage type, and a full registration."""
    import torch
    spec = synthetic.spec_tiny()
    R = synthetic.make_sequence(spec)
    R64 = R.astype(np.float64)
    # per-call: J, |g| at the finest level
    ctx = _ctx(S, R, 2, dtype)
    try:
        frames = list(range(R.shape[0]))
        rng = np.random.default_rng(34)
        m = R.shape[1:]
        u = synthetic.random_field(rng, len(frames), 2, m, amp=1.5, rough=0.3)
        g = torch.empty((len(frames), 2) + m, device="cuda")
        out = S.stml_eval(ctx.ptr, 1, frames, _dev(u), g)
        p = _oparams(ctx.params)
        ev = objective.evaluate(R64, u.astype(np.float64), frames, 1.0, p)
        rel_J = abs(out[0] - ev["J"]) / abs(ev["J"])
        gn = float(np.sqrt(np.sum(ev["g"] ** 2)))
        rel_g = abs(np.sqrt(out[4]) - gn) / gn
        # Hessian product with the solver's 16-bit grad T
        dTq = quantize(ev["dT"], dtype)
        v = synthetic.random_field(rng, len(frames), 2, m, amp=1.0, rough=0.5)
        Hv = torch.empty_like(_dev(v))
        S.stml_hessvec(ctx.ptr, 1, frames, _dev(dTq), _dev(v), Hv)
        ref = objective.hessvec(ev["dT"], v.astype(np.float64), frames, 1.0, p)
        rel_H = float(np.abs(Hv.cpu().numpy() - ref).max() / np.abs(ref).max())
    finally:
        ctx.close()
    # end to end: STML registration, final objective on the float frames
    def register(dt):
        c = _ctx(S, R, 2, dt, n_tlevels=2)
        try:
            S.stml_register(c.ptr, 0)
            y = np.empty((R.shape[0], 2) + m, np.float32)
            S.stml_get_field(c.ptr, 1, y)
            return y, c.params
        finally:
            c.close()
    y16, prm = register(dtype)
    y32, _ = register(0)
    from oracle import Params as OP
    op = OP(alpha=prm.alpha, alpha_t=prm.alpha_t, lam=prm.lambda_, beta=prm.beta)
    J16 = multilevel.final_objective(R64, y16.astype(np.float64), op)["J"]
    J32 = multilevel.final_objective(R64, y32.astype(np.float64), op)["J"]
    rms = float(np.sqrt(np.mean((y16 - y32) ** 2)))
    print(f"\n{name}: rel err J {rel_J:.2e}, |g| {rel_g:.2e}, Hv {rel_H:.2e}; "
          f"registration: J {J16:.6g} vs f32 {J32:.6g} (rel {abs(J16 - J32) / J32:.2e}), "
          f"field RMS diff {rms:.3e} px")
    eps = 2.0 ** -11 if dtype == 1 else 2.0 ** -8     # unit roundoff of the storage
    assert rel_J <= 50 * eps and rel_g <= 50 * eps
    assert rel_H <= 20 * eps
    assert abs(J16 - J32) <= 1e-2 * J32
    assert rms <= 0.05
