"""GPU parity of the coarse displacement grid (params.u_coarsen = s > 0): the
interpolation P_s and its adjoint gather, the objective, gradient, Jacobi
diagonal and Hessian product of the unknowns on the coarse grid, one GIR and
whole STML / SpML registrations, against the oracle (C ABI)."""
import numpy as np
import pytest

from _util import assert_array, assert_scalar, cuda_lib, gir_counts, oracle_branch
from oracle import Params, grid, multilevel, solver, ugrid
from paper_2001_06613_gb300 import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    return cuda_lib()


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _ctx(S, R, **kw):
    prm = S.stml_default_params(**kw)
    ctx = S.Context(prm)
    S.stml_load_sequence(ctx.ptr, _dev(R))
    S.stml_build_pyramid(ctx.ptr)
    return ctx


def _oparams(prm, **kw):
    base = dict(alpha=prm.alpha, alpha_t=prm.alpha_t, lam=prm.lambda_, beta=prm.beta,
                eps_stop=prm.eps_stop, stop_rule=bool(prm.stop_rule), n_levels=prm.n_levels,
                n_tlevels=prm.n_tlevels, tol_J=prm.tol_J, tol_Y=prm.tol_Y, tol_G=prm.tol_G,
                max_gn=prm.max_gn, tol_cg=prm.tol_cg, max_cg=prm.max_cg, max_ls=prm.max_ls,
                armijo_c=prm.armijo_c, g_abs=prm.g_abs, u_coarsen=prm.u_coarsen)
    base.update(kw)
    return Params(**base)


@pytest.mark.parametrize("fine,s,planes", [((32, 48), 1, 3), ((40, 24), 2, 2), ((64, 32), 3, 1),
                                           ((8, 12, 16), 1, 2), ((16, 8, 24), 2, 1)])
def test_prolongation_and_adjoint_gather(S, fine, s, planes):
    import torch
    rng = np.random.default_rng(1)
    coarse = tuple(m // 2 ** s for m in fine)
    w = rng.normal(size=(planes,) + coarse)
    f = rng.normal(size=(planes,) + fine)
    u = torch.empty((planes,) + fine, device="cuda")
    S.stml_ugrid_prolong(_dev(w), u, planes, fine, s)
    assert_array(u.cpu().numpy(), ugrid.prolong(w, fine, s), rtol=1e-6, what="P_s w")
    wa = torch.empty((planes,) + coarse, device="cuda")
    S.stml_ugrid_adjoint(_dev(f), wa, planes, fine, s)
    assert_array(wa.cpu().numpy(), ugrid.adjoint(f, fine, s), rtol=1e-6, what="P_s^T f")


CASES = [
    # image shape, frames n, levels, level, frames of K, s, extra params
    ((64, 48), 6, 2, 1, [0, 1, 2, 3, 4, 5], 1, {}),
    ((64, 48), 6, 2, 0, [0, 2, 5], 1, dict(alpha_t=0.3)),
    ((96, 80), 5, 1, 0, [0, 1, 3, 4], 2, dict(alpha=0.3, lambda_=2.5)),
    ((16, 24, 32), 4, 2, 1, [0, 1, 2, 3], 1, {}),                     # 3-D
]


@pytest.mark.parametrize("shape,n,levels,level,frames,s,extra", CASES)
def test_eval_gradient_jacobi_hessian_parity(S, shape, n, levels, level, frames, s, extra):
    import torch
    spec = synthetic.spec_custom(n, shape, seed=5, amp=1.5)
    R = synthetic.make_sequence(spec)
    ctx = _ctx(S, R, n_levels=levels, u_coarsen=s, **extra)
    try:
        T = multilevel.pyramid(R.astype(np.float64), levels)[level][frames]
        h = grid.level_h(levels, level)
        m = T.shape[1:]
        cm = tuple(x // 2 ** s for x in m)
        d = len(m)
        rng = np.random.default_rng(7)
        w = synthetic.random_field(rng, len(frames), d, cm, amp=1.2 * h, rough=0.3 * h)
        op = _oparams(ctx.params)
        g = torch.empty((len(frames), d) + cm, device="cuda")
        Minv = torch.empty_like(g)
        dT = torch.empty((len(frames), d) + m, device="cuda")
        out = S.stml_eval_ugrid(ctx.ptr, level, frames, _dev(w), g, dT, Minv)
        ev = ugrid.evaluate(T, w.astype(np.float64), frames, h, s, op)
        for i, k in enumerate(("J", "D", "S", "P")):
            assert_scalar(out[i], ev[k], what=k)
        assert_scalar(out[4], float(np.sum(ev["g"] ** 2)), what="|g|^2")
        assert_scalar(out[5], float(np.sum(w.astype(np.float64) ** 2)), what="|w|^2")
        assert_array(dT.cpu().numpy(), ev["dT"], what="grad T")
        assert_array(g.cpu().numpy(), ev["g"], what="coarse gradient")
        dTg = dT.cpu().numpy().astype(np.float64)
        assert_array(Minv.cpu().numpy(), 1.0 / ugrid.jacobi_diag(dTg, frames, h, s, op), what="Jacobi inverse")
        obj = S.stml_eval_ugrid(ctx.ptr, level, frames, _dev(w))
        assert_scalar(obj[0], ev["J"], what="objective-only J")
        v = synthetic.random_field(rng, len(frames), d, cm, amp=1.0, rough=0.5)
        Hv = torch.empty_like(g)
        vhv = S.stml_hessvec_ugrid(ctx.ptr, level, frames, dT, _dev(v), Hv)
        href = ugrid.hessvec(dTg, v.astype(np.float64), frames, h, s, op)
        assert_array(Hv.cpu().numpy(), href, what="Hv")
        assert_scalar(vhv, float(np.sum(v.astype(np.float64) * href)), what="<v, Hv>")
    finally:
        ctx.close()


@pytest.mark.parametrize("max_gn", [1, 3])
def test_gir_matches_oracle_gauss_newton(S, max_gn):
    R = synthetic.make_sequence(synthetic.spec_custom(5, (64, 80), seed=21, amp=1.5))
    ctx = _ctx(S, R, n_levels=1, max_gn=max_gn, u_coarsen=1)
    try:
        frames = [0, 1, 2, 3, 4]
        w0 = np.zeros((5, 2, 32, 40), np.float32)
        wd = _dev(w0)
        st = S.stml_gir(ctx.ptr, 0, frames, wd)
        op = _oparams(ctx.params)
        T = R.astype(np.float64)
        wo, so = solver.gauss_newton(T, w0, frames, 1.0, op, model=ugrid.Model(T, frames, 1.0, 1, op))
        assert (st["gn_iters"], st["cg_iters"], st["ls_trials"]) == (so.gn_iters, so.cg_iters, so.ls_trials)
        assert_scalar(st["J0"], so.J0, 1e-5, "J0")
        assert_scalar(st["J"], so.J, 1e-5 * max_gn, "J after GN")
        diff = wd.cpu().numpy() - wo
        assert np.sqrt(np.mean(diff ** 2)) <= 1e-4 * max(1.0, np.sqrt(np.mean(wo ** 2)))
    finally:
        ctx.close()


def _register(S, R, mode, **kw):
    ctx = _ctx(S, R, **kw)
    try:
        stats = S.stml_register(ctx.ptr, mode)
        prm = ctx.params
        s = prm.u_coarsen
        L = prm.n_levels
        y = np.empty((R.shape[0], R.ndim - 1) + tuple(m // 2 ** s for m in R.shape[1:]), np.float32)
        S.stml_get_field(ctx.ptr, L - 1, y)
        return stats, y, prm
    finally:
        ctx.close()


@pytest.mark.parametrize("mode,s", [(0, 1), (1, 1), (0, 2)])
def test_register_matches_oracle(S, mode, s):
    """16 frames of 64x64 (the tiny workload), 2 spatial x 2 temporal levels,
    unknowns on the image grid coarsened by 2^s: the same GIR sequence with
    the same iteration counts, the final objective within 1e-4 and the
    fields within 1e-3 px of the oracle's."""
    spec = synthetic.spec_tiny()
    R = synthetic.make_sequence(spec)
    stats, y, prm = _register(S, R, mode, n_levels=2, n_tlevels=2, u_coarsen=s)
    op = _oparams(prm)
    res, _ = oracle_branch(lambda fl: multilevel.register(R.astype(np.float64), op, "stml" if mode == 0 else "spml",
                                                          flips=fl), gir_counts(stats), op.tol_cg)
    assert gir_counts(stats) == gir_counts(res.stats)
    Jg = multilevel.final_objective(R.astype(np.float64), y.astype(np.float64), op)["J"]
    Jo = multilevel.final_objective(R.astype(np.float64), res.y, op)["J"]
    assert abs(Jg - Jo) <= 1e-4 * Jo, (Jg, Jo)
    assert float(np.sqrt(np.mean((y - res.y) ** 2))) <= 1e-3
    # the prolonged fields register the planted motion
    u = ugrid.prolong(y.astype(np.float64), R.shape[1:], s)
    truth = synthetic.planted_registration(spec)
    c = lambda f: f - f.mean(axis=0, keepdims=True)
    e = (c(u) - c(truth))[..., 4:-4, 4:-4]
    assert float(np.sqrt((e ** 2).sum(axis=1).mean())) < 0.25


def test_invalid_combinations_are_refused(S):
    R = synthetic.make_sequence(synthetic.spec_custom(3, (20, 20), seed=1))
    with pytest.raises(S.StmlError):
        S.Context(S.stml_default_params(u_coarsen=1, image_dtype=1))
    with pytest.raises(S.StmlError):
        S.Context(S.stml_default_params(u_coarsen=5))
    ctx = S.Context(S.stml_default_params(n_levels=2, u_coarsen=2))
    try:
        with pytest.raises(S.StmlError):   # 20 is not a multiple of 2^(2 - 1 + 2)
            S.stml_load_sequence(ctx.ptr, _dev(R))
    finally:
        ctx.close()
    ctx = _ctx(S, R, n_levels=2, pcg_cooperative=0)
    try:
        with pytest.raises(S.StmlError):   # a coarse-grid evaluation needs u_coarsen > 0
            S.stml_eval_ugrid(ctx.ptr, 1, [0, 1], _dev(np.zeros((2, 2, 10, 10))))
    finally:
        ctx.close()


def test_lowering_u_coarsen_on_a_loaded_context(S):
    """The coarse-grid buffers made for 2^2 coarsening are made again, larger,
    when stml_set_params lowers u_coarsen to 1 on the loaded context: the
    evaluation equals that of a context created with u_coarsen = 1."""
    import torch
    R = synthetic.make_sequence(synthetic.spec_custom(4, (64, 48), seed=9, amp=1.2))
    frames = [0, 1, 2, 3]
    rng = np.random.default_rng(3)
    w1 = _dev(synthetic.random_field(rng, 4, 2, (32, 24), amp=1.0, rough=0.3))
    w2 = _dev(synthetic.random_field(rng, 4, 2, (16, 12), amp=1.0, rough=0.3))
    ref = _ctx(S, R, n_levels=1, u_coarsen=1)
    ctx = _ctx(S, R, n_levels=1, u_coarsen=2)
    try:
        g_ref = torch.empty_like(w1)
        out_ref = S.stml_eval_ugrid(ref.ptr, 0, frames, w1, g_ref)
        S.stml_eval_ugrid(ctx.ptr, 0, frames, w2, torch.empty_like(w2))   # buffers for s = 2
        S.stml_set_params(ctx.ptr, S.stml_default_params(n_levels=1, u_coarsen=1))
        g = torch.empty_like(w1)
        out = S.stml_eval_ugrid(ctx.ptr, 0, frames, w1, g)
        assert np.array_equal(out, out_ref)
        assert torch.equal(g, g_ref)
    finally:
        ctx.close()
        ref.close()


def test_register_3d_matches_oracle(S):
    """4 volumes of 16^3, 2 x 2 levels, unknowns on the image grid coarsened
    by 2 (the oracle's CG ratios stay >= 0.8 % from tol_cg here): the same
    counts, J within 1e-4 and the fields within 1e-3 voxel of the oracle's."""
    R = synthetic.make_sequence(synthetic.spec_custom(4, (16, 16, 16), seed=6, amp=1.0))
    stats, y, prm = _register(S, R, 0, n_levels=2, n_tlevels=2, u_coarsen=1)
    op = _oparams(prm)
    res, _ = oracle_branch(lambda fl: multilevel.register(R.astype(np.float64), op, "stml", flips=fl),
                           gir_counts(stats), op.tol_cg)
    assert gir_counts(stats) == gir_counts(res.stats)
    Jg = multilevel.final_objective(R.astype(np.float64), y.astype(np.float64), op)["J"]
    Jo = multilevel.final_objective(R.astype(np.float64), res.y, op)["J"]
    assert abs(Jg - Jo) <= 1e-4 * Jo, (Jg, Jo)
    assert float(np.sqrt(np.mean((y - res.y) ** 2))) <= 1e-3


def test_full_size_finest_level(S):
    """All 200 frames of 256 x 256 (the paper-scale sequence) with the unknowns
    on the 128 x 128 grid: objective, gradient, Jacobi inverse and Hessian
    product element by element against the oracle."""
    import torch
    R = synthetic.make_sequence(synthetic.spec_paper_scale())
    ctx = _ctx(S, R, n_levels=4, u_coarsen=1)
    try:
        frames = list(range(200))
        rng = np.random.default_rng(11)
        # values on a 2^-10 grid: their interpolation (weights 1/4, 3/4) is exact
        # in FP32 as in FP64, so both sides sample the images at the same
        # positions (on 26 M sample points some lie within FP32 rounding of a
        # cell edge, where grad T is one-sided and a rounding would pick the
        # other cell)
        w = synthetic.random_field(rng, 200, 2, (128, 128), amp=3.0, rough=0.2, modes=2)
        w = (np.round(w * 1024.0) / 1024.0).astype(np.float32)
        g = torch.empty((200, 2, 128, 128), device="cuda")
        Minv = torch.empty_like(g)
        dT = torch.empty((200, 2, 256, 256), device="cuda")
        out = S.stml_eval_ugrid(ctx.ptr, 3, frames, _dev(w), g, dT, Minv)
        op = _oparams(ctx.params)
        T = R.astype(np.float64)
        ev = ugrid.evaluate(T, w.astype(np.float64), frames, 1.0, 1, op)
        for i, k in enumerate(("J", "D", "S", "P")):
            assert_scalar(out[i], ev[k], what=k)
        assert_array(dT.cpu().numpy(), ev["dT"], what="grad T")
        assert_array(g.cpu().numpy(), ev["g"], what="coarse gradient")
        dTg = dT.cpu().numpy().astype(np.float64)
        assert_array(Minv.cpu().numpy(), 1.0 / ugrid.jacobi_diag(dTg, frames, 1.0, 1, op), what="Jacobi inverse")
        v = synthetic.random_field(rng, 200, 2, (128, 128), amp=1.0, rough=0.5, modes=2)
        Hv = torch.empty_like(g)
        S.stml_hessvec_ugrid(ctx.ptr, 3, frames, dT, _dev(v), Hv)
        assert_array(Hv.cpu().numpy(), ugrid.hessvec(dTg, v.astype(np.float64), frames, 1.0, 1, op), what="Hv")
    finally:
        ctx.close()
