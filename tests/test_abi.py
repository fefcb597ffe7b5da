"""The C ABI library builds, loads and exports every symbol of include/stml.h
(no GPU needed: nothing here launches a kernel)."""
import ctypes

import pytest

from _util import header_functions
from oracle import Params


@pytest.fixture(scope="module")
def lib():
    from paper_2001_06613_gb300 import _build
    _build.build()
    import paper_2001_06613_gb300 as S
    return S


def test_every_declared_function_is_exported(lib):
    raw = ctypes.CDLL(lib.binding.LIB_PATH)
    declared = header_functions()
    assert len(declared) >= 25
    for name in declared:
        assert hasattr(raw, name), name
    assert sorted(lib.exported_symbols()) == declared


def test_default_params_match_the_oracle_defaults(lib):
    p = lib.stml_default_params()
    o = Params()
    assert (p.alpha, p.alpha_t, p.lambda_, p.beta) == (o.alpha, o.alpha_t, o.lam, o.beta)
    assert (p.eps_stop, bool(p.stop_rule)) == (o.eps_stop, o.stop_rule)
    assert (p.tol_J, p.tol_Y, p.tol_G, p.g_abs) == (o.tol_J, o.tol_Y, o.tol_G, o.g_abs)
    assert (p.max_gn, p.tol_cg, p.max_cg, p.max_ls, p.armijo_c) == (
        o.max_gn, o.tol_cg, o.max_cg, o.max_ls, o.armijo_c)


def test_invalid_parameters_are_rejected_before_any_device_work(lib):
    bad = lib.stml_default_params(n_levels=0)
    with pytest.raises(lib.StmlError) as e:
        lib.stml_create(bad)
    assert e.value.status == -1
    assert "n_levels" in lib.stml_last_error(None)
    bad = lib.stml_default_params(alpha=-1.0)
    with pytest.raises(lib.StmlError):
        lib.stml_create(bad)


def test_coop_sync_floor_rejects_bad_arguments_before_any_device_work(lib):
    for blocks, iters in ((0, 10), (4, 0), (-1, -1)):
        with pytest.raises(lib.StmlError) as e:
            lib.stml_coop_sync_floor(blocks, iters)
        assert e.value.status == -1
        assert "stml_coop_sync_floor" in lib.stml_last_error(None)


@pytest.mark.parametrize("overrides, message", [
    ({"n_levels": 13}, "n_levels"),
    ({"n_tlevels": 0}, "n_tlevels"),
    ({"alpha_t": -0.5}, "alpha_t"),
    ({"lam": float("nan")}, "lambda"),
    ({"max_ls": 0}, "iteration limits"),
    ({"max_cg": -1}, "iteration limits"),
    ({"tol_cg": 0.0}, "tol_cg"),
    ({"armijo_c": 1.0}, "armijo_c"),
    ({"pcg_cooperative": 2}, "pcg_cooperative"),
    ({"autotune": -1}, "autotune"),
    ({"transform": 2}, "transform"),
    ({"distance": 1, "transform": 0}, "distance 1"),
    ({"lbfgs_m": 65}, "lbfgs_m"),
    ({"target_J": -1.0}, "target_J"),
    ({"target_tol": 1.0}, "target_tol"),
    ({"image_dtype": 3}, "image_dtype"),
    ({"u_coarsen": 5}, "u_coarsen must be in 0..4"),
    ({"u_coarsen": 1, "transform": 1}, "u_coarsen > 0 needs"),
    ({"u_coarsen": 2, "image_dtype": 1}, "u_coarsen > 0 needs"),
    ({"u_coarsen": 1, "target_J": 10.0}, "u_coarsen > 0 needs"),
])
def test_every_parameter_rule_is_checked_before_any_device_work(lib, overrides, message):
    """Each documented parameter constraint of stml_params is refused by
    stml_create with STML_EINVAL and a message naming it, before any CUDA
    call (so this runs without a GPU)."""
    bad = lib.stml_default_params(**overrides)
    with pytest.raises(lib.StmlError) as e:
        lib.stml_create(bad)
    assert e.value.status == -1
    assert message in lib.stml_last_error(None)


# The context-free operators check their arguments before they touch the
# device: these calls pass stand-in device addresses that are never used.
_P = 256          # a 16-byte aligned stand-in address
_MIS = 260        # one that is not 16-byte aligned


def _ia(*v):
    return (ctypes.c_int * len(v))(*v)


@pytest.mark.parametrize("call, message", [
    (lambda L: L.stml_restrict(_P, _P, 1, 2, _ia(8, 7), None), "stml_restrict: odd axis"),
    (lambda L: L.stml_restrict(None, _P, 1, 2, _ia(8, 8), None), "stml_restrict: bad arguments"),
    (lambda L: L.stml_restrict(_P, _P, 1, 4, _ia(8, 8, 8, 8), None), "stml_restrict: bad arguments"),
    (lambda L: L.stml_prolong(_P, _P, -1, 2, _ia(8, 8), None), "stml_prolong: bad arguments"),
    (lambda L: L.stml_prolong_adjoint(_P, _P, 1, 2, _ia(0, 8), None), "stml_prolong_adjoint: bad arguments"),
    (lambda L: L.stml_ugrid_prolong(_P, _P, 1, 2, _ia(16, 16), 5, None), "stml_ugrid_prolong: bad arguments"),
    (lambda L: L.stml_ugrid_adjoint(_P, _P, 1, 2, _ia(16, 12), 3, None),
     "stml_ugrid_adjoint: an axis is not a multiple of 2^s"),
    (lambda L: L.stml_predict_linear(_P, _ia(0, 4, 2), 3, _P, _ia(1), 1, 64, None),
     "stml_predict_linear: bad arguments"),
    (lambda L: L.stml_predict_linear(_P, _ia(0, 4), 2, _P, _ia(5), 1, 64, None),
     "stml_predict_linear: target outside the span of K"),
    (lambda L: L.stml_predict_ls(_P, _ia(0, 4), 2, _P, _P, 5, 1.0, 64, None),
     "stml_predict_ls: omega and zeta must differ"),
    (lambda L: L.stml_predict_ls(_P, _ia(0, 5), 2, _P, _P + 64, 5, 1.0, 64, None), "stml_predict_ls: bad arguments"),
    (lambda L: L.stml_predict_ls(_P, _ia(0, 4), 2, _P, _P + 64, 5, -1.0, 64, None), "stml_predict_ls: bad arguments"),
])
def test_context_free_operators_refuse_bad_arguments_before_any_device_work(lib, call, message):
    L = lib.load()
    assert call(L) == -1
    assert message in lib.stml_last_error(None)


def test_allocation_free_hessian_product_refuses_before_any_device_work(lib):
    L = lib.load()
    p = lib.stml_default_params()
    cases = [
        ((_MIS, _P, _P, 2, _ia(8, 8), 1.0, _ia(0, 1), 2), "16-byte aligned"),
        ((_P, _P, _P, 2, _ia(8, 8), 1.0, _ia(1, 1), 2), "frames must increase"),
        ((_P, _P, _P, 2, _ia(8, 0), 1.0, _ia(0, 1), 2), "bad shape"),
        ((_P, _P, _P, 2, _ia(8, 8), 0.0, _ia(0, 1), 2), "bad arguments"),
        # 4096 x 4096 pixels need 192 MiB of per-pixel sums: more than the static array
        ((_P, _P, _P, 2, _ia(4096, 4096), 1.0, _ia(0, 1), 2), "scratch bytes"),
    ]
    for (dT, v, Hv, dim, shape, h, frames, nK), message in cases:
        st = L.stml_hessvec_noalloc(dT, v, Hv, dim, shape, h, frames, nK, ctypes.byref(p), None, None)
        assert st == -1, message
        assert message in lib.stml_last_error(None)
