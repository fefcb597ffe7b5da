"""Thin ctypes binding of ``libstml.so`` (include/stml.h).

Argument marshalling only: every function forwards to the C entry point of
the same name.  Device buffers are passed as ``torch`` CUDA tensors (their
``data_ptr()``), host buffers as numpy arrays.  There is no fallback: if the
library cannot be loaded every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libstml.so")

STATUS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ENONFINITE", -5: "EBREAKDOWN",
          -6: "ELINESEARCH", -7: "ETIMEOUT", -8: "ESTATE"}
MODE_STML, MODE_SPML = 0, 1
DTYPE_F32, DTYPE_F16, DTYPE_BF16 = 0, 1, 2     # stml_dtype: image / grad T storage


class StmlError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"stml error {STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(C.Structure):
    _fields_ = [("alpha", C.c_double), ("alpha_t", C.c_double), ("lambda_", C.c_double),
                ("beta", C.c_double), ("eps_stop", C.c_double), ("stop_rule", C.c_int),
                ("n_levels", C.c_int), ("n_tlevels", C.c_int),
                ("tol_J", C.c_double), ("tol_Y", C.c_double), ("tol_G", C.c_double),
                ("g_abs", C.c_double), ("max_gn", C.c_int), ("tol_cg", C.c_double),
                ("max_cg", C.c_int), ("max_ls", C.c_int), ("armijo_c", C.c_double),
                ("image_dtype", C.c_int), ("pcg_cooperative", C.c_int), ("autotune", C.c_int),
                ("transform", C.c_int), ("lbfgs_m", C.c_int), ("max_lbfgs", C.c_int), ("distance", C.c_int),
                ("target_J", C.c_double), ("target_tol", C.c_double), ("u_coarsen", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Stats(C.Structure):
    _fields_ = [("level", C.c_int), ("tlevel", C.c_int), ("n_frames", C.c_int),
                ("gn_iters", C.c_int), ("cg_iters", C.c_int), ("ls_trials", C.c_int),
                ("stopped_early", C.c_int), ("status", C.c_int),
                ("J0", C.c_double), ("J", C.c_double), ("D", C.c_double), ("S", C.c_double),
                ("P", C.c_double), ("seconds", C.c_double),
                ("pred_learned", C.c_int), ("fill_learned", C.c_int), ("J0_classic", C.c_double),
                ("J_fill_classic", C.c_double), ("J_fill", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class NetSample(C.Structure):
    """stml_net_sample (include/stml_net.h): device pointers of one sample."""
    _fields_ = [("y_l", C.c_void_p), ("y_r", C.c_void_p), ("T_l", C.c_void_p), ("T_k", C.c_void_p),
                ("T_r", C.c_void_p), ("target", C.c_void_p), ("out", C.c_void_p),
                ("plane", C.c_longlong), ("ld", C.c_int), ("ld_img", C.c_int),
                ("w_l", C.c_float), ("h", C.c_float)]


class Adam(C.Structure):
    _fields_ = [("lr", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double), ("eps", C.c_double)]


_lib = None
_vp, _ip, _dp, _fp = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double), C.c_void_p

_SIGS = {
    "stml_default_params": (None, [C.POINTER(Params)]),
    "stml_create": (C.c_int, [C.POINTER(Params), _vp, C.POINTER(_vp)]),
    "stml_destroy": (None, [_vp]),
    "stml_last_error": (C.c_char_p, [_vp]),
    "stml_set_params": (C.c_int, [_vp, C.POINTER(Params)]),
    "stml_load_sequence": (C.c_int, [_vp, _fp, C.c_int, C.c_int, C.c_int, _ip]),
    "stml_build_pyramid": (C.c_int, [_vp]),
    "stml_level_info": (C.c_int, [_vp, C.c_int, _ip, _dp]),
    "stml_temporal_set": (C.c_int, [_vp, C.c_int, _ip, C.c_int, _ip]),
    "stml_get_images": (C.c_int, [_vp, C.c_int, _fp, C.c_int]),
    "stml_get_field": (C.c_int, [_vp, C.c_int, _fp, C.c_int]),
    "stml_set_field": (C.c_int, [_vp, C.c_int, _fp, C.c_int]),
    "stml_register": (C.c_int, [_vp, C.c_int, C.POINTER(Stats), C.c_int, _ip]),
    "stml_register_batch": (C.c_int, [C.POINTER(_vp), C.c_int, C.c_int, C.c_int, _ip]),
    "stml_batch_create": (C.c_int, [C.POINTER(_vp), C.c_int, C.POINTER(_vp)]),
    "stml_batch_register": (C.c_int, [_vp, C.c_int, _ip]),
    "stml_batch_report": (C.c_int, [_vp, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)]),
    "stml_batch_last_error": (C.c_char_p, [_vp]),
    "stml_batch_destroy": (None, [_vp]),
    "stml_last_stats": (C.c_int, [_vp, C.POINTER(Stats), C.c_int, _ip]),
    "stml_check_batch_barrier": (C.c_int, [_vp, _ip]),
    "stml_predict": (C.c_int, [_vp, C.c_int, C.c_int]),
    "stml_correct": (C.c_int, [_vp, C.c_int, C.c_int, C.POINTER(Stats), _ip]),
    "stml_eval": (C.c_int, [_vp, C.c_int, _ip, C.c_int, _fp, _dp, _fp, _fp]),
    "stml_eval_trial": (C.c_int, [_vp, C.c_int, _ip, C.c_int, _fp, _fp, C.c_double, _fp, _dp]),
    "stml_hessvec": (C.c_int, [_vp, C.c_int, _ip, C.c_int, _fp, _fp, _fp, _dp]),
    "stml_gir": (C.c_int, [_vp, C.c_int, _ip, C.c_int, _fp, C.POINTER(Stats)]),
    "stml_corr_coeff": (C.c_int, [_vp, C.c_int, _dp]),
    "stml_restrict": (C.c_int, [_fp, _fp, C.c_int, C.c_int, _ip, _vp]),
    "stml_prolong": (C.c_int, [_fp, _fp, C.c_int, C.c_int, _ip, _vp]),
    "stml_prolong_adjoint": (C.c_int, [_fp, _fp, C.c_int, C.c_int, _ip, _vp]),
    "stml_predict_linear": (C.c_int, [_fp, _ip, C.c_int, _fp, _ip, C.c_int, C.c_size_t, _vp]),
    "stml_predict_ls": (C.c_int, [_fp, _ip, C.c_int, _fp, _fp, C.c_int, C.c_double, C.c_size_t, _vp]),
    "stml_hessvec_noalloc": (C.c_int, [_fp, _fp, _fp, C.c_int, _ip, C.c_double, _ip, C.c_int,
                                       C.POINTER(Params), _dp, _vp]),
    "stml_profile_enable": (C.c_int, [_vp, C.c_int]),
    "stml_profile_read": (C.c_int, [_vp, C.POINTER(C.c_longlong), _dp, _dp, _dp]),
    "stml_profile_report": (C.c_int, [_vp, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)]),
    "stml_launch_count": (C.c_longlong, [_vp]),
    "stml_coop_sync_floor": (C.c_int, [C.c_int, C.c_int, _dp]),
    "stml_tuning_report": (C.c_int, [_vp, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)]),
    "stml_eval_affine": (C.c_int, [_vp, C.c_int, _ip, C.c_int, _dp, _dp, _dp]),
    "stml_affine_field": (C.c_int, [_vp, C.c_int, _ip, C.c_int, _dp, _fp]),
    "stml_gir_affine": (C.c_int, [_vp, C.c_int, _ip, C.c_int, _dp, C.POINTER(Stats)]),
    "stml_get_affine": (C.c_int, [_vp, _dp, C.c_size_t]),
    # learned temporal predictor (include/stml_net.h)
    "stml_net_param_count": (C.c_size_t, []),
    "stml_net_create": (C.c_int, [_fp, C.c_size_t, C.c_int, C.c_int, C.c_int, _vp, C.POINTER(_vp)]),
    "stml_net_destroy": (None, [_vp]),
    "stml_net_last_error": (C.c_char_p, [_vp]),
    "stml_net_set_params": (C.c_int, [_vp, _fp, C.c_size_t]),
    "stml_net_get_params": (C.c_int, [_vp, _fp, C.c_size_t]),
    "stml_net_forward": (C.c_int, [_vp, C.POINTER(NetSample), C.c_int, C.c_int, C.c_int]),
    "stml_net_loss_grad": (C.c_int, [_vp, C.POINTER(NetSample), C.c_int, C.c_int, C.c_int, _dp, _fp]),
    "stml_net_train_step": (C.c_int, [_vp, C.POINTER(NetSample), C.c_int, C.c_int, C.c_int,
                                      C.POINTER(Adam), _dp]),
    "stml_set_predictor_net": (C.c_int, [_vp, _vp]),
    "stml_net_conv3_block": (C.c_int, [C.c_int, _fp, _fp, _fp, _fp, _fp, C.c_int, C.c_int, C.c_int, C.c_int,
                                       C.c_int, _vp]),
    "stml_check_bounded_wait": (C.c_int, [_vp, _ip]),
    "stml_eval_ugrid": (C.c_int, [_vp, C.c_int, _ip, C.c_int, _vp, _dp, _vp, _vp, _vp]),
    "stml_hessvec_ugrid": (C.c_int, [_vp, C.c_int, _ip, C.c_int, _vp, _vp, _vp, _dp]),
    "stml_ugrid_prolong": (C.c_int, [_vp, _vp, C.c_int, C.c_int, _ip, C.c_int, _vp]),
    "stml_ugrid_adjoint": (C.c_int, [_vp, _vp, C.c_int, C.c_int, _ip, C.c_int, _vp]),
}


def load(path: str = LIB_PATH):
    """Load libstml.so (built in-tree by ``_build.build``); raises if missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2001_06613_gb300._build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols() -> List[str]:
    return list(_SIGS)


# ------------------------------------------------------------------ helpers
def _ints(seq: Sequence[int]):
    arr = (C.c_int * len(seq))(*[int(v) for v in seq])
    return arr


def _dev(t) -> int:
    """Device pointer of a CUDA tensor (float32, contiguous)."""
    if t is None:
        return None
    if not (hasattr(t, "is_cuda") and t.is_cuda):
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _ptr(x):
    """(pointer, on_device) for a CUDA tensor or a host numpy array / CPU tensor."""
    if hasattr(x, "is_cuda"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), int(x.is_cuda)
    if not isinstance(x, np.ndarray) or not x.flags["C_CONTIGUOUS"] or x.dtype != np.float32:
        raise TypeError("host buffers must be C-contiguous float32 numpy arrays")
    return x.ctypes.data, 0


def _stream(stream):
    if stream is not None:
        return stream
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


def _check(status: int, ctx=None):
    if status != 0:
        raise StmlError(status, stml_last_error(ctx))


# ------------------------------------------------------------------ API
def stml_default_params(**overrides) -> Params:
    p = Params()
    load().stml_default_params(C.byref(p))
    for k, v in overrides.items():
        setattr(p, "lambda_" if k in ("lambda", "lam") else k, v)
    return p


def stml_create(params: Params, stream=None):
    out = _vp()
    _check(load().stml_create(C.byref(params), _stream(stream), C.byref(out)))
    return out


def stml_destroy(ctx):
    if ctx:
        load().stml_destroy(ctx)


def stml_last_error(ctx=None) -> str:
    s = load().stml_last_error(ctx)
    return s.decode() if s else ""


def stml_set_params(ctx, params: Params):
    _check(load().stml_set_params(ctx, C.byref(params)), ctx)


def stml_load_sequence(ctx, frames, shape: Optional[Sequence[int]] = None):
    """frames: (n, *shape) float32 CUDA tensor or host array."""
    shape = list(frames.shape[1:]) if shape is None else list(shape)
    if hasattr(frames, "dtype") and str(frames.dtype) not in ("float32", "torch.float32"):
        raise TypeError("frames must be float32")
    if not hasattr(frames, "is_cuda"):
        frames = np.ascontiguousarray(frames, dtype=np.float32)
    ptr, on_dev = _ptr(frames)
    _check(load().stml_load_sequence(ctx, ptr, on_dev, int(frames.shape[0]), len(shape), _ints(shape)), ctx)


def stml_build_pyramid(ctx):
    _check(load().stml_build_pyramid(ctx), ctx)


def stml_level_info(ctx, level: int):
    sh = (C.c_int * 3)()
    h = C.c_double()
    _check(load().stml_level_info(ctx, level, sh, C.byref(h)), ctx)
    return tuple(sh), h.value


def stml_temporal_set(ctx, tlevel: int) -> List[int]:
    cnt = C.c_int()
    _check(load().stml_temporal_set(ctx, tlevel, None, 0, C.byref(cnt)), ctx)
    buf = (C.c_int * cnt.value)()
    _check(load().stml_temporal_set(ctx, tlevel, buf, cnt.value, C.byref(cnt)), ctx)
    return list(buf)


def stml_get_images(ctx, level: int, out):
    ptr, on_dev = _ptr(out)
    _check(load().stml_get_images(ctx, level, ptr, on_dev), ctx)
    return out


def stml_get_field(ctx, level: int, out):
    ptr, on_dev = _ptr(out)
    _check(load().stml_get_field(ctx, level, ptr, on_dev), ctx)
    return out


def stml_set_field(ctx, level: int, src):
    ptr, on_dev = _ptr(src)
    _check(load().stml_set_field(ctx, level, ptr, on_dev), ctx)


def stml_register(ctx, mode: int = MODE_STML, cap: int = 512):
    stats = (Stats * cap)()
    n = C.c_int()
    _check(load().stml_register(ctx, mode, stats, cap, C.byref(n)), ctx)
    return [stats[i].as_dict() for i in range(min(n.value, cap))]


def stml_register_batch(ctxs: Sequence, mode: int = MODE_STML, max_threads: int = 0) -> List[int]:
    """Registers several contexts concurrently; returns each context's status."""
    arr = (_vp * len(ctxs))(*[c.ptr if hasattr(c, "ptr") else c for c in ctxs])
    st = (C.c_int * len(ctxs))()
    status = load().stml_register_batch(arr, len(ctxs), mode, max_threads, st)
    if status != 0:
        raise StmlError(status, stml_last_error(None) or "; ".join(
            stml_last_error(c.ptr if hasattr(c, "ptr") else c) for c in ctxs))
    return list(st)


def stml_batch_create(ctxs: Sequence):
    """A batch over the given contexts (Context objects or raw pointers)."""
    arr = (_vp * len(ctxs))(*[c.ptr if hasattr(c, "ptr") else c for c in ctxs])
    out = _vp()
    _check(load().stml_batch_create(arr, len(ctxs), C.byref(out)))
    return out


def stml_batch_last_error(batch) -> str:
    msg = load().stml_batch_last_error(batch)
    return msg.decode() if msg else ""


def stml_batch_register(batch, n_ctx: int, mode: int = MODE_STML) -> List[int]:
    """Registers every context of the batch with the persistent solver;
    returns each context's status (raises on the first failure)."""
    st = (C.c_int * n_ctx)()
    status = load().stml_batch_register(batch, mode, st)
    if status != 0:
        raise StmlError(status, stml_batch_last_error(batch))
    return list(st)


def stml_batch_report(batch) -> list:
    import json
    need = C.c_size_t()
    _check(load().stml_batch_report(batch, None, 0, C.byref(need)))
    buf = C.create_string_buffer(need.value)
    _check(load().stml_batch_report(batch, buf, need.value, C.byref(need)))
    return json.loads(buf.value.decode())


def stml_batch_destroy(batch):
    load().stml_batch_destroy(batch)


class Batch:
    """Owns one stml_batch over a list of Context objects."""

    def __init__(self, ctxs: Sequence):
        self.ctxs = list(ctxs)
        self.ptr = stml_batch_create(self.ctxs)

    def register(self, mode: int = MODE_STML) -> List[int]:
        return stml_batch_register(self.ptr, len(self.ctxs), mode)

    def report(self) -> list:
        return stml_batch_report(self.ptr)

    def close(self):
        if self.ptr:
            stml_batch_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def stml_last_stats(ctx, cap: int = 512) -> list:
    stats = (Stats * cap)()
    n = C.c_int()
    _check(load().stml_last_stats(ctx, stats, cap, C.byref(n)), ctx)
    return [stats[i].as_dict() for i in range(min(n.value, cap))]


def stml_check_batch_barrier(stream=None) -> bool:
    """True when a grid barrier of the batched solver that cannot complete
    gives up after its bound and reports it (takes about 2 s)."""
    out = C.c_int(0)
    _check(load().stml_check_batch_barrier(_stream(stream), C.byref(out)))
    return out.value == 1


def stml_predict(ctx, level: int, tlevel: int):
    _check(load().stml_predict(ctx, level, tlevel), ctx)


def stml_correct(ctx, level: int, tlevel: int):
    st = Stats()
    fin = C.c_int()
    _check(load().stml_correct(ctx, level, tlevel, C.byref(st), C.byref(fin)), ctx)
    return st.as_dict(), bool(fin.value)


def stml_eval(ctx, level: int, frames: Sequence[int], u, g=None, dT=None) -> np.ndarray:
    out = (C.c_double * 6)()
    _check(load().stml_eval(ctx, level, _ints(frames), len(frames), _dev(u), out, _dev(g), _dev(dT)), ctx)
    return np.array(out[:])


def stml_eval_trial(ctx, level: int, frames: Sequence[int], u, d, t: float, gd=None) -> np.ndarray:
    out = (C.c_double * 8)()
    _check(load().stml_eval_trial(ctx, level, _ints(frames), len(frames), _dev(u), _dev(d), C.c_double(t),
                                  _dev(gd), out), ctx)
    return np.array(out[:])


def stml_hessvec(ctx, level: int, frames: Sequence[int], dT, v, Hv) -> float:
    vhv = C.c_double()
    _check(load().stml_hessvec(ctx, level, _ints(frames), len(frames), _dev(dT), _dev(v), _dev(Hv),
                               C.byref(vhv)), ctx)
    return vhv.value


def stml_gir(ctx, level: int, frames: Sequence[int], u) -> dict:
    st = Stats()
    _check(load().stml_gir(ctx, level, _ints(frames), len(frames), _dev(u), C.byref(st)), ctx)
    return st.as_dict()


def stml_eval_ugrid(ctx, level: int, frames: Sequence[int], w, g=None, dT=None, Minv=None) -> np.ndarray:
    """Objective (J, D, S, P, |g|^2, |w|^2) at coarse-grid fields w (params.u_coarsen > 0)."""
    out = (C.c_double * 6)()
    _check(load().stml_eval_ugrid(ctx, level, _ints(frames), len(frames), _dev(w), out, _dev(g), _dev(dT),
                                  _dev(Minv)), ctx)
    return np.array(out[:])


def stml_hessvec_ugrid(ctx, level: int, frames: Sequence[int], dT, v, Hv) -> float:
    vhv = C.c_double()
    _check(load().stml_hessvec_ugrid(ctx, level, _ints(frames), len(frames), _dev(dT), _dev(v), _dev(Hv),
                                     C.byref(vhv)), ctx)
    return vhv.value


def stml_ugrid_prolong(w, u, planes: int, fine_shape: Sequence[int], s: int, stream=None):
    _check(load().stml_ugrid_prolong(_dev(w), _dev(u), planes, len(fine_shape), _ints(fine_shape), s,
                                     _stream(stream)))


def stml_ugrid_adjoint(u, w, planes: int, fine_shape: Sequence[int], s: int, stream=None):
    _check(load().stml_ugrid_adjoint(_dev(u), _dev(w), planes, len(fine_shape), _ints(fine_shape), s,
                                     _stream(stream)))


def stml_corr_coeff(ctx, level: int, n: int) -> np.ndarray:
    rho = (C.c_double * max(1, n - 1))()
    _check(load().stml_corr_coeff(ctx, level, rho), ctx)
    return np.array(rho[:n - 1])


def stml_restrict(fine, coarse, planes: int, fine_shape: Sequence[int], stream=None):
    _check(load().stml_restrict(_dev(fine), _dev(coarse), planes, len(fine_shape), _ints(fine_shape),
                                _stream(stream)))


def stml_prolong(coarse, fine, planes: int, coarse_shape: Sequence[int], stream=None):
    _check(load().stml_prolong(_dev(coarse), _dev(fine), planes, len(coarse_shape), _ints(coarse_shape),
                               _stream(stream)))


def stml_prolong_adjoint(fine, coarse, planes: int, coarse_shape: Sequence[int], stream=None):
    _check(load().stml_prolong_adjoint(_dev(fine), _dev(coarse), planes, len(coarse_shape),
                                       _ints(coarse_shape), _stream(stream)))


def stml_predict_linear(yK, K: Sequence[int], z, targets: Sequence[int], plane_elems: int, stream=None):
    _check(load().stml_predict_linear(_dev(yK), _ints(K), len(K), _dev(z), _ints(targets), len(targets),
                                      plane_elems, _stream(stream)))


def stml_predict_ls(eta, K: Sequence[int], omega, zeta, n: int, beta: float, n_comp: int, stream=None):
    _check(load().stml_predict_ls(_dev(eta), _ints(K), len(K), _dev(omega), _dev(zeta), n, beta, n_comp,
                                  _stream(stream)))


def stml_hessvec_noalloc(dT, v, Hv, shape: Sequence[int], h: float, frames: Sequence[int],
                         params: Params, stream=None) -> float:
    """Hessian product without any device allocation (static scratch array)."""
    vhv = C.c_double()
    _check(load().stml_hessvec_noalloc(_dev(dT), _dev(v), _dev(Hv), len(shape), _ints(shape), float(h),
                                       _ints(frames), len(frames), C.byref(params), C.byref(vhv),
                                       _stream(stream)))
    return vhv.value


def stml_profile_enable(ctx, mode: int = 1):
    """mode 1: time every solver launch; 2: only the Hessian product; 0: off."""
    _check(load().stml_profile_enable(ctx, int(mode)), ctx)


def stml_profile_read(ctx):
    n = C.c_longlong()
    ms, by, pf = C.c_double(), C.c_double(), C.c_double()
    _check(load().stml_profile_read(ctx, C.byref(n), C.byref(ms), C.byref(by), C.byref(pf)), ctx)
    return {"launches": n.value, "ms": ms.value, "bytes": by.value, "pixel_frames": pf.value}


def stml_profile_report(ctx) -> list:
    import json
    need = C.c_size_t()
    _check(load().stml_profile_report(ctx, None, 0, C.byref(need)), ctx)
    buf = C.create_string_buffer(need.value)
    _check(load().stml_profile_report(ctx, buf, need.value, C.byref(need)), ctx)
    return json.loads(buf.value.decode())


def stml_tuning_report(ctx) -> list:
    import json
    need = C.c_size_t()
    _check(load().stml_tuning_report(ctx, None, 0, C.byref(need)), ctx)
    buf = C.create_string_buffer(need.value)
    _check(load().stml_tuning_report(ctx, buf, need.value, C.byref(need)), ctx)
    return json.loads(buf.value.decode())


def stml_launch_count(ctx=None) -> int:
    return int(load().stml_launch_count(ctx))


def stml_coop_sync_floor(blocks: int, iters: int = 200) -> float:
    """Microseconds per CG step of the cooperative PCG solve's synchronisation
    alone (two partial-sum / grid-barrier / total rounds) on `blocks` CTAs."""
    us = C.c_double()
    _check(load().stml_coop_sync_floor(int(blocks), int(iters), C.byref(us)))
    return us.value


class Context:
    """Owns one stml_ctx; destroys it on close()/garbage collection."""

    def __init__(self, params: Params, stream=None):
        self.params = params
        self.ptr = stml_create(params, stream)

    def close(self):
        if self.ptr:
            stml_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------- affine variant
def _f64_host(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def stml_eval_affine(ctx, level: int, frames: Sequence[int], theta, want_grad: bool = True):
    """(J, D, S, P) and dJ/dtheta (nK, d(d+1)) at the affine fields of theta."""
    th, thp = _f64_host(theta)
    out = np.zeros(4)
    g = np.zeros_like(th) if want_grad else None
    _check(load().stml_eval_affine(ctx, level, _ints(frames), len(frames), thp, out.ctypes.data_as(_dp),
                                   g.ctypes.data_as(_dp) if want_grad else None), ctx)
    return out, g


def stml_affine_field(ctx, level: int, frames: Sequence[int], theta, u):
    th, thp = _f64_host(theta)
    _check(load().stml_affine_field(ctx, level, _ints(frames), len(frames), thp, _dev(u)), ctx)


def stml_gir_affine(ctx, level: int, frames: Sequence[int], theta):
    """L-BFGS GIR over the affine parameters from theta; returns (theta, stats)."""
    th = np.array(theta, dtype=np.float64, copy=True, order="C")
    st = Stats()
    _check(load().stml_gir_affine(ctx, level, _ints(frames), len(frames), th.ctypes.data_as(_dp), C.byref(st)), ctx)
    return th, st.as_dict()


def stml_get_affine(ctx, n: int, d: int) -> np.ndarray:
    out = np.zeros((n, d * (d + 1)))
    _check(load().stml_get_affine(ctx, out.ctypes.data_as(_dp), out.size), ctx)
    return out


# ------------------------------------------------- learned temporal predictor
def stml_net_param_count() -> int:
    return int(load().stml_net_param_count())


def _net_check(status: int, net=None):
    if status != 0:
        msg = load().stml_net_last_error(net).decode() if net else stml_last_error(None)
        raise StmlError(status, msg)


def _f32_host(a, n):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.size != n:
        raise ValueError(f"expected {n} parameters, got {a.size}")
    return a


def net_samples(y_l, y_r, T_l, T_k, T_r, h, w_l, target=None, out=None):
    """NetSample array for a batch of contiguous CUDA tensors: fields (B, 2, H, W),
    images (B, H, W), h and w_l per sample (sequences or scalars).  The tensors
    must stay alive while the samples are used."""
    B, _, H, W = y_l.shape
    h = np.broadcast_to(np.asarray(h, dtype=np.float64), (B,))
    w_l = np.broadcast_to(np.asarray(w_l, dtype=np.float64), (B,))
    arr = (NetSample * B)()
    fb, ib = 2 * H * W * 4, H * W * 4
    ptrs = [_dev(t) if t is not None else None for t in (y_l, y_r, T_l, T_k, T_r, target, out)]
    for b in range(B):
        s = arr[b]
        s.y_l, s.y_r = ptrs[0] + b * fb, ptrs[1] + b * fb
        s.T_l, s.T_k, s.T_r = ptrs[2] + b * ib, ptrs[3] + b * ib, ptrs[4] + b * ib
        s.target = ptrs[5] + b * fb if ptrs[5] else None
        s.out = ptrs[6] + b * fb if ptrs[6] else None
        s.plane, s.ld, s.ld_img = H * W, W, W
        s.w_l, s.h = float(w_l[b]), float(h[b])
    return arr


class Net:
    """A learned-predictor network (stml_net) with host parameters ``params``."""

    def __init__(self, params, max_batch: int, max_h: int, max_w: int, stream=None):
        n = stml_net_param_count()
        out = _vp()
        _net_check(load().stml_net_create(_f32_host(params, n).ctypes.data, n, int(max_batch), int(max_h),
                                          int(max_w), _stream(stream), C.byref(out)))
        self.ptr = out

    def close(self):
        if self.ptr:
            load().stml_net_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def stml_net_set_params(net: Net, params):
    n = stml_net_param_count()
    _net_check(load().stml_net_set_params(net.ptr, _f32_host(params, n).ctypes.data, n), net.ptr)


def stml_net_get_params(net: Net) -> np.ndarray:
    n = stml_net_param_count()
    out = np.empty(n, np.float32)
    _net_check(load().stml_net_get_params(net.ptr, out.ctypes.data, n), net.ptr)
    return out


def stml_net_forward(net: Net, samples, H: int, W: int):
    _net_check(load().stml_net_forward(net.ptr, samples, len(samples), int(H), int(W)), net.ptr)


def stml_net_loss_grad(net: Net, samples, H: int, W: int, want_grad: bool = True):
    loss = C.c_double()
    g = np.empty(stml_net_param_count(), np.float32) if want_grad else None
    _net_check(load().stml_net_loss_grad(net.ptr, samples, len(samples), int(H), int(W), C.byref(loss),
                                         g.ctypes.data if want_grad else None), net.ptr)
    return loss.value, g


def stml_net_train_step(net: Net, samples, H: int, W: int, lr: float = 1e-3, beta1: float = 0.9,
                        beta2: float = 0.999, eps: float = 1e-8, want_loss: bool = True):
    opt = Adam(lr, beta1, beta2, eps)
    loss = C.c_double()
    _net_check(load().stml_net_train_step(net.ptr, samples, len(samples), int(H), int(W), C.byref(opt),
                                          C.byref(loss) if want_loss else None), net.ptr)
    return loss.value if want_loss else None


def stml_set_predictor_net(ctx, net: Optional[Net]):
    ptr = ctx.ptr if hasattr(ctx, "ptr") else ctx
    _check(load().stml_set_predictor_net(ptr, net.ptr if net is not None else None), ptr)


def stml_net_conv3_block(mode: int, x, a, W, b, y, stream=None):
    """One convolution of the network on channels-last CUDA tensors (see stml_net.h):
    x (B, H, W, C), W (3, 3, Cin, Cout), b (Cout,)."""
    Bn, H, Wd = x.shape[:3]
    Cin, Cout = W.shape[2], W.shape[3]
    _check(load().stml_net_conv3_block(int(mode), _dev(x), _dev(a), _dev(W), _dev(b), _dev(y), Bn, H, Wd,
                                       Cin, Cout, _stream(stream)))


def stml_check_bounded_wait(stream=None) -> bool:
    """True when a device wait on an mbarrier nothing completes gave up as designed."""
    out = C.c_int()
    _check(load().stml_check_bounded_wait(_stream(stream), C.byref(out)))
    return bool(out.value)
