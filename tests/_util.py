"""Helpers shared by the test modules (tolerances, device fixtures)."""
import re
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# FP32 paths against the FP64 oracle: relative 1e-5 on scalars; arrays are
# compared elementwise against 1e-5 of the array's largest magnitude (values
# near zero have no meaningful relative error).
RTOL = 1e-5


def assert_scalar(got, ref, rtol=RTOL, what=""):
    assert abs(got - ref) <= rtol * abs(ref) + 1e-300, f"{what}: got {got!r} ref {ref!r} rel {abs(got-ref)/max(abs(ref),1e-300):.3e}"


def assert_array(got, ref, rtol=RTOL, what=""):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape, f"{what}: shape {got.shape} vs {ref.shape}"
    scale = float(np.abs(ref).max()) if ref.size else 0.0
    err = float(np.abs(got - ref).max()) if ref.size else 0.0
    assert err <= rtol * scale + 1e-30, f"{what}: max abs err {err:.3e} > {rtol:.1e} * {scale:.3e}"


def header_functions():
    import glob
    txt = "".join(open(f).read() for f in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))))
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(stml_[a-z0-9_]+)\s*\(", txt)))


def cuda_lib():
    """Build (if stale) and load the library on a CUDA machine, else skip."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_06613_gb300 import _build
    _build.build()
    import paper_2001_06613_gb300 as S
    S.load()
    return S
