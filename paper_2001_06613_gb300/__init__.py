"""GB300-native spatio-temporal multilevel (STML) image-sequence registration.

The computation lives in ``libstml.so`` (CUDA for sm_103a behind the C ABI of
``include/stml.h``); :mod:`.binding` marshals arguments to it and
:mod:`.synthetic` generates seeded OCT-like test sequences.
"""
from .binding import *  # noqa: F401,F403
from .binding import Context, Params, Stats, StmlError, load, exported_symbols  # noqa: F401
from .binding import Net, NetSample, net_samples  # noqa: F401
from .binding import Batch  # noqa: F401

__all__ = [n for n in dir() if n.startswith("stml_")] + [
    "Context", "Params", "Stats", "StmlError", "load", "exported_symbols", "MODE_STML", "MODE_SPML",
    "Net", "NetSample", "net_samples", "Batch",
    "DTYPE_F32", "DTYPE_F16", "DTYPE_BF16"]
