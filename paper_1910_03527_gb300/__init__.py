"""GB300 (sm_103a) engine for the MBE-FCI tuple-CASCI hot path.

The compute lives in libmbe_gb300.so (CUDA kernels behind the C ABI of
include/mbe.h).  This package is its thin ctypes binding: ``Context`` wraps an
``mbe_ctx`` and exposes the ABI calls under the same names, and ``run_mbe``
strings them into one pass of the hot path (tuples -> tuple CASCI ->
increments -> totals).
"""

from .binding import (  # noqa: F401
    EXPANSION_TYPES,
    EXPORTS,
    Context,
    MBEEnergy,
    MbeError,
    Opts,
    STATUS_NAMES,
    expansion_spaces,
    lib,
    library_path,
    mbe_gradient,
    run_mbe,
    run_mbe_screened,
)
from ._build import build  # noqa: F401
