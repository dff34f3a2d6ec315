"""ctypes view of ``librdcnn.so`` (the C ABI declared in ``include/rdcnn.h``).

Argument marshalling only.  Loading fails loudly when the library has not
been built: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

from .build import LIB

c_int = ctypes.c_int
c_i64 = ctypes.c_int64
c_size = ctypes.c_size_t
c_vp = ctypes.c_void_p
c_double = ctypes.c_double

OK = 0
WARN_CFL = 1
EINVAL = -1
ECUDA = -2
ETIMEOUT = -3
ENONFINITE = -4
ESTATE = -5
ESPACE = -6

BC_PERIODIC = 0
BC_ZEROFLUX = 1
F32 = 0
F64 = 1
BF16 = 2
F16 = 3
REACTION_FHN = 0
REACTION_NONE = 1
REACTION_CENN = 2
VARIANT_AUTO = 0
VARIANT_STEP1 = 1
VARIANT_TEMPORAL = 2
VARIANT_GENERIC = 3
VARIANT_TEMPORAL2 = 4
VARIANT_TEMPORAL_WIDE = 5

PARAM_FIELDS = ("dt", "a", "b", "eps", "c", "Du", "Dv")
STATIC_SCRATCH_BYTES = 16 << 20  # RDCNN_STATIC_SCRATCH_BYTES


class Params(ctypes.Structure):
    _fields_ = [(name, c_double) for name in PARAM_FIELDS]


class Tune(ctypes.Structure):
    _fields_ = [("k", c_int), ("rows", c_int)]


class Instance(ctypes.Structure):
    _fields_ = [("nn", c_i64), ("nm", c_i64), ("params", Params),
                ("u", c_vp), ("v", c_vp), ("su", c_vp), ("sv", c_vp)]


# (name, restype, argtypes) for every function of include/rdcnn.h
SIGNATURES = [
    ("rdcnn_create", c_int, [ctypes.POINTER(c_vp), c_i64, c_i64, ctypes.POINTER(Params), c_int, c_int, c_int]),
    ("rdcnn_set_params", c_int, [c_vp, ctypes.POINTER(Params)]),
    ("rdcnn_set_tune", c_int, [c_vp, ctypes.POINTER(Tune)]),
    ("rdcnn_workspace_bytes", c_int, [c_vp, ctypes.POINTER(c_size)]),
    ("rdcnn_bind", c_int, [c_vp, c_vp, c_vp, c_vp, c_size, c_vp]),
    ("rdcnn_init", c_int, [c_vp, c_vp, c_double, c_int]),
    ("rdcnn_set_state", c_int, [c_vp, c_vp, c_vp, c_int]),
    ("rdcnn_run", c_int, [c_vp, c_i64, c_int, c_int]),
    ("rdcnn_plan", c_int, [c_vp, ctypes.POINTER(c_int), ctypes.POINTER(Tune)]),
    ("rdcnn_get_state", c_int, [c_vp, c_vp, c_vp, c_int]),
    ("rdcnn_run_snapshots", c_int, [c_vp, c_i64, c_i64, c_vp, c_vp, c_int, c_vp, c_size]),
    ("rdcnn_destroy", None, [c_vp]),
    ("rdcnn_batch_workspace_bytes", c_int, [ctypes.POINTER(Instance), c_int, c_int, ctypes.POINTER(Tune),
                                            ctypes.POINTER(c_size)]),
    ("rdcnn_batch_run", c_int, [ctypes.POINTER(Instance), c_int, c_i64, c_int, c_int, ctypes.POINTER(Tune),
                                c_vp, c_size, c_vp]),
    ("rdcnn_batch_run_model", c_int, [ctypes.POINTER(Instance), c_int, c_i64, c_int, c_int, c_int,
                                      ctypes.POINTER(Tune), c_vp, c_size, c_vp]),
    ("rdcnn_summary_workspace_bytes", c_int, [ctypes.POINTER(Instance), c_int, ctypes.POINTER(c_size)]),
    ("rdcnn_batch_summary", c_int, [ctypes.POINTER(Instance), c_int, c_int, c_double, ctypes.POINTER(c_double),
                                    c_vp, c_size, c_vp]),
    ("rdcnn_adjoint_workspace_bytes", c_int, [c_vp, c_i64, c_i64, ctypes.POINTER(c_size)]),
    ("rdcnn_adjoint", c_int, [c_vp, c_i64, c_vp, c_vp, c_vp, c_vp, c_i64, c_vp, c_vp,
                              ctypes.POINTER(c_double), c_vp, c_size]),
    ("rdcnn_tape_bytes", c_int, [c_vp, c_i64, c_i64, ctypes.POINTER(c_size), ctypes.POINTER(c_size)]),
    ("rdcnn_run_record", c_int, [c_vp, c_i64, c_i64, c_vp, c_size]),
    ("rdcnn_adjoint_tape", c_int, [c_vp, c_i64, c_i64, c_vp, c_size, c_vp, c_vp, c_vp, c_vp,
                                   ctypes.POINTER(c_double), c_vp, c_size]),
    ("rdcnn_run_static", c_int, [c_i64, c_i64, ctypes.POINTER(Params), c_int, c_int, c_vp, c_vp, c_i64,
                                 c_int, c_vp]),
    ("rdcnn_last_error", ctypes.c_char_p, []),
    ("rdcnn_launch_count", ctypes.c_uint64, []),
    ("rdcnn_version", ctypes.c_char_p, []),
]

_lock = threading.Lock()
_lib = None


class RDCNNError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"rdcnn error {code}: {message}")
        self.code = code


def load(path: str | None = None):
    """Load librdcnn.so (built in-tree by ``build.build()``); raise if it is missing."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB
        if not os.path.exists(p):
            raise RuntimeError(
                f"librdcnn.so not found at {p}: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback exists)")
        lib = ctypes.CDLL(p)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        if path is None:
            _lib = lib
        return lib


def last_error() -> str:
    msg = load().rdcnn_last_error()
    return msg.decode() if msg else ""


def check(rc: int) -> int:
    """Raise RDCNNError for a negative status; pass OK and warnings through."""
    if rc < 0:
        raise RDCNNError(rc, last_error())
    return rc


def params_struct(params: dict) -> Params:
    return Params(*[float(params[k]) for k in PARAM_FIELDS])
