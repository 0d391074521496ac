"""ctypes loader for libperm.so (declarations in include/perm.h).

There is no fallback: if the library is missing or fails to load, every entry
point raises.  Build it with ``python -m paper_1606_05836_gb300.build``.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "lib", "libperm.so")

PERM_MAX_N = 48
PERM_FP64, PERM_FP64_DD, PERM_FP32P_DD, PERM_FP64_DF, PERM_FP32X2 = 0, 1, 2, 3, 4
PRECISIONS = {"fp64": PERM_FP64, "fp64_dd": PERM_FP64_DD, "fp32p_dd": PERM_FP32P_DD, "fp64_df": PERM_FP64_DF,
              "fp32x2": PERM_FP32X2}

# every symbol include/perm.h declares
EXPORTS = (
    "perm_workspace_size",
    "perm_glynn",
    "perm_ryser",
    "perm_ryser_nw",
    "perm_glynn_range",
    "perm_ryser_range",
    "perm_combine_partials",
    "perm_batched_workspace_size",
    "perm_batched",
    "perm_glynn_mult_workspace_size",
    "perm_glynn_mult",
    "prob_sample_workspace_size",
    "prob_sample",
    "perm_grad_workspace_size",
    "perm_grad",
    "perm_glynn_noalloc",
    "perm_row_minors_workspace_size",
    "perm_row_minors",
    "boson_sample_workspace_size",
    "boson_sample",
    "perm_fp64_fma_probe",
    "perm_strerror",
    "perm_last_cuda_error",
    "perm_version",
)


class PermError(RuntimeError):
    def __init__(self, status: int, what: str):
        msg = "%s failed: %s (status %d)" % (what, strerror(status), status)
        if status == -4 and _lib is not None:
            msg += ", cudaError %d" % _lib.perm_last_cuda_error()
        super().__init__(msg)
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("chunk_log2", ctypes.c_int), ("block", ctypes.c_int), ("grid", ctypes.c_int),
                ("unit_log2", ctypes.c_int)]


_lib = None


def load(path: str | None = None):
    """Load libperm.so once and declare the ctypes signatures."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError("libperm.so not found at %s; build it with `python -m paper_1606_05836_gb300.build`"
                           % path)
    lib = ctypes.CDLL(path)
    vp, i32, u64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_size_t
    op = ctypes.POINTER(Opts)
    lib.perm_workspace_size.argtypes = [i32, op]
    lib.perm_workspace_size.restype = sz
    for f in ("perm_glynn", "perm_ryser", "perm_ryser_nw"):
        getattr(lib, f).argtypes = [vp, i32, i32, vp, vp, sz, op, vp]
        getattr(lib, f).restype = i32
    for f in ("perm_glynn_range", "perm_ryser_range"):
        getattr(lib, f).argtypes = [vp, i32, i32, u64, u64, vp, vp, sz, op, vp]
        getattr(lib, f).restype = i32
    lib.perm_combine_partials.argtypes = [vp, i32, i32, i32, vp]
    lib.perm_combine_partials.restype = i32
    lib.perm_fp64_fma_probe.argtypes = [i32, i32, i32, vp, vp]
    lib.perm_fp64_fma_probe.restype = i32
    i32p = ctypes.POINTER(ctypes.c_int32)
    lib.perm_batched_workspace_size.argtypes = [i32, i32p, i32, op]
    lib.perm_batched_workspace_size.restype = sz
    lib.perm_batched.argtypes = [vp, vp, vp, i32p, i32, i32, vp, vp, vp, vp, sz, op, vp]
    lib.perm_batched.restype = i32
    lib.perm_glynn_mult_workspace_size.argtypes = [i32, i32, i32p, op]
    lib.perm_glynn_mult_workspace_size.restype = sz
    lib.perm_glynn_mult.argtypes = [vp, i32, i32, i32, i32p, vp, vp, sz, op, vp]
    lib.perm_glynn_mult.restype = i32
    lib.prob_sample_workspace_size.argtypes = [i32, op]
    lib.prob_sample_workspace_size.restype = sz
    lib.prob_sample.argtypes = [vp, i32, i32, i32p, i32p, ctypes.POINTER(ctypes.c_double), vp, vp, sz, op, vp]
    lib.prob_sample.restype = i32
    lib.perm_grad_workspace_size.argtypes = [i32, op]
    lib.perm_grad_workspace_size.restype = sz
    lib.perm_grad.argtypes = [vp, i32, i32, i32, ctypes.c_int64, vp, vp, vp, vp, vp, sz, op, vp]
    lib.perm_grad.restype = i32
    lib.perm_glynn_noalloc.argtypes = [vp, i32, i32, vp, op, vp]
    lib.perm_glynn_noalloc.restype = i32
    lib.perm_row_minors_workspace_size.argtypes = [i32, i32, op]
    lib.perm_row_minors_workspace_size.restype = sz
    lib.perm_row_minors.argtypes = [vp, i32, i32, i32, ctypes.c_int64, vp, vp, sz, op, vp]
    lib.perm_row_minors.restype = i32
    lib.boson_sample_workspace_size.argtypes = [i32, i32, i32, op]
    lib.boson_sample_workspace_size.restype = sz
    lib.boson_sample.argtypes = [vp, i32, i32, i32, ctypes.POINTER(ctypes.c_int32), i32, vp, vp, vp, vp, sz, op, vp]
    lib.boson_sample.restype = i32
    lib.perm_strerror.argtypes = [i32]
    lib.perm_strerror.restype = ctypes.c_char_p
    lib.perm_last_cuda_error.argtypes = []
    lib.perm_last_cuda_error.restype = i32
    lib.perm_version.argtypes = []
    lib.perm_version.restype = i32
    _lib = lib
    return lib


def strerror(status: int) -> str:
    if _lib is None:
        return "status %d" % status
    return _lib.perm_strerror(status).decode()


def check(status: int, what: str):
    if status != 0:
        raise PermError(status, what)
