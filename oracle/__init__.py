"""CPU oracle for the matrix permanent — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s ``cpu_baseline`` /
``--impl reference`` leg may import this package.  The GPU product path never
imports, links or executes it.  It shares no code with
``paper_1606_05836_gb300`` (neither imports the other).

The arithmetic lives in ``oracle.c`` (complex ``_Float128``, exact ``__int128``,
OpenMP); this module only marshals numpy arrays into it.  What each function
evaluates, and which passage of arXiv 1606.05836 it follows:

* :func:`perm_def`      -- the definition, sum over permutations (n <= 11).
* :func:`ryser`         -- Ryser's formula, Supp. Eq. (S1), subsets from the bits
                           of the iteration index as in Algorithm 1 (n <= 30).
* :func:`glynn`         -- the BB/FG formula, Supp. Eq. (S2), Algorithm 2 (n <= 30).
* :func:`glynn_gray`    -- Eq. (S2) in reflected-Gray order with one-sign row-sum
                           updates (the O(n 2^n) order the paper names), n <= 40.
* :func:`ryser_range`,
  :func:`glynn_range`   -- partial sums of the un-normalised terms over an index
                           range, binary or reflected-Gray index-to-set mapping.
* :func:`glynn_f64dd`,
  :func:`glynn_f64dd_range`,
  :func:`ryser_f64dd_range` -- Eq. (S2) / (S1) in reflected-Gray order in FP64
                           (row sums, updates, products) with every term added to
                           a double-double accumulator; pieces of 2^6 indices
                           start from row sums computed from scratch.  The
                           oracle for n = 29-40, where quad precision is too slow.
* :func:`ryser_int`     -- Eq. (S1) exactly, integers modulo 2^128.
* :func:`minors`        -- Per of every (n-1)x(n-1) minor = dPer/da_ij.
* :func:`prob`          -- Eq. (1), |Per(U_ST)|^2 / (prod s_i! prod t_j!).
* :mod:`oracle.sampler` -- row minors and boson-sampling draws from Eq. (1) by the
                           chain rule over the photons (numpy over the functions above).

Parity pins: tests/test_oracle_pins.py, tests/test_sampler_oracle.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (OpenMP).  Returns the path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        # no contraction of a*b+c into FMAs: the same rounding on every host
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-std=gnu11", "-o", tmp, _SRC,
               "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        u64 = ctypes.c_uint64
        lib.oracle_perm_def.argtypes = [ctypes.c_int, dp, dp]
        lib.oracle_ryser.argtypes = [ctypes.c_int, dp, ctypes.c_int, dp]
        lib.oracle_glynn.argtypes = [ctypes.c_int, dp, ctypes.c_int, dp]
        lib.oracle_glynn_gray.argtypes = [ctypes.c_int, dp, ctypes.c_int, dp]
        lib.oracle_ryser_range.argtypes = [ctypes.c_int, dp, u64, u64, ctypes.c_int, ctypes.c_int, dp]
        lib.oracle_glynn_range.argtypes = [ctypes.c_int, dp, u64, u64, ctypes.c_int, ctypes.c_int, dp]
        lib.oracle_glynn_f64dd.argtypes = [ctypes.c_int, dp, ctypes.c_int, dp]
        lib.oracle_glynn_f64dd_range.argtypes = [ctypes.c_int, dp, u64, u64, ctypes.c_int, dp]
        lib.oracle_ryser_f64dd_range.argtypes = [ctypes.c_int, dp, u64, u64, ctypes.c_int, dp]
        lib.oracle_ryser_z128.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_uint64)]
        lib.oracle_minors.argtypes = [ctypes.c_int, dp, ctypes.c_int, dp]
        lib.oracle_prob.argtypes = [ctypes.c_int, dp, ctypes.POINTER(ctypes.c_int32),
                                    ctypes.POINTER(ctypes.c_int32), ctypes.c_int, dp, dp]
        for f in ("oracle_perm_def", "oracle_ryser", "oracle_glynn", "oracle_glynn_gray", "oracle_ryser_range",
                  "oracle_glynn_range", "oracle_ryser_z128", "oracle_minors", "oracle_prob", "oracle_glynn_f64dd",
                  "oracle_glynn_f64dd_range", "oracle_ryser_f64dd_range"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
    return _lib


@dataclass(frozen=True)
class QC:
    """A complex number carried as hi + lo (about 106 significant bits)."""

    hi: complex
    lo: complex

    def __complex__(self) -> complex:
        return self.hi

    @property
    def value(self) -> complex:
        return self.hi

    def err(self, x: complex) -> float:
        """|x - (hi + lo)| evaluated so that hi cancels first."""
        d = (complex(x) - self.hi) - self.lo
        return abs(d)

    def rel_err(self, x: complex) -> float:
        return self.err(x) / abs(self.hi)


def _as_c128(A) -> np.ndarray:
    A = np.ascontiguousarray(np.asarray(A, dtype=np.complex128))
    if A.ndim != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("square matrix expected, got shape %r" % (A.shape,))
    return A


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _qc(out4: np.ndarray) -> QC:
    return QC(complex(out4[0], out4[2]), complex(out4[1], out4[3]))


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError("oracle %s rejected its arguments (rc=%d)" % (what, rc))


def perm_def(A) -> QC:
    """Per(A) = sum_s prod_i a[i][s(i)] (definition), n <= 11."""
    A = _as_c128(A)
    out = np.zeros(4)
    _check(_load().oracle_perm_def(A.shape[0], _dp(A), _dp(out)), "perm_def")
    return _qc(out)


def ryser(A, threads: int = 0) -> QC:
    """Per(A) by Supp. Eq. (S1) in complex _Float128, n <= 30."""
    A = _as_c128(A)
    out = np.zeros(4)
    _check(_load().oracle_ryser(A.shape[0], _dp(A), threads, _dp(out)), "ryser")
    return _qc(out)


def glynn(A, threads: int = 0) -> QC:
    """Per(A) by Supp. Eq. (S2) in complex _Float128, n <= 30."""
    A = _as_c128(A)
    out = np.zeros(4)
    _check(_load().oracle_glynn(A.shape[0], _dp(A), threads, _dp(out)), "glynn")
    return _qc(out)


def glynn_gray(A, threads: int = 0) -> QC:
    """Per(A) by Eq. (S2) in reflected-Gray order (one sign flips per step), quad, n <= 40."""
    A = _as_c128(A)
    out = np.zeros(4)
    _check(_load().oracle_glynn_gray(A.shape[0], _dp(A), threads, _dp(out)), "glynn_gray")
    return _qc(out)


def ryser_range(A, k_begin: int, k_end: int, gray: bool = True, threads: int = 0) -> QC:
    """sum_{k in [k_begin,k_end)} (-1)^{|S_k|} prod_i sum_{j in S_k} a_ij, no (-1)^n."""
    A = _as_c128(A)
    out = np.zeros(4)
    _check(_load().oracle_ryser_range(A.shape[0], _dp(A), int(k_begin), int(k_end), int(bool(gray)),
                                      threads, _dp(out)), "ryser_range")
    return _qc(out)


def glynn_range(A, k_begin: int, k_end: int, gray: bool = True, threads: int = 0) -> QC:
    """sum_{k in [k_begin,k_end)} (prod delta) prod_i sum_j delta_j a_ij, no 1/2^{n-1}."""
    A = _as_c128(A)
    out = np.zeros(4)
    _check(_load().oracle_glynn_range(A.shape[0], _dp(A), int(k_begin), int(k_end), int(bool(gray)),
                                      threads, _dp(out)), "glynn_range")
    return _qc(out)


def glynn_f64dd(A, threads: int = 0) -> QC:
    """Per(A) by Eq. (S2) in Gray order: FP64 terms, double-double sum, n <= 48."""
    A = _as_c128(A)
    out = np.zeros(4)
    _check(_load().oracle_glynn_f64dd(A.shape[0], _dp(A), threads, _dp(out)), "glynn_f64dd")
    return _qc(out)


def glynn_f64dd_range(A, k_begin: int, k_end: int, threads: int = 0) -> QC:
    """FP64 / double-double Glynn partial sum over Gray indices [k_begin, k_end), no 1/2^{n-1}."""
    A = _as_c128(A)
    out = np.zeros(4)
    _check(_load().oracle_glynn_f64dd_range(A.shape[0], _dp(A), int(k_begin), int(k_end), threads, _dp(out)),
           "glynn_f64dd_range")
    return _qc(out)


def ryser_f64dd_range(A, k_begin: int, k_end: int, threads: int = 0) -> QC:
    """FP64 / double-double Ryser partial sum over Gray indices [k_begin, k_end), no (-1)^n."""
    A = _as_c128(A)
    out = np.zeros(4)
    _check(_load().oracle_ryser_f64dd_range(A.shape[0], _dp(A), int(k_begin), int(k_end), threads, _dp(out)),
           "ryser_f64dd_range")
    return _qc(out)


def ryser_int(A, threads: int = 0) -> int:
    """Exact Per(A) of an integer matrix (valid while |Per| < 2^127)."""
    A = np.ascontiguousarray(np.asarray(A, dtype=np.int64))
    if A.ndim != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("square matrix expected")
    out = np.zeros(2, dtype=np.uint64)
    _check(_load().oracle_ryser_z128(A.shape[0], A.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), threads,
                                     out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))), "ryser_int")
    v = int(out[0]) | (int(out[1]) << 64)
    if v >= 1 << 127:
        v -= 1 << 128
    return v


def minors(A, threads: int = 0) -> np.ndarray:
    """M[i, j] = Per(A without row i, column j) (= dPer/da_ij), complex128 (hi)."""
    A = _as_c128(A)
    n = A.shape[0]
    out = np.zeros(4 * n * n)
    _check(_load().oracle_minors(n, _dp(A), threads, _dp(out)), "minors")
    o = out.reshape(n, n, 4)
    return o[..., 0] + 1j * o[..., 2]


def prob(U, s, t, threads: int = 0):
    """Eq. (1): (probability as float, Per(U_ST) as QC)."""
    U = _as_c128(U)
    m = U.shape[0]
    s = np.ascontiguousarray(np.asarray(s, dtype=np.int32))
    t = np.ascontiguousarray(np.asarray(t, dtype=np.int32))
    if s.shape != (m,) or t.shape != (m,):
        raise ValueError("occupation vectors must have length m")
    out2 = np.zeros(2)
    per4 = np.zeros(4)
    _check(_load().oracle_prob(m, _dp(U), s.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                               t.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), threads,
                               _dp(out2), _dp(per4)), "prob")
    return float(out2[0]) + float(out2[1]), _qc(per4)
