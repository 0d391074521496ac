"""The C-ABI library builds, loads and exports every symbol include/perm.h declares.

No compute call is made here (no GPU on this host); only host-side helpers
(perm_strerror, perm_version) are called.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b([A-Za-z_][A-Za-z0-9_]*)\s*\(", text):
            name = m.group(1)
            if name.startswith(("perm_", "prob_", "boson_")) and not name.startswith("perm_c128"):
                names.append(name)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1606_05836_gb300 import build, _native
    build.build()
    return _native.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "perm_glynn" in names and "perm_ryser" in names
    for name in names:
        assert hasattr(lib, name), name


def test_python_binding_lists_the_same_symbols():
    from paper_1606_05836_gb300 import _native
    assert sorted(_native.EXPORTS) == declared_functions()


def test_host_helpers(lib):
    assert lib.perm_version() == 1
    assert lib.perm_strerror(0) == b"ok"
    assert lib.perm_strerror(-2).startswith(b"size")
    assert lib.perm_strerror(12345) == b"unknown status"


def test_argument_errors_before_any_launch(lib):
    """Host-detectable errors return before touching the device."""
    from paper_1606_05836_gb300._native import Opts
    o = Opts(0, 0, 0, 0, 0)
    # n out of range
    assert lib.perm_glynn(None, 49, 49, None, None, 0, ctypes.byref(o), None) == -2
    assert lib.perm_ryser(None, -1, 0, None, None, 0, ctypes.byref(o), None) == -2
    # null output
    assert lib.perm_glynn(ctypes.c_void_p(16), 4, 4, None, ctypes.c_void_p(16), 1 << 20, ctypes.byref(o), None) == -1
    # lda < n
    assert lib.perm_glynn(ctypes.c_void_p(16), 4, 3, ctypes.c_void_p(32), ctypes.c_void_p(64), 1 << 20,
                          ctypes.byref(o), None) == -1
    # misaligned matrix pointer
    assert lib.perm_ryser(ctypes.c_void_p(8), 4, 4, ctypes.c_void_p(32), ctypes.c_void_p(64), 1 << 20,
                          ctypes.byref(o), None) == -1
    # bad options
    bad = Opts(7, 0, 0, 0, 0)
    assert lib.perm_glynn(ctypes.c_void_p(16), 4, 4, ctypes.c_void_p(32), ctypes.c_void_p(64), 1 << 20,
                          ctypes.byref(bad), None) == -1
    bad = Opts(0, 0, 100, 0, 0)
    assert lib.perm_glynn(ctypes.c_void_p(16), 4, 4, ctypes.c_void_p(32), ctypes.c_void_p(64), 1 << 20,
                          ctypes.byref(bad), None) == -1
    # range beyond 2^(n-1) for Glynn
    assert lib.perm_glynn_range(ctypes.c_void_p(16), 4, 4, 0, 9, ctypes.c_void_p(32), ctypes.c_void_p(64), 1 << 20,
                                ctypes.byref(o), None) == -2
    assert lib.perm_ryser_range(ctypes.c_void_p(16), 4, 4, 5, 3, ctypes.c_void_p(32), ctypes.c_void_p(64), 1 << 20,
                                ctypes.byref(o), None) == -2


def test_argument_errors_of_minors_and_draws(lib):
    """The row-minor and draw entry points reject bad arguments before touching the device."""
    from paper_1606_05836_gb300._native import Opts
    o = Opts(0, 0, 0, 0, 0)
    p16, p32, p256 = ctypes.c_void_p(16), ctypes.c_void_p(32), ctypes.c_void_p(256)
    assert lib.perm_row_minors(p16, 0, 1, 1, 0, p32, p256, 1 << 20, ctypes.byref(o), None) == -2
    assert lib.perm_row_minors(p16, 33, 33, 1, 0, p32, p256, 1 << 20, ctypes.byref(o), None) == -2
    assert lib.perm_row_minors(p16, 5, 5, -1, 0, p32, p256, 1 << 20, ctypes.byref(o), None) == -1
    assert lib.perm_row_minors(p16, 5, 5, 1, 0, None, p256, 1 << 20, ctypes.byref(o), None) == -1
    assert lib.perm_row_minors(None, 5, 5, 1, 0, p32, p256, 1 << 20, ctypes.byref(o), None) == -1
    assert lib.perm_row_minors(p16, 5, 4, 1, 0, p32, p256, 1 << 20, ctypes.byref(o), None) == -1  # ldm < k
    assert lib.perm_row_minors(p16, 5, 5, 0, 0, p32, p256, 1 << 20, ctypes.byref(o), None) == 0  # empty batch
    ins = (ctypes.c_int32 * 3)(0, 1, 2)
    rep = (ctypes.c_int32 * 3)(0, 1, 1)
    far = (ctypes.c_int32 * 3)(0, 1, 9)
    args = lambda m, n, inp, ns, u=p16: (u, m, m, n, inp, ns, p32, p32, p32, p256, 1 << 20, ctypes.byref(o), None)
    assert lib.boson_sample(*args(8, 0, ins, 1)) == -2
    assert lib.boson_sample(*args(40, 33, ins, 1)) == -2
    assert lib.boson_sample(*args(2, 3, ins, 1)) == -1      # fewer modes than photons
    assert lib.boson_sample(*args(8, 3, rep, 1)) == -1      # two photons in one input mode
    assert lib.boson_sample(*args(8, 3, far, 1)) == -1      # input mode out of range
    assert lib.boson_sample(*args(8, 3, ins, -1)) == -1
    assert lib.boson_sample(*args(8, 3, ins, 0)) == 0       # no draws: nothing to do
    assert lib.boson_sample(*args(8, 3, ins, 2, u=None)) == -1
    assert lib.boson_sample(*args(8, 3, None, 2)) == -1


def test_argument_errors_of_combine_and_probe(lib):
    """perm_combine_partials validates its arguments (host code only), and the
    FP64 probe rejects bad launch shapes before any launch."""
    parts = (ctypes.c_double * 4)(1.0, 0.0, 0.0, 0.0)
    out = (ctypes.c_double * 4)()
    assert lib.perm_combine_partials(None, 1, 4, 0, out) == -1
    assert lib.perm_combine_partials(parts, 0, 4, 0, out) == -1
    assert lib.perm_combine_partials(parts, 1, 4, 2, out) == -1
    assert lib.perm_combine_partials(parts, 1, 0, 0, out) == -2
    assert lib.perm_combine_partials(parts, 1, 4, 0, out) == 0 and out[0] == 1.0 / 8
    sink = ctypes.c_void_p(256)
    assert lib.perm_fp64_fma_probe(0, 1, 128, sink, None) == -1
    assert lib.perm_fp64_fma_probe(1, 1, 100, sink, None) == -1
    assert lib.perm_fp64_fma_probe(1, 0, 128, sink, None) == -1
    assert lib.perm_fp64_fma_probe(1, 1, 128, None, None) == -1
