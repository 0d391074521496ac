"""perm_glynn_noalloc: Glynn permanents without any device allocation by the caller
or the library — for callers that may not allocate GPU memory (an embedding
application that owns the GPU's memory budget, or a path that must not call
cudaMalloc because it can synchronise the device).  Its scratch is a fixed array
inside libperm.

Called through the C ABI (ctypes) and compared with perm_glynn, the entry point
that takes a caller workspace, on two calls in a row, and with the CPU oracle
(quad precision) on calls that alternate between two matrices, so that partial
sums left in the shared array by one call cannot pass for the next one's.  This
file is collected last on purpose; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synthetic as S

pytestmark = pytest.mark.gpu

REL_TOL = 1e-10


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_1606_05836_gb300 import build, _native
    build.build()
    torch.cuda.init()
    return _native.load()


def _dev(A):
    import torch
    return torch.as_tensor(np.ascontiguousarray(A, dtype=np.complex128)).cuda()


def _glynn_with_workspace(lib, dA, n, stream):
    import torch
    from paper_1606_05836_gb300._native import Opts
    o = Opts(0, 0, 0, 0, 0)
    ws_bytes = lib.perm_workspace_size(n, ctypes.byref(o))
    assert ws_bytes > 0
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    out = torch.empty(1, dtype=torch.complex128, device="cuda")
    st = lib.perm_glynn(ctypes.c_void_p(dA.data_ptr()), n, n, ctypes.c_void_p(out.data_ptr()),
                        ctypes.c_void_p(ws.data_ptr()), ws_bytes, ctypes.byref(o), ctypes.c_void_p(stream))
    assert st == 0, st
    return out


def _glynn_noalloc(lib, dA, n, stream, opts=None):
    import torch
    from paper_1606_05836_gb300._native import Opts
    o = opts or Opts(0, 0, 0, 0, 0)
    out = torch.empty(1, dtype=torch.complex128, device="cuda")
    st = lib.perm_glynn_noalloc(ctypes.c_void_p(dA.data_ptr()), n, n, ctypes.c_void_p(out.data_ptr()),
                                ctypes.byref(o), ctypes.c_void_p(stream))
    return st, out


@pytest.mark.parametrize("n,seed", [(20, 3), (24, 4)])
def test_noalloc_matches_workspace_entry_point_twice(lib, n, seed):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    A = S.gaussian(n, seed)
    dA = _dev(A)
    want = complex(_glynn_with_workspace(lib, dA, n, stream).cpu().item())
    for _ in range(2):  # the shared scratch keeps the previous call's contents
        st, out = _glynn_noalloc(lib, dA, n, stream)
        assert st == 0, st
        got = complex(out.cpu().item())
        assert abs(got - want) <= REL_TOL * abs(want), (got, want)


def test_noalloc_against_the_oracle_alternating_matrices(lib):
    """Two different n = 20 matrices, A B A B: every result within 1e-10 of the
    quad-precision Glynn oracle."""
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    mats = [S.gaussian(20, 31), S.gaussian(20, 32)]
    want = [oracle.glynn(A) for A in mats]
    devs = [_dev(A) for A in mats]
    for call in range(4):
        k = call % 2
        st, out = _glynn_noalloc(lib, devs[k], 20, stream)
        assert st == 0, st
        assert want[k].rel_err(complex(out.cpu().item())) < REL_TOL, (call, k)


def test_noalloc_rejects_grid_beyond_its_scratch(lib):
    import torch
    from paper_1606_05836_gb300._native import Opts
    stream = torch.cuda.current_stream().cuda_stream
    dA = _dev(S.gaussian(12, 5))
    st, _ = _glynn_noalloc(lib, dA, 12, stream, Opts(0, 0, 0, 4097, 0))
    assert st == -3  # PERM_ENOMEM: more blocks than the fixed partial-sum array holds
    st, out = _glynn_noalloc(lib, dA, 12, stream, Opts(0, 0, 0, 4096, 0))
    assert st == 0
