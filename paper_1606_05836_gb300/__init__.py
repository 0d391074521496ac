"""GB300 (sm_103a) engine for matrix permanents — the boson-sampling hot path.

Thin Python binding over the C ABI in ``include/perm.h`` (``libperm.so``):
argument marshalling only.  Every step of the computation runs in the CUDA
kernels of ``csrc/``; PyTorch is used for device memory and streams.  There is
no CPU fallback: calls raise if the library is missing or no GPU is present.

Functions mirror the C entry points:

* :func:`glynn`  -- Per(A), BB/FG formula (Supp. Eq. (S2), Algorithm 2 of arXiv 1606.05836)
* :func:`ryser`  -- Per(A), Ryser formula (Supp. Eq. (S1), Algorithm 1)
* :func:`ryser_nw` -- Per(A), Ryser's formula halved to 2^(n-1) subsets
* :func:`glynn_mult` -- Per with repeated columns (photon collisions), multiplicity expansion
* :func:`glynn_range`, :func:`ryser_range` -- partial sums over a Gray-index range
* :func:`combine_partials` -- Per(A) from such partials (the final reduce of
  Algorithms 1/2 and the normalisation), host arithmetic in the C library
* :func:`batched`, :class:`BatchedPermanents` -- many permanents of mixed sizes in
  one persistent launch (CUDA-graph capture, autotuned launch shape)
* :func:`prob` -- Eq. (1): |Per(U_ST)|^2 / (prod s_i! prod t_j!) for one (S, T)
* :func:`grad`, :class:`PermAbs2` -- the adjoint: dPer/dA and d|Per|^2/dA in the
  same Gray-code pass, behind a torch.autograd.Function
* :func:`row_minors` -- the k permanents Per(M without column j) of a (k-1) x k matrix
* :class:`BosonSampler`, :func:`boson_sample` -- draws from Eq. (1) by the chain rule
  over the photons, each step one row-minor pass (CUDA-graph capture)
"""
from __future__ import annotations

import ctypes

import torch

from . import _native
from ._native import PERM_MAX_N, PRECISIONS, Opts, PermError
from ._workspace import workspace as _workspace

__all__ = ["glynn", "glynn_mult", "ryser", "ryser_nw", "glynn_range", "ryser_range", "combine_partials",
           "fp64_fma_probe", "workspace_size", "PermError",
           "PERM_MAX_N", "PRECISIONS", "library", "batched", "BatchedPermanents", "grad", "PermAbs2", "prob",
           "row_minors", "BosonSampler", "boson_sample"]


def library():
    """The loaded ctypes library (raises if libperm.so is missing)."""
    return _native.load()


def _opts(prec="fp64", chunk_log2=0, block=0, grid=0, unit_log2=0):
    if isinstance(prec, str):
        if prec not in PRECISIONS:
            raise ValueError("prec must be one of %s" % sorted(PRECISIONS))
        prec = PRECISIONS[prec]
    return Opts(int(prec), int(chunk_log2), int(block), int(grid), int(unit_log2))


def _matrix(A: torch.Tensor):
    if not isinstance(A, torch.Tensor) or not A.is_cuda:
        raise TypeError("A must be a CUDA tensor")
    if A.dtype != torch.complex128:
        raise TypeError("A must be complex128")
    if A.dim() != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("A must be square, got %s" % (tuple(A.shape),))
    n = A.shape[0]
    if n > 0 and (A.stride(1) != 1 or A.stride(0) < n):
        A = A.contiguous()
    lda = A.stride(0) if n > 0 else 0
    return A, n, max(lda, n)


def _stream_ptr(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def workspace_size(n: int, **opts) -> int:
    o = _opts(**opts)
    return int(library().perm_workspace_size(int(n), ctypes.byref(o)))


def _run(fname, A, extra, out_len, **opts):
    lib = library()
    A, n, lda = _matrix(A)
    o = _opts(**opts)
    dev = A.device
    out = torch.empty(out_len, dtype=torch.complex128, device=dev)
    ws_bytes = int(lib.perm_workspace_size(int(n), ctypes.byref(o)))
    ws = _workspace(dev, ws_bytes)
    with torch.cuda.device(dev):
        st = getattr(lib, fname)(ctypes.c_void_p(A.data_ptr()), n, lda, *extra, ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(ws.data_ptr()), ws.numel(), ctypes.byref(o),
                                 ctypes.c_void_p(_stream_ptr(dev)))
    _native.check(st, fname)
    return out


def glynn(A: torch.Tensor, prec="fp64", chunk_log2=0, block=0, grid=0) -> torch.Tensor:
    """Per(A) by the Gray-ordered BB/FG (Glynn) sum; returns a 0-dim complex128 CUDA tensor."""
    return _run("perm_glynn", A, (), 1, prec=prec, chunk_log2=chunk_log2, block=block, grid=grid)[0]


def ryser(A: torch.Tensor, prec="fp64", chunk_log2=0, block=0, grid=0) -> torch.Tensor:
    """Per(A) by the Gray-ordered Ryser sum; returns a 0-dim complex128 CUDA tensor."""
    return _run("perm_ryser", A, (), 1, prec=prec, chunk_log2=chunk_log2, block=block, grid=grid)[0]


def prob(U: torch.Tensor, s, t, prec="fp64", chunk_log2=0, block=0, grid=0):
    """Eq. (1) for input occupations s and output occupations t of the m x m unitary U
    (complex128 CUDA tensor, U[i][j] = amplitude input i -> output j).  Returns
    (probability, Per(U_ST)) as Python numbers; synchronises the current stream."""
    import numpy as np

    lib = library()
    U, m, ldu = _matrix(U)
    s = np.ascontiguousarray(np.asarray(s, dtype=np.int32))
    t = np.ascontiguousarray(np.asarray(t, dtype=np.int32))
    if s.shape != (m,) or t.shape != (m,):
        raise ValueError("occupation vectors must have length m = %d" % m)
    n = int(s.sum())
    o = _opts(prec=prec, chunk_log2=chunk_log2, block=block, grid=grid)
    dev = U.device
    with torch.cuda.device(dev):
        nbytes = int(lib.prob_sample_workspace_size(n, ctypes.byref(o)))
        if nbytes == 0:
            raise ValueError("photon number %d outside 0..%d" % (n, PERM_MAX_N))
        ws = _workspace(dev, nbytes + 256)
        base = (ws.data_ptr() + 255) & ~255
        p = ctypes.c_double(0.0)
        per = (ctypes.c_double * 2)()
        i32p = ctypes.POINTER(ctypes.c_int32)
        st = lib.prob_sample(ctypes.c_void_p(U.data_ptr()), m, ldu, s.ctypes.data_as(i32p), t.ctypes.data_as(i32p),
                             ctypes.byref(p), ctypes.cast(per, ctypes.c_void_p), ctypes.c_void_p(base),
                             nbytes, ctypes.byref(o), ctypes.c_void_p(_stream_ptr(dev)))
    _native.check(st, "prob_sample")
    return p.value, complex(per[0], per[1])


def glynn_mult(B: torch.Tensor, mult, prec="fp64", chunk_log2=0, block=0, grid=0) -> torch.Tensor:
    """Per of the n x n matrix whose columns are B[:, c] repeated mult[c] times
    (B: n x g complex128 CUDA tensor, sum(mult) = n), by the multiplicity expansion
    of the Glynn sum; returns a 0-dim complex128 CUDA tensor."""
    import numpy as np

    lib = library()
    if not isinstance(B, torch.Tensor) or not B.is_cuda or B.dtype != torch.complex128 or B.dim() != 2:
        raise TypeError("B must be a 2-D complex128 CUDA tensor")
    B = B.contiguous()
    n, g = B.shape
    mult = np.ascontiguousarray(np.asarray(mult, dtype=np.int32))
    if mult.shape != (g,):
        raise ValueError("mult must have one entry per column of B")
    o = _opts(prec=prec, chunk_log2=chunk_log2, block=block, grid=grid)
    i32p = ctypes.POINTER(ctypes.c_int32)
    dev = B.device
    out = torch.empty(1, dtype=torch.complex128, device=dev)
    with torch.cuda.device(dev):
        nbytes = int(lib.perm_glynn_mult_workspace_size(n, g, mult.ctypes.data_as(i32p), ctypes.byref(o)))
        if nbytes == 0:
            raise ValueError("invalid multiplicities %s for n = %d" % (mult.tolist(), n))
        ws = _workspace(dev, nbytes + 256)
        base = (ws.data_ptr() + 255) & ~255
        st = lib.perm_glynn_mult(ctypes.c_void_p(B.data_ptr()), n, g, g, mult.ctypes.data_as(i32p),
                                 ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(base), nbytes, ctypes.byref(o),
                                 ctypes.c_void_p(_stream_ptr(dev)))
    _native.check(st, "perm_glynn_mult")
    return out[0]


def ryser_nw(A: torch.Tensor, prec="fp64", chunk_log2=0, block=0, grid=0) -> torch.Tensor:
    """Per(A) by Ryser's formula over 2^(n-1) subsets (Nijenhuis-Wilf form); 0-dim complex128."""
    return _run("perm_ryser_nw", A, (), 1, prec=prec, chunk_log2=chunk_log2, block=block, grid=grid)[0]


def _range(fname, A, k_begin, k_end, **opts):
    out = _run(fname, A, (ctypes.c_uint64(int(k_begin)), ctypes.c_uint64(int(k_end))), 2, **opts)
    return out  # (hi, lo)


def glynn_range(A, k_begin: int, k_end: int, prec="fp64", chunk_log2=0, block=0, grid=0) -> torch.Tensor:
    """Un-normalised Glynn partial sum over Gray indices [k_begin, k_end): tensor (hi, lo)."""
    return _range("perm_glynn_range", A, k_begin, k_end, prec=prec, chunk_log2=chunk_log2, block=block, grid=grid)


def ryser_range(A, k_begin: int, k_end: int, prec="fp64", chunk_log2=0, block=0, grid=0) -> torch.Tensor:
    """Un-normalised Ryser partial sum over Gray indices [k_begin, k_end): tensor (hi, lo)."""
    return _range("perm_ryser_range", A, k_begin, k_end, prec=prec, chunk_log2=chunk_log2, block=block, grid=grid)


def combine_partials(parts, n: int, method: str = "glynn") -> tuple[complex, complex]:
    """Per(A) as (hi, lo) from (hi, lo) partial sums over disjoint Gray ranges that
    cover the whole index space, summed in the given order (``perm_combine_partials``;
    host arithmetic, no device needed)."""
    import numpy as np

    if method not in ("glynn", "ryser"):
        raise ValueError("method must be 'glynn' or 'ryser'")
    buf = np.ascontiguousarray(np.asarray([[complex(h), complex(l)] for h, l in parts], dtype=np.complex128))
    if buf.ndim != 2 or buf.shape[0] < 1:
        raise ValueError("at least one (hi, lo) partial is needed")
    out = np.zeros(2, dtype=np.complex128)
    st = library().perm_combine_partials(ctypes.c_void_p(buf.ctypes.data), buf.shape[0], int(n),
                                         0 if method == "glynn" else 1, ctypes.c_void_p(out.ctypes.data))
    _native.check(st, "perm_combine_partials")
    return complex(out[0]), complex(out[1])


def fp64_fma_probe(iters: int, grid: int, block: int = 256, device=None) -> int:
    """Launch the FP64 FMA throughput probe on the current stream of ``device``;
    returns the number of DFMA instructions it issues (time it with CUDA events)."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    sink = _workspace(dev, 256)
    with torch.cuda.device(dev):
        st = library().perm_fp64_fma_probe(int(iters), int(grid), int(block), ctypes.c_void_p(sink.data_ptr()),
                                           ctypes.c_void_p(_stream_ptr(dev)))
    _native.check(st, "perm_fp64_fma_probe")
    return int(iters) * int(grid) * int(block) * 4


from .batch import BatchedPermanents, batched  # noqa: E402
from .grad import PermAbs2, grad  # noqa: E402
from .sampler import BosonSampler, boson_sample, row_minors  # noqa: E402
