"""Row minors and boson-sampling draws (``perm_row_minors`` and ``boson_sample``
in libperm).

``row_minors(M)`` gives the k permanents Per(M without column j) of a (k-1) x k
complex128 CUDA matrix (or a batch of them) from one Gray-code pass of the Glynn
formula, Supp. Eq. (S2) of arXiv 1606.05836, with the free last row's
coefficients read off.

``BosonSampler`` draws output patterns of Eq. (1) for n photons in n distinct
input modes of an m x m unitary: the chain rule over the photons (Clifford and
Clifford, SODA 2018), step k weighing every output mode by the squared
permanent of a k x k submatrix expanded along its last row.  The random photon
orders and uniforms are inputs (device tensors), so a draw is a deterministic
function of them; ``capture()`` records all 2n - 1 launches in one CUDA graph.
"""
from __future__ import annotations

import ctypes

import torch

from . import _native
from ._native import PRECISIONS, Opts
from ._workspace import workspace as _workspace

PERM_MINORS_MAX_K = 32
BOSON_SAMPLE_MAX_N = 32


def _stream(dev):
    return ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def _prec(prec) -> int:
    if prec not in ("fp64", "fp64_df", "fp32x2"):
        raise ValueError("row minors and draws support prec 'fp64', 'fp64_df' or 'fp32x2'")
    return PRECISIONS[prec]


def row_minors(M: torch.Tensor, prec: str = "fp64", chunk_log2: int = 0, grid: int = 0) -> torch.Tensor:
    """m_j = Per(M without column j) for M of shape (k-1, k) or (batch, k-1, k).

    Returns complex128 of shape (k,) or (batch, k).  ``prec`` "fp64_df" takes the
    products in double-float on the FP32 pipe (R3: FP64 row sums); "fp32x2" runs
    the whole walk in double-float (R4).  ``grid`` > 0 fixes the blocks per matrix.
    """
    lib = _native.load()
    if not isinstance(M, torch.Tensor) or not M.is_cuda or M.dtype != torch.complex128:
        raise TypeError("M must be a complex128 CUDA tensor")
    squeeze = M.dim() == 2
    if squeeze:
        M = M.unsqueeze(0)
    if M.dim() != 3 or M.shape[2] != M.shape[1] + 1:
        raise ValueError("M must be (k-1, k) or (batch, k-1, k)")
    M = M.contiguous()
    batch, k = M.shape[0], M.shape[2]
    if k > PERM_MINORS_MAX_K:
        raise ValueError("row_minors supports k <= %d" % PERM_MINORS_MAX_K)
    dev = M.device
    o = Opts(_prec(prec), int(chunk_log2), 0, int(grid), 0)
    out = torch.empty(batch, k, dtype=torch.complex128, device=dev)
    with torch.cuda.device(dev):
        nbytes = int(lib.perm_row_minors_workspace_size(k, batch, ctypes.byref(o)))
        if nbytes == 0:
            raise ValueError("invalid options for perm_row_minors")
        ws = _workspace(dev, nbytes)
        # an empty (0 x 1) matrix has no storage: pass a dummy aligned pointer
        mp = M.data_ptr() if M.numel() else ws.data_ptr()
        st = lib.perm_row_minors(ctypes.c_void_p(mp), k, k, batch, (k - 1) * k, ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(ws.data_ptr()), ws.numel(), ctypes.byref(o), _stream(dev))
    _native.check(st, "perm_row_minors")
    return out[0] if squeeze else out


class BosonSampler:
    """Draws for a fixed unitary U (m x m, complex128, CUDA), input modes and batch size.

    ``run(alpha, unif)`` takes int32 (nsamples, n) photon orders (each row a
    permutation of 0..n-1) and float64 (nsamples, n) uniforms in [0, 1), both on
    U's device, and returns the int32 (nsamples, n) drawn output modes (draw
    order; -1 for a draw with invalid inputs or a step of zero total weight).
    ``prec`` "fp64_df" (R3: FP64 row sums, double-float products) or "fp32x2"
    (R4: the whole walk in double-float) compute the row minors faster; their
    weights differ from FP64's by ~1e-13 .. 1e-12, which can change a draw only
    at a near-tie.
    """

    def __init__(self, U: torch.Tensor, inputs, nsamples: int, prec: str = "fp64", chunk_log2: int = 0,
                 grid: int = 0):
        self.lib = _native.load()
        if not isinstance(U, torch.Tensor) or not U.is_cuda or U.dtype != torch.complex128:
            raise TypeError("U must be a complex128 CUDA tensor")
        if U.dim() != 2 or U.shape[0] != U.shape[1]:
            raise ValueError("U must be m x m")
        self.U = U.contiguous()
        self.m = int(U.shape[0])
        self.inputs = [int(x) for x in inputs]
        self.n = len(self.inputs)
        if not 1 <= self.n <= BOSON_SAMPLE_MAX_N:
            raise ValueError("1 <= n <= %d photons" % BOSON_SAMPLE_MAX_N)
        self.nsamples = int(nsamples)
        self.device = U.device
        self.opts = Opts(_prec(prec), int(chunk_log2), 0, int(grid), 0)
        self.h_inputs = (ctypes.c_int32 * self.n)(*self.inputs)
        with torch.cuda.device(self.device):
            nbytes = int(self.lib.boson_sample_workspace_size(self.m, self.n, self.nsamples, ctypes.byref(self.opts)))
        if nbytes == 0:
            raise ValueError("invalid sizes or options for boson_sample")
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.alpha = torch.zeros(self.nsamples, self.n, dtype=torch.int32, device=self.device)
        self.unif = torch.zeros(self.nsamples, self.n, dtype=torch.float64, device=self.device)
        self.out = torch.empty(self.nsamples, self.n, dtype=torch.int32, device=self.device)
        self.graph = None

    def _launch(self):
        st = self.lib.boson_sample(ctypes.c_void_p(self.U.data_ptr()), self.m, self.m, self.n, self.h_inputs,
                                   self.nsamples, ctypes.c_void_p(self.alpha.data_ptr()),
                                   ctypes.c_void_p(self.unif.data_ptr()), ctypes.c_void_p(self.out.data_ptr()),
                                   ctypes.c_void_p(self.ws.data_ptr()), self.ws.numel(), ctypes.byref(self.opts),
                                   _stream(self.device))
        _native.check(st, "boson_sample")

    def load(self, alpha: torch.Tensor, unif: torch.Tensor):
        """Copy a batch of random inputs into the sampler's device buffers (stream-ordered)."""
        if tuple(alpha.shape) != (self.nsamples, self.n) or tuple(unif.shape) != (self.nsamples, self.n):
            raise ValueError("alpha and unif must be (%d, %d)" % (self.nsamples, self.n))
        self.alpha.copy_(alpha, non_blocking=True)
        self.unif.copy_(unif, non_blocking=True)

    def run(self, alpha: torch.Tensor | None = None, unif: torch.Tensor | None = None) -> torch.Tensor:
        if alpha is not None or unif is not None:
            self.load(alpha, unif)
        with torch.cuda.device(self.device):
            self._launch()
        return self.out

    def capture(self):
        """Record the 2n - 1 launches of one batch of draws in a CUDA graph."""
        s = torch.cuda.Stream(self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(s):
            self.run()  # warm-up outside capture (kernel attributes, occupancy cache)
        torch.cuda.current_stream(self.device).wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run()
        self.graph = g
        return g

    def replay(self) -> torch.Tensor:
        if self.graph is None:
            self.capture()
        self.graph.replay()
        return self.out


def boson_sample(U: torch.Tensor, inputs, alpha: torch.Tensor, unif: torch.Tensor, prec: str = "fp64",
                 chunk_log2: int = 0, grid: int = 0) -> torch.Tensor:
    """One batch of draws (see ``BosonSampler``)."""
    S = BosonSampler(U, inputs, int(alpha.shape[0]), prec=prec, chunk_log2=chunk_log2, grid=grid)
    return S.run(alpha.to(U.device, torch.int32), unif.to(U.device, torch.float64)).clone()
