"""The adjoint form: Per, |Per|^2 and their derivatives in one Gray-code pass
(``perm_grad`` in libperm), and a ``torch.autograd.Function`` on top of it.

``PermAbs2.apply(A)`` maps a (batch, n, n) or (n, n) complex128 CUDA tensor to
|Per(A_b)|^2 (float64).  Its forward already produces d|Per|^2/dA in PyTorch's
convention for real losses (d/dRe a + i d/dIm a = 2 Per conj(dPer/da)), so the
backward pass only scales the saved tensor by the upstream gradient.
"""
from __future__ import annotations

import ctypes

import torch

from . import _native
from ._native import PRECISIONS, Opts
from ._workspace import workspace as _workspace

PERM_GRAD_MAX_N = 32


def grad(A: torch.Tensor, minor: bool = True, grad_abs2: bool = False, chunk_log2: int = 0, grid: int = 0,
         prec: str = "fp64"):
    """Per(A_b), |Per(A_b)|^2 and, on request, dPer/da_ij and 2 Per conj(dPer/da_ij).

    prec: "fp64" (default) or "fp64_df" (the products in double-float on the FP32
    pipe; row sums, accumulators and the flips in FP64).
    Returns (per[batch], abs2[batch], minor[batch, n, n] or None, grad_abs2[batch, n, n] or None);
    a 2-D input gives 0-dim / 2-D results.
    """
    lib = _native.load()
    if not isinstance(A, torch.Tensor) or not A.is_cuda or A.dtype != torch.complex128:
        raise TypeError("A must be a complex128 CUDA tensor")
    squeeze = A.dim() == 2
    if squeeze:
        A = A.unsqueeze(0)
    if A.dim() != 3 or A.shape[1] != A.shape[2]:
        raise ValueError("A must be (n, n) or (batch, n, n)")
    A = A.contiguous()
    batch, n = A.shape[0], A.shape[1]
    if n > PERM_GRAD_MAX_N:
        raise ValueError("perm_grad supports n <= %d" % PERM_GRAD_MAX_N)
    dev = A.device
    if prec not in ("fp64", "fp64_df"):
        raise ValueError("perm_grad supports prec 'fp64' and 'fp64_df'")
    o = Opts(PRECISIONS[prec], int(chunk_log2), 0, int(grid), 0)
    per = torch.empty(batch, dtype=torch.complex128, device=dev)
    abs2 = torch.empty(batch, dtype=torch.float64, device=dev)
    M = torch.empty(batch, n, n, dtype=torch.complex128, device=dev) if minor else None
    G = torch.empty(batch, n, n, dtype=torch.complex128, device=dev) if grad_abs2 else None
    with torch.cuda.device(dev):
        nbytes = int(lib.perm_grad_workspace_size(n, ctypes.byref(o)))
        if nbytes == 0:
            raise ValueError("invalid options for perm_grad")
        ws = _workspace(dev, nbytes)
        st = lib.perm_grad(ctypes.c_void_p(A.data_ptr()), n, n, batch, n * n, ctypes.c_void_p(per.data_ptr()),
                           ctypes.c_void_p(abs2.data_ptr()), ctypes.c_void_p(M.data_ptr() if M is not None else 0),
                           ctypes.c_void_p(G.data_ptr() if G is not None else 0), ctypes.c_void_p(ws.data_ptr()),
                           ws.numel(), ctypes.byref(o), ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream))
    _native.check(st, "perm_grad")
    if squeeze:
        return per[0], abs2[0], (M[0] if M is not None else None), (G[0] if G is not None else None)
    return per, abs2, M, G


class PermAbs2(torch.autograd.Function):
    """|Per(A)|^2 with its gradient from the adjoint kernel."""

    @staticmethod
    def forward(ctx, A):
        _, abs2, _, g = grad(A.detach(), minor=False, grad_abs2=True)
        ctx.save_for_backward(g)
        return abs2

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        if g.dim() == 2:
            return grad_out * g
        return grad_out[:, None, None] * g
