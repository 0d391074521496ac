"""Scratch buffers for the C calls' caller-owned workspaces.

One growable device buffer per (device, stream): calls on one stream run in
order, so the next call may reuse the buffer while the previous kernels are
still queued; calls on different streams get different buffers.
"""
from __future__ import annotations

import torch

_cache: dict = {}


def workspace(device, nbytes: int) -> torch.Tensor:
    """A uint8 device tensor of at least ``nbytes`` (256-byte aligned) for the current stream."""
    key = (device.index, torch.cuda.current_stream(device).cuda_stream)
    buf = _cache.get(key)
    if buf is None or buf.numel() < nbytes:
        _cache.pop(key, None)
        buf = torch.empty(max(int(nbytes), 4096), dtype=torch.uint8, device=device)
        _cache[key] = buf
    return buf
