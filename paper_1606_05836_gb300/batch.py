"""Batched permanents: packing, CUDA-graph capture and the launch-shape autotuner.

``BatchedPermanents`` packs many matrices of mixed sizes (n <= 32) into one
device buffer and runs ``perm_batched`` (one planner, one prep, ONE persistent
size-bucketed walk kernel, one per-item reduce — all in libperm) on the current
stream; ``capture()`` records that sequence once in a CUDA graph so that each
replay is a single graph launch.  ``autotune()`` times replays for a few
(unit size, block size) shapes and caches the winner in a JSON file keyed by
(GPU name, method, precision, size histogram).
"""
from __future__ import annotations

import ctypes
import hashlib
import json
import os

import numpy as np
import torch

from . import _native
from ._native import Opts, PRECISIONS

PERM_BATCH_MAX_N = 32
METHODS = {"glynn": 0, "ryser": 1}

TUNE_CACHE = os.environ.get("PERM_TUNE_CACHE",
                            os.path.join(os.path.expanduser("~"), ".cache", "paper_1606_05836_gb300",
                                         "batched_tune.json"))


class BatchedPermanents:
    """A packed batch bound to device buffers; ``run()`` computes every permanent.

    mats: sequence of square complex matrices (numpy or torch), 1 <= n <= 32.
    scale: optional per-item factors; ``prob`` = |Per|^2 * scale (Eq. (1) with
    scale = 1/(prod s_i! prod t_j!)).
    """

    def __init__(self, mats, method="glynn", scale=None, prec="fp64", chunk_log2=0, unit_log2=0, block=0, grid=0,
                 device=None):
        self.lib = _native.load()
        device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.device = device
        if method not in METHODS:
            raise ValueError("method must be glynn or ryser")
        self.method = method
        flat, ns, offs = [], [], []
        off = 0
        for m in mats:
            t = torch.as_tensor(m)
            if t.dim() != 2 or t.shape[0] != t.shape[1]:
                raise ValueError("square matrices expected")
            n = int(t.shape[0])
            if not 1 <= n <= PERM_BATCH_MAX_N:
                raise ValueError("batched sizes must be 1..%d, got %d" % (PERM_BATCH_MAX_N, n))
            flat.append(t.to(torch.complex128).reshape(-1))
            ns.append(n)
            offs.append(off)
            off += n * n
        self.count = len(ns)
        self.hN = np.ascontiguousarray(np.array(ns, dtype=np.int32))
        self.packed = (torch.cat([f.to(device) for f in flat]) if flat
                       else torch.empty(0, dtype=torch.complex128, device=device))
        self.offsets = torch.tensor(offs, dtype=torch.int64, device=device)
        self.ns = torch.tensor(ns, dtype=torch.int32, device=device)
        self.scale = (torch.as_tensor(np.asarray(scale, dtype=np.float64)).to(device) if scale is not None else None)
        self.out = torch.empty(self.count, dtype=torch.complex128, device=device)
        self.prob = torch.empty(self.count, dtype=torch.float64, device=device)
        self.set_options(prec=prec, chunk_log2=chunk_log2, unit_log2=unit_log2, block=block, grid=grid)
        self.graph = None

    def set_options(self, prec="fp64", chunk_log2=0, unit_log2=0, block=0, grid=0):
        p = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
        self.prec = prec
        self.opts = Opts(p, int(chunk_log2), int(block), int(grid), int(unit_log2))
        hn = self.hN.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        nbytes = int(self.lib.perm_batched_workspace_size(self.count, hn, METHODS[self.method],
                                                          ctypes.byref(self.opts)))
        if self.count and nbytes == 0:
            raise ValueError("invalid batched options or sizes")
        self.work = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
        self.graph = None

    def run(self):
        """Launch the batched pipeline on the current stream; returns (per, prob)."""
        if self.count == 0:
            return self.out, self.prob
        stream = torch.cuda.current_stream(self.device).cuda_stream
        hn = self.hN.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        with torch.cuda.device(self.device):
            st = self.lib.perm_batched(
                ctypes.c_void_p(self.packed.data_ptr()), ctypes.c_void_p(self.offsets.data_ptr()),
                ctypes.c_void_p(self.ns.data_ptr()), hn, self.count, METHODS[self.method],
                ctypes.c_void_p(self.scale.data_ptr() if self.scale is not None else 0),
                ctypes.c_void_p(self.out.data_ptr()), ctypes.c_void_p(self.prob.data_ptr()),
                ctypes.c_void_p(self.work.data_ptr()), self.work.numel(), ctypes.byref(self.opts),
                ctypes.c_void_p(stream))
        _native.check(st, "perm_batched")
        return self.out, self.prob

    def capture(self):
        """Record run() once in a CUDA graph (warm-up run first); returns the graph."""
        s = torch.cuda.Stream(self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(s):
            self.run()  # warm-up outside capture (sets kernel attributes, loads modules)
        torch.cuda.current_stream(self.device).wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run()
        self.graph = g
        return g

    def replay(self):
        if self.graph is None:
            self.capture()
        self.graph.replay()
        return self.out, self.prob

    # ------------------------------------------------------------------ tuning
    def signature(self) -> str:
        hist = np.bincount(self.hN, minlength=PERM_BATCH_MAX_N + 1).tolist()
        name = torch.cuda.get_device_name(self.device)
        key = json.dumps([name, self.method, str(self.prec), hist])
        return hashlib.sha1(key.encode()).hexdigest()

    def autotune(self, candidates=None, reps=2, use_cache=True):
        """Pick (unit_log2, block) by timing graph replays; cached per signature."""
        sig = self.signature()
        cache = _load_cache() if use_cache else {}
        if sig in cache:
            best = cache[sig]
            self.set_options(prec=self.prec, unit_log2=best["unit_log2"], block=best["block"])
            return best
        if candidates is None:
            candidates = [(u, b) for u in (9, 11, 13) for b in (64, 128, 256)]
        results = []
        for u, b in candidates:
            self.set_options(prec=self.prec, unit_log2=u, block=b)
            self.capture()
            times = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                self.graph.replay()
                e1.record()
                torch.cuda.synchronize(self.device)
                times.append(e0.elapsed_time(e1))
            results.append((min(times), u, b))
        results.sort()
        t, u, b = results[0]
        best = {"unit_log2": u, "block": b, "ms": t, "tried": [[r[1], r[2], r[0]] for r in results]}
        self.set_options(prec=self.prec, unit_log2=u, block=b)
        if use_cache:
            cache[sig] = best
            _save_cache(cache)
        return best


def _load_cache():
    try:
        with open(TUNE_CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save_cache(cache):
    try:
        os.makedirs(os.path.dirname(TUNE_CACHE), exist_ok=True)
        tmp = TUNE_CACHE + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, TUNE_CACHE)
    except OSError:
        pass


def batched(mats, method="glynn", scale=None, prec="fp64", **opts):
    """Per of every matrix (and |Per|^2 * scale) in one batched launch; returns (per, prob)."""
    b = BatchedPermanents(mats, method=method, scale=scale, prec=prec, **opts)
    return b.run()
