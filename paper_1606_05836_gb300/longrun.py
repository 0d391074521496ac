"""Checkpointed long runs of one large permanent (n = 40-48 takes minutes to
hours on one GPU).

The Gray index range [0, 2^M) (Glynn M = n-1, Ryser M = n) is cut into fixed
chunks; chunk c is computed by one ``perm_glynn_range`` / ``perm_ryser_range``
launch, and its double-double partial sum is appended to a JSON-lines log,
flushed and fsync'd, before the next chunk starts.  A restarted run reads the log,
skips the chunks it already holds and continues; because each chunk's row sums
are recomputed from scratch at its start, a chunk is re-runnable with no other
state.  Ranks (processes or boxes) take disjoint chunk sets (chunk c belongs to
rank c mod world) and write one log each; ``combine`` reads all logs and sums
the partials in chunk order (deterministic) and scales them (Glynn: / 2^(n-1);
Ryser: x (-1)^n) with ``perm_combine_partials`` — the paper's Algorithms 1/2
split of the iteration range, with the final reduce done from the logs.

Each log line carries a hash of the matrix, the method and the chunking, so a
log from another problem is rejected instead of mixed in.  A line torn by an
interrupted write is skipped (its chunk counts as missing) and the next record
starts on a new line.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np



def problem_key(A, method: str, chunk_log2: int, prec: str) -> str:
    A = np.ascontiguousarray(np.asarray(A, dtype=np.complex128))
    h = hashlib.sha256(A.tobytes())
    h.update(("%s|%d|%d|%s" % (method, A.shape[0], chunk_log2, prec)).encode())
    return h.hexdigest()


def n_chunks(n: int, method: str, chunk_log2: int) -> int:
    M = n - 1 if method == "glynn" else n
    return max(1, 1 << max(0, M - chunk_log2))


def chunk_range(n: int, method: str, chunk_log2: int, c: int) -> tuple[int, int]:
    M = n - 1 if method == "glynn" else n
    size = 1 << min(M, chunk_log2)
    return c * size, min((c + 1) * size, 1 << M)


def read_log(path: str, key: str) -> dict:
    """{chunk: (hi, lo)} from a log; raises if a line belongs to another problem."""
    done = {}
    if not os.path.exists(path):
        return done
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line:
                continue
            try:
                rec = json.loads(line)
            except ValueError:
                continue  # a torn line from an interrupted write: its chunk is recomputed
            if rec.get("key") != key:
                raise ValueError("log %s belongs to another problem" % path)
            done[int(rec["chunk"])] = (complex(*rec["hi"]), complex(*rec["lo"]))
    return done


def append_log(path: str, key: str, chunk: int, kb: int, ke: int, hi: complex, lo: complex):
    rec = {"key": key, "chunk": chunk, "k_begin": kb, "k_end": ke, "hi": [hi.real, hi.imag], "lo": [lo.real, lo.imag]}
    # After an interrupted write the file ends inside a record: start on a fresh
    # line so that the new record stays parsable.
    torn = False
    if os.path.exists(path) and os.path.getsize(path) > 0:
        with open(path, "rb") as f:
            f.seek(-1, os.SEEK_END)
            torn = f.read(1) != b"\n"
    with open(path, "a") as f:
        f.write(("\n" if torn else "") + json.dumps(rec) + "\n")
        f.flush()
        os.fsync(f.fileno())


def run(A, log_path: str, partial_fn, method: str = "glynn", chunk_log2: int = 34, prec: str = "fp64",
        rank: int = 0, world: int = 1, max_chunks: int | None = None) -> int:
    """Compute this rank's missing chunks (at most max_chunks of them); returns
    the number of chunks computed.  partial_fn(k_begin, k_end) -> (hi, lo)."""
    A = np.asarray(A)
    n = A.shape[0]
    key = problem_key(A, method, chunk_log2, prec)
    done = read_log(log_path, key)
    computed = 0
    for c in range(rank, n_chunks(n, method, chunk_log2), world):
        if c in done:
            continue
        if max_chunks is not None and computed >= max_chunks:
            break
        kb, ke = chunk_range(n, method, chunk_log2, c)
        hi, lo = partial_fn(kb, ke)
        append_log(log_path, key, c, kb, ke, hi, lo)
        computed += 1
    return computed


def combine(A, log_paths, method: str = "glynn", chunk_log2: int = 34, prec: str = "fp64"):
    """Per(A) from the logs of all ranks, or None while chunks are missing."""
    A = np.asarray(A)
    n = A.shape[0]
    key = problem_key(A, method, chunk_log2, prec)
    done = {}
    for p in log_paths:
        done.update(read_log(p, key))
    total = n_chunks(n, method, chunk_log2)
    if any(c not in done for c in range(total)):
        return None
    from . import combine_partials

    hi, lo = combine_partials([done[c] for c in range(total)], n, method)
    return hi + lo


def gpu_run(A, log_path: str, method: str = "glynn", chunk_log2: int = 34, prec: str = "fp64", rank: int = 0,
            world: int = 1, max_chunks: int | None = None, device=None) -> int:
    """``run`` with the GPU range kernel on ``device`` (default: current)."""
    import torch

    from .shard import gpu_partial_fn

    dA = torch.as_tensor(np.ascontiguousarray(np.asarray(A, dtype=np.complex128)))
    dA = dA.to(device if device is not None else torch.device("cuda", torch.cuda.current_device()))
    fn = gpu_partial_fn(dA, method, prec=prec)
    return run(A, log_path, fn, method=method, chunk_log2=chunk_log2, prec=prec, rank=rank, world=world,
               max_chunks=max_chunks)
