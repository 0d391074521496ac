"""Multi-GPU sharding: one large permanent over the Gray index range, and a
batch of permanents by item.

The split is Algorithm 2's (and Algorithm 1's) of arXiv 1606.05836: each rank
takes one contiguous range of the iteration index, here of the Gray index
[0, 2^M) (Glynn M = n-1, Ryser M = n), with lengths differing by at most one.
Each rank computes its un-normalised double-double partial sum on its own GPU
(``perm_glynn_range`` / ``perm_ryser_range``), and the one exchange of the method
— the paper's final MPI reduce of the per-process sums — is an all-gather of the
32-byte partials; every rank then hands them, in rank order, to
``perm_combine_partials`` (double-double sum and the formula's scaling, in the C
library), so all ranks get the same value.

A batch (the many output patterns of one interferometer) shards by item: every
rank derives the same assignment from the item sizes alone (largest work first,
each item to the rank with the least work so far, work ~ 2^n), runs its items in
one batched launch, and one all-gather returns every item's result to every rank.
"""
from __future__ import annotations

import torch


def shard_range(total: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [begin, end) of ``total`` indices for ``rank`` of ``world``."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    q, r = divmod(total, world)
    begin = rank * q + min(rank, r)
    return begin, begin + q + (1 if rank < r else 0)


def exchange_partials(part: tuple[complex, complex], group=None) -> list[tuple[complex, complex]]:
    """All-gather every rank's (hi, lo) complex partial; returns them in rank order."""
    import torch.distributed as dist

    world = dist.get_world_size(group)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    mine = torch.tensor([part[0].real, part[0].imag, part[1].real, part[1].imag], dtype=torch.float64, device=dev)
    bufs = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(bufs, mine, group=group)
    vals = [b.cpu().tolist() for b in bufs]
    return [(complex(v[0], v[1]), complex(v[2], v[3])) for v in vals]


def sharded_permanent(n: int, method: str, partial_fn, rank: int, world: int, group=None) -> complex:
    """Per(A) from per-rank Gray-range partials.

    partial_fn(k_begin, k_end) -> (hi, lo) must return this rank's un-normalised
    partial sum (e.g. a closure over ``paper_1606_05836_gb300.glynn_range`` on this
    rank's GPU).  With world == 1 no collective is used.
    """
    if n == 0:
        return 1.0 + 0.0j
    from . import combine_partials

    M = n - 1 if method == "glynn" else n
    kb, ke = shard_range(1 << M, rank, world)
    part = partial_fn(kb, ke)
    parts = exchange_partials(part, group) if world > 1 else [part]
    hi, lo = combine_partials(parts, n, method)
    return hi + lo


def gpu_partial_fn(A: torch.Tensor, method: str = "glynn", **opts):
    """partial_fn for sharded_permanent running the GPU range kernel on A's device."""
    from . import glynn_range, ryser_range

    f = glynn_range if method == "glynn" else ryser_range

    def run(kb: int, ke: int):
        r = f(A, kb, ke, **opts).cpu()
        return complex(r[0].item()), complex(r[1].item())

    return run


def item_work(n: int, method: str = "glynn") -> int:
    """Gray-code terms of one item: 2^(n-1) (Glynn) or 2^n (Ryser)."""
    return 1 << (n - 1 if method == "glynn" else n) if n > 0 else 1


def shard_items(ns, world: int, method: str = "glynn") -> list[list[int]]:
    """Item indices per rank, balanced by Gray-code work.

    Longest-processing-time order: items by decreasing work (ties by index), each
    to the rank with the least assigned work (ties to the lower rank).  Depends on
    the sizes only, so every rank computes the same lists.  Each list is in
    increasing item order.
    """
    if world < 1:
        raise ValueError("bad world")
    order = sorted(range(len(ns)), key=lambda i: (-item_work(int(ns[i]), method), i))
    load = [0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += item_work(int(ns[i]), method)
    return [sorted(x) for x in out]


def sharded_batched(mats, rank: int, world: int, run_fn, method: str = "glynn", group=None):
    """Per(A_i) of every item, computed by item shards over the ranks.

    run_fn(list_of_matrices) -> sequence of complex results for this rank's items
    (e.g. a closure over ``paper_1606_05836_gb300.batched`` on this rank's GPU).
    Returns the complex results of all items, in item order, on every rank.
    """
    ns = [int(A.shape[0]) for A in mats]
    mine = shard_items(ns, world, method)[rank]
    vals = list(run_fn([mats[i] for i in mine])) if mine else []
    if world == 1:
        return [complex(v) for v in vals]
    import torch.distributed as dist

    pieces = [None] * world
    dist.all_gather_object(pieces, [(i, complex(v)) for i, v in zip(mine, vals)], group=group)
    out = [None] * len(mats)
    for piece in pieces:
        for i, v in piece:
            out[i] = v
    return out


def gpu_batched_fn(device, method: str = "glynn", **opts):
    """run_fn for sharded_batched: the batched kernel on ``device``."""
    from . import batched

    def run(mats):
        per, _ = batched(mats, method=method, device=device, **opts)
        return per.cpu().tolist()

    return run
