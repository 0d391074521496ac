"""Sharding of one permanent over ranks (the Gray-range split of Algorithms 1/2
and the final reduce of the per-rank sums), tested on CPU with gloo ranks and
the oracle computing each rank's partial; and on one GPU as K logical shards."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
import synthetic as S
from paper_1606_05836_gb300 import combine_partials
from paper_1606_05836_gb300.shard import item_work, shard_items, shard_range, sharded_batched, sharded_permanent


def test_shard_range_partitions_exactly():
    for total in (0, 1, 7, 1 << 20, (1 << 39) + 5):
        for world in (1, 2, 3, 8, 13):
            ranges = [shard_range(total, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == total
            for (a, b), (c, d) in zip(ranges, ranges[1:]):
                assert b == c
            lens = [b - a for a, b in ranges]
            assert max(lens) - min(lens) <= 1


def test_combine_partials_double_double_and_scaling():
    """perm_combine_partials (host code of the C library): the partials cancel
    exactly in double-double, Glynn scales by 2^-(n-1), Ryser by (-1)^n, and it
    matches the oracle's full sum when handed the oracle's range partials."""
    parts = [(1e16 + 0j, 1.0 + 0j), (-1e16 + 2j, 0.5 + 0j), (3.0 + 0j, 0j)]
    hi, lo = combine_partials(parts, 1, "glynn")
    assert hi + lo == 4.5 + 2j
    hi, lo = combine_partials(parts, 4, "glynn")
    assert hi + lo == (4.5 + 2j) / 8
    hi, lo = combine_partials(parts, 3, "ryser")
    assert hi + lo == -(4.5 + 2j)
    A = S.gaussian(13, 5)
    cuts = [0, 17, 1000, 4095, 1 << 12]
    g = [oracle.glynn_range(A, a, b, gray=True) for a, b in zip(cuts[:-1], cuts[1:])]
    hi, lo = combine_partials([(p.hi, p.lo) for p in g], 13, "glynn")
    assert oracle.glynn(A).rel_err(hi + lo) < 1e-15
    cuts = [0, 5, 3000, 1 << 13]
    r = [oracle.ryser_range(A, a, b, gray=True) for a, b in zip(cuts[:-1], cuts[1:])]
    hi, lo = combine_partials([(p.hi, p.lo) for p in r], 13, "ryser")
    assert oracle.ryser(A).rel_err(hi + lo) < 1e-15
    import pytest as _pt
    from paper_1606_05836_gb300 import PermError
    with _pt.raises(PermError):
        combine_partials(parts, 0, "glynn")
    with _pt.raises(PermError):
        combine_partials(parts, 49, "ryser")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, n, method, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    A = S.gaussian(n, 77)
    f = oracle.glynn_range if method == "glynn" else oracle.ryser_range

    def partial(kb, ke):
        r = f(A, kb, ke, gray=True, threads=1)
        return r.hi, r.lo

    per = sharded_permanent(n, method, partial, rank, world)
    q.put((rank, per))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("method", ["glynn", "ryser"])
def test_gloo_two_ranks_equal_the_full_sum(method):
    n, world = 11, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, n, method, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(world))
    want = oracle.ryser(S.gaussian(n, 77))
    for r in range(world):
        assert want.rel_err(got[r]) < 1e-14
    assert got[0] == got[1]  # every rank sums the gathered partials in the same order


@pytest.mark.gpu
def test_logical_shards_on_one_gpu():
    """K logical shards (disjoint Gray ranges on one GPU) add up to the single launch."""
    import torch
    import paper_1606_05836_gb300 as pg
    from paper_1606_05836_gb300.shard import gpu_partial_fn
    A = S.gaussian(26, 88)
    dA = torch.as_tensor(A).cuda()
    full = complex(pg.glynn(dA).cpu().item())
    fn = gpu_partial_fn(dA, "glynn")
    K = 5
    parts = [fn(*shard_range(1 << 25, r, K)) for r in range(K)]
    hi, lo = combine_partials(parts, 26, "glynn")
    assert abs((hi + lo) - full) <= 1e-12 * abs(full)
    assert abs(sharded_permanent(26, "glynn", fn, 0, 1) - full) <= 1e-12 * abs(full)


def _dying_rank_main(rank, world, port, q):
    import datetime
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    A = S.gaussian(9, 78)
    if rank == 1:
        os._exit(0)  # this rank fails before the exchange of partials

    def partial(kb, ke):
        r = oracle.glynn_range(A, kb, ke, gray=True, threads=1)
        return r.hi, r.lo

    try:
        sharded_permanent(9, "glynn", partial, rank, world)
        q.put("no error")
    except Exception as e:  # the surviving rank must see an error, not hang
        q.put("error: %s" % type(e).__name__)


def test_a_dead_rank_fails_the_exchange_instead_of_hanging():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dying_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(90)
    alive = [p for p in procs if p.is_alive()]
    for p in alive:
        p.kill()
    assert not alive, "a rank hung"
    msg = q.get(timeout=10)
    assert msg.startswith("error"), msg


def test_shard_items_covers_and_balances():
    g = np.random.default_rng(3)
    ns = [int(x) for x in g.integers(8, 25, size=500)]
    for world in (1, 2, 3, 8):
        parts = shard_items(ns, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(ns)))
        assert parts == shard_items(ns, world)  # every rank derives the same lists
        loads = [sum(item_work(ns[i]) for i in p) for p in parts]
        # greedy LPT: no rank exceeds the mean by more than the largest item
        assert max(loads) <= sum(loads) / world + max(item_work(n) for n in ns)


def _batched_rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = np.random.default_rng(11)
    mats = [S.gaussian(int(n), 500 + i) for i, n in enumerate(g.integers(3, 11, size=17))]

    def run(ms):
        return [complex(oracle.perm_def(A).hi) for A in ms]

    q.put((rank, sharded_batched(mats, rank, world, run)))
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_two_ranks_batched_by_item():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_batched_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(world))
    g = np.random.default_rng(11)
    mats = [S.gaussian(int(n), 500 + i) for i, n in enumerate(g.integers(3, 11, size=17))]
    want = [complex(oracle.perm_def(A).hi) for A in mats]
    assert got[0] == got[1] == want


@pytest.mark.gpu
def test_logical_item_shards_on_one_gpu():
    """Three item shards, run one after another on one GPU, equal one batched launch bit for bit."""
    import torch
    from paper_1606_05836_gb300 import batched
    from paper_1606_05836_gb300.shard import gpu_batched_fn
    g = np.random.default_rng(12)
    mats = [S.gaussian(int(n), 600 + i) for i, n in enumerate(g.integers(8, 21, size=40))]
    whole, _ = batched(mats)
    whole = whole.cpu().tolist()
    fn = gpu_batched_fn(torch.device("cuda", 0))
    parts = shard_items([A.shape[0] for A in mats], 3)
    out = [None] * len(mats)
    for p in parts:
        for i, v in zip(p, fn([mats[i] for i in p])):
            out[i] = v
    assert out == whole


def _gpu_rank_main(rank, world, port, n, q):
    import torch
    import torch.distributed as dist
    from paper_1606_05836_gb300.shard import gpu_partial_fn
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dA = torch.as_tensor(S.gaussian(n, 88)).cuda()
    q.put((rank, sharded_permanent(n, "glynn", gpu_partial_fn(dA, "glynn"), rank, world)))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.gpu
def test_two_processes_share_one_permanent_on_the_gpu():
    """The sharded path end to end with real processes: two ranks (gloo for the
    exchange of partials) each sum their half of the Gray range with the GPU range
    kernel, and perm_combine_partials on every rank gives the single launch's
    value.  (Both processes use this box's one GPU; their kernels never wait on
    each other.)"""
    import torch
    import paper_1606_05836_gb300 as pg
    n, world = 26, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gpu_rank_main, args=(r, world, port, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(world))
    single = complex(pg.glynn(torch.as_tensor(S.gaussian(n, 88)).cuda()).cpu().item())
    assert got[0] == got[1]
    assert abs(got[0] - single) <= 1e-12 * abs(single)
