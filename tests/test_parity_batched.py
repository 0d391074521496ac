"""GPU parity of the batched form (perm_batched: one persistent size-bucketed
launch, per-item reduce and the Eq. (1) probability epilogue) against the oracle,
through the C ABI, plus its CUDA-graph replay and its device-side guards."""
import math

import numpy as np
import pytest

import oracle
import synthetic as S
from gpu_util import REL_TOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    import paper_1606_05836_gb300 as pg
    from paper_1606_05836_gb300 import build
    build.build()
    pg.library()
    return pg


def _mixed(count, n_lo, n_hi, seed):
    g = np.random.default_rng(seed)
    return [S.gaussian(int(n), seed * 1000 + i, 1.0) for i, n in enumerate(g.integers(n_lo, n_hi + 1, size=count))]


@pytest.mark.parametrize("method", ["glynn", "ryser"])
def test_batched_small_mixed_all_rungs(pg, method):
    mats = _mixed(48, 1, 14, 1)
    want = [oracle.perm_def(A) if A.shape[0] <= 8 else oracle.ryser(A) for A in mats]
    tol = {"fp64": REL_TOL, "fp64_dd": REL_TOL, "fp32p_dd": 1e-4 if method == "glynn" else 1e-2, "fp64_df": REL_TOL,
           "fp32x2": REL_TOL}
    rungs = ("fp64", "fp64_dd", "fp32p_dd", "fp64_df") + (("fp32x2",) if method == "glynn" else ())
    for prec in rungs:
        per, _ = pg.batched(mats, method=method, prec=prec)
        got = per.cpu().numpy()
        for i, w in enumerate(want):
            assert w.rel_err(got[i]) < tol[prec], (prec, i, mats[i].shape[0], got[i], w.hi)


def test_batched_fp32x2_larger_items_and_ryser_rejected(pg):
    """R4 on items up to n = 22 with several units per item, against the oracle; Ryser refuses R4."""
    mats = _mixed(12, 16, 22, 5)
    per, _ = pg.batched(mats, method="glynn", prec="fp32x2", unit_log2=6)
    got = per.cpu().numpy()
    for i, A in enumerate(mats):
        assert oracle.ryser(A).rel_err(got[i]) < REL_TOL, (i, A.shape[0])
    with pytest.raises(Exception):
        pg.batched(mats[:2], method="ryser", prec="fp32x2")


def test_batched_matches_single_permanent_path(pg):
    mats = _mixed(40, 14, 22, 2)
    import torch
    per, _ = pg.batched(mats, method="glynn", unit_log2=5)  # many units per item
    got = per.cpu().numpy()
    for i, A in enumerate(mats):
        single = complex(pg.glynn(torch.as_tensor(A).cuda()).cpu().item())
        assert abs(got[i] - single) <= REL_TOL * abs(single)


def test_batched_probabilities_with_collisions(pg):
    """Eq. (1): output patterns of one Haar unitary, one photon per input mode,
    20 % of the outputs with repeated columns; prob = |Per(U_ST)|^2 / prod t_j!."""
    U = S.haar_unitary(30, 7)
    mats, ns, rows, cols, collide = S.batch_patterns(U, 60, 2, 9, 8)
    assert collide.any() and not collide.all()
    scale, s_vecs, t_vecs = [], [], []
    for r, c in zip(rows, cols):
        s = np.zeros(30, dtype=np.int32)
        t = np.zeros(30, dtype=np.int32)
        s[r] = 1
        for j in c:
            t[j] += 1
        s_vecs.append(s)
        t_vecs.append(t)
        scale.append(1.0 / float(np.prod([math.factorial(int(x)) for x in t])))
    per, prob = pg.batched(mats, method="glynn", scale=scale)
    per, prob = per.cpu().numpy(), prob.cpu().numpy()
    for i in range(len(mats)):
        p_want, per_want = oracle.prob(U, s_vecs[i], t_vecs[i])
        assert per_want.rel_err(per[i]) < REL_TOL
        assert abs(prob[i] - p_want) <= 1e-9 * p_want + 1e-300


def test_batched_graph_replay_and_autotune(pg, tmp_path, monkeypatch):
    from paper_1606_05836_gb300 import batch as B
    monkeypatch.setattr(B, "TUNE_CACHE", str(tmp_path / "tune.json"))
    mats = _mixed(64, 8, 18, 3)
    bp = B.BatchedPermanents(mats, method="glynn")
    eager = bp.run()[0].clone()
    best = bp.autotune(candidates=[(7, 64), (9, 128)], reps=1)
    assert best["unit_log2"] in (7, 9)
    bp.capture()
    for _ in range(2):
        per, _ = bp.replay()
        assert np.allclose(per.cpu().numpy(), eager.cpu().numpy(), rtol=1e-12, atol=0)
    again = B.BatchedPermanents(mats, method="glynn")
    assert again.autotune(candidates=[(7, 64)], reps=1) == best  # served from the cache


def test_batched_device_guards_give_nan_not_a_fault(pg):
    """Sizes on the device that disagree with the host sizes: the planner
    refuses the batch and the outputs are NaN (no out-of-bounds access)."""
    import ctypes
    import torch
    from paper_1606_05836_gb300 import batch as B
    mats = [S.gaussian(5, 11, 1.0), S.gaussian(5, 12, 1.0)]
    bp = B.BatchedPermanents(mats)
    bp.ns.copy_(torch.tensor([5, 33], dtype=torch.int32))   # n beyond the batched maximum
    per, prob = bp.run()
    assert torch.isnan(per.real).all() and torch.isnan(prob).all()
    bp = B.BatchedPermanents(mats)
    bp.ns.copy_(torch.tensor([5, 20], dtype=torch.int32))   # more work than the workspace was sized for
    bp.packed = torch.zeros(500, dtype=torch.complex128, device="cuda")
    per, _ = bp.run()
    assert torch.isnan(per.real).all()


def test_batched_empty(pg):
    per, prob = pg.batched([])
    assert per.numel() == 0


@pytest.mark.slow
def test_config4_batch_full_size_against_the_oracle(pg):
    """The benchmark's batch itself: 4096 output patterns of one Haar 1000 x 1000
    unitary (n uniform in 8..24, 20 % with repeated output modes), in its launch
    configuration (one CUDA graph replay of the persistent walk, default shape).
    Every item of n >= 23 (the ones that dominate its time) and every collision
    item is compared with the oracle (FP64 Gray-order Glynn with double-double
    accumulation, pinned against the quad oracle), element by element: Per within
    1e-10 and the Eq. (1) probability |Per|^2 / prod t_j! within 2e-10 (twice Per's
    relative error bounds |Per|^2's)."""
    from paper_1606_05836_gb300 import batch as B
    U = S.haar_unitary(1000, 0)
    mats, ns, _, cols, collide = S.batch_patterns(U, 4096, 8, 24, 1)
    scale = [1.0 / float(np.prod([math.factorial(int(x)) for x in np.bincount(c)])) for c in cols]
    bp = B.BatchedPermanents(mats, method="glynn", scale=scale)
    bp.capture()
    per, prob = bp.replay()
    per, prob = per.cpu().numpy(), prob.cpu().numpy()
    check = [i for i in range(len(mats)) if ns[i] >= 23 or collide[i]]
    assert sum(1 for i in check if ns[i] >= 23) > 300 and int(collide.sum()) > 700
    worst = 0.0
    for i in check:
        want = oracle.glynn_f64dd(mats[i])
        e = want.rel_err(per[i])
        worst = max(worst, e)
        assert e < REL_TOL, (i, int(ns[i]), bool(collide[i]), per[i], want.hi)
        p_want = abs(want.hi + want.lo) ** 2 * scale[i]
        assert abs(prob[i] - p_want) <= 2 * REL_TOL * p_want, (i, prob[i], p_want)
    print("\nconfig-4 batch: %d items checked, max relative error of Per %.2e" % (len(check), worst))


def _repeated(n, mult, seed):
    """n x n matrix whose columns are g Gaussian columns repeated mult[c] times,
    in a shuffled column order."""
    B = S.circular_gaussian((n, len(mult)), seed, 1.0)
    E = np.repeat(B, mult, axis=1)
    perm = np.random.default_rng(seed + 1).permutation(n)
    return np.ascontiguousarray(E[:, perm])


@pytest.mark.parametrize("prec", ["fp64", "fp64_dd", "fp64_df", "fp32x2"])
def test_batched_repeated_columns_every_structure(pg, prec):
    """Items with repeated columns (a pair, a triple, several pairs, no singleton
    at all, every column equal) walk the multiplicity expansion inside the
    batch (R0-R2; R3 and R4 walk the expanded matrix); mixed with plain items, each
    against the oracle on the expanded matrix."""
    cases = [(6, [2, 1, 1, 1, 1]), (9, [3, 1, 1, 1, 1, 1, 1]), (12, [2, 2, 2] + [1] * 6), (8, [2, 2, 2, 2]),
             (7, [7]), (10, [4, 3, 1, 1, 1]), (13, [2] + [1] * 11), (5, [1, 1, 1, 1, 1]), (14, [3, 3, 2] + [1] * 6),
             (2, [2]), (1, [1]), (11, [5, 6])]
    mats = [_repeated(n, m, 40 + i) for i, (n, m) in enumerate(cases)]
    mats += _mixed(6, 3, 12, 9)
    want = [oracle.perm_def(A) if A.shape[0] <= 8 else oracle.ryser(A) for A in mats]
    per, _ = pg.batched(mats, method="glynn", prec=prec)
    got = per.cpu().numpy()
    tol = REL_TOL
    for i, w in enumerate(want):
        assert w.rel_err(got[i]) < tol, (prec, i, mats[i].shape[0], got[i], w.hi)
    # Ryser does not use the expansion: same values from its plain walk
    if prec == "fp64":
        per_r, _ = pg.batched(mats, method="ryser")
        got_r = per_r.cpu().numpy()
        for i, w in enumerate(want):
            assert w.rel_err(got_r[i]) < 1e-9, (i, got_r[i], w.hi)


def test_batched_repeated_columns_many_units(pg):
    """Items of n = 18-22 with repeated columns cut into many small work units
    (units cross class boundaries and classes span several units)."""
    cases = [(18, [2] + [1] * 16), (20, [3, 2, 2] + [1] * 13), (22, [2, 2] + [1] * 18), (19, [4, 4, 4, 4, 3])]
    mats = [_repeated(n, m, 70 + i) for i, (n, m) in enumerate(cases)]
    for unit_log2 in (2, 5, 11):
        per, _ = pg.batched(mats, method="glynn", unit_log2=unit_log2)
        got = per.cpu().numpy()
        for i, A in enumerate(mats):
            assert oracle.glynn_f64dd(A).rel_err(got[i]) < REL_TOL, (unit_log2, i)


def test_batched_largest_items_against_the_oracle(pg):
    """Items up to the batched maximum's neighbourhood (n = 25-29, plus a repeated-
    column item at n = 30) in one launch, each against the FP64 / double-double
    oracle."""
    mats = [S.gaussian(n, 500 + n) for n in (25, 27, 29)] + [_repeated(30, [2, 2] + [1] * 26, 530)]
    per, _ = pg.batched(mats, method="glynn")
    got = per.cpu().numpy()
    for i, A in enumerate(mats):
        assert oracle.glynn_f64dd(A).rel_err(got[i]) < REL_TOL, (i, A.shape[0])
