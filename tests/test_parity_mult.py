"""GPU parity of the repeated-column (photon-collision) permanent, perm_glynn_mult,
and of prob_sample on colliding patterns, through the C ABI, against the oracle's
permanent of the expanded matrix."""
import math

import numpy as np
import pytest

import oracle
import synthetic as S
from gpu_util import REL_TOL, to_dev, val

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    import paper_1606_05836_gb300 as pg
    from paper_1606_05836_gb300 import build
    build.build()
    pg.library()
    return pg


def expand(B, mult):
    return np.ascontiguousarray(np.repeat(B, mult, axis=1))


@pytest.mark.parametrize("mult", [
    [2, 1, 1, 1],            # one pair, singletons present (delta = +1 on a singleton)
    [1, 3, 2, 1, 1],
    [2, 2, 2],               # no singleton: delta = +1 taken in a repeated group
    [5],                     # all columns equal: Per = n! prod_i b_i
    [1, 1, 1, 1, 1, 1, 1],   # no repeats: plain Glynn through the base-vector walk
    [4, 1, 3, 1, 2],
    [3, 3, 3, 1],
])
def test_mult_vs_oracle(pg, mult):
    n, g = sum(mult), len(mult)
    B = S.circular_gaussian((n, g), 1000 + n * 7 + g, 1.0)
    A = expand(B, mult)
    want = oracle.perm_def(A) if n <= 10 else oracle.ryser(A)
    got = val(pg.glynn_mult(to_dev(B), mult))
    assert want.rel_err(got) < REL_TOL, (mult, got, want.hi)
    if mult == [5]:
        assert abs(got - math.factorial(5) * np.prod(B[:, 0])) <= 1e-12 * abs(got)


def test_mult_matches_plain_path_n24(pg):
    mult = [2, 1, 1, 3, 1, 1, 1, 2] + [1] * 12
    n, g = sum(mult), len(mult)
    assert n == 24
    B = S.circular_gaussian((n, g), 2424, 1.0 / n)
    plain = val(pg.glynn(to_dev(expand(B, mult))))
    got = val(pg.glynn_mult(to_dev(B), mult))
    assert abs(got - plain) <= REL_TOL * abs(plain)


def test_mult_many_classes(pg):
    """13 pairs and no singleton: 2 x 3^12 classes of one term each."""
    mult = [2] * 13
    n, g = 26, 13
    B = S.circular_gaussian((n, g), 2626, 1.0 / n)
    plain = val(pg.glynn(to_dev(expand(B, mult))))
    got = val(pg.glynn_mult(to_dev(B), mult))
    assert abs(got - plain) <= REL_TOL * abs(plain)


def test_mult_rejects_bad_multiplicities(pg):
    from paper_1606_05836_gb300 import PermError
    B = to_dev(S.circular_gaussian((4, 2), 5, 1.0))
    with pytest.raises((ValueError, PermError)):
        pg.glynn_mult(B, [2, 1])  # sums to 3, not 4
    with pytest.raises((ValueError, PermError)):
        pg.glynn_mult(B, [4, 0])


def test_prob_bunching_and_collisions(pg):
    """All n photons in one output mode: Per(U_ST) = n! prod_r U[s_r][j]; mixed
    input and output collisions against the oracle (both orientations)."""
    U = S.haar_unitary(8, 41)
    dU = to_dev(U)
    s = [1, 1, 1, 1, 0, 0, 0, 0]
    t = [0, 0, 0, 0, 0, 4, 0, 0]
    p, per = pg.prob(dU, s, t)
    want_per = math.factorial(4) * np.prod([U[i, 5] for i in range(4)])
    assert abs(per - want_per) <= 1e-12 * abs(want_per)
    assert abs(p - abs(want_per) ** 2 / math.factorial(4)) <= 1e-12 * p
    for s, t in [([2, 1, 0, 1, 0, 0, 0, 0], [1, 0, 0, 3, 0, 0, 0, 0]),
                 ([3, 0, 0, 0, 2, 0, 0, 0], [1, 1, 1, 1, 1, 0, 0, 0]),
                 ([1, 1, 1, 1, 1, 1, 0, 0], [2, 0, 2, 0, 2, 0, 0, 0])]:
        p, per = pg.prob(dU, s, t)
        pw, perw = oracle.prob(U, s, t)
        assert perw.rel_err(per) < REL_TOL
        assert abs(p - pw) <= 1e-9 * pw


@pytest.mark.parametrize("mult", [[2, 2, 2] + [1] * 14, [3, 2, 2, 1] + [1] * 12])
@pytest.mark.parametrize("opts", [{}, {"grid": 2}, {"grid": 997}, {"grid": 5, "chunk_log2": 3}])
def test_mult_warp_aligned_split_vs_oracle(pg, mult, opts):
    """>= 5 free columns: the warp-aligned class layout (every warp's lanes in one
    class at a time), with a ragged warp split and short chunks, against the oracle."""
    n, g = sum(mult), len(mult)
    B = S.circular_gaussian((n, g), 3000 + g, 1.0 / n)
    want = oracle.ryser(expand(B, mult))
    got = val(pg.glynn_mult(to_dev(B), mult, **opts))
    assert want.rel_err(got) < REL_TOL, (mult, opts, got, want.hi)
