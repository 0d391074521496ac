"""GPU parity of prob_sample (Eq. (1)) through the C ABI against the oracle, and
the probability identities the paper's Eq. (1) must satisfy."""
import itertools
import math

import numpy as np
import pytest

import oracle
import synthetic as S
from gpu_util import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    import paper_1606_05836_gb300 as pg
    from paper_1606_05836_gb300 import build
    build.build()
    pg.library()
    return pg


def test_prob_vs_oracle_with_collisions(pg):
    U = S.haar_unitary(12, 31)
    dU = to_dev(U)
    g = np.random.default_rng(5)
    for _ in range(20):
        n = int(g.integers(1, 9))
        s = np.bincount(g.choice(12, size=n, replace=True), minlength=12)
        t = np.bincount(g.choice(12, size=n, replace=True), minlength=12)
        p, per = pg.prob(dU, s, t)
        pw, perw = oracle.prob(U, s, t)
        assert perw.rel_err(per) < 1e-10
        assert abs(p - pw) <= 1e-9 * pw + 1e-300


def test_prob_sums_to_one_over_outputs(pg):
    U = S.haar_unitary(6, 32)
    dU = to_dev(U)
    s = [1, 1, 0, 1, 0, 0]
    total = 0.0
    for c in itertools.combinations_with_replacement(range(6), 3):
        t = np.bincount(c, minlength=6)
        total += pg.prob(dU, s, t)[0]
    assert abs(total - 1.0) < 1e-12


def test_prob_hong_ou_mandel_and_zero_photons(pg):
    U = np.array([[1, 1], [1, -1]], dtype=np.complex128) / math.sqrt(2)
    dU = to_dev(U)
    assert abs(pg.prob(dU, [1, 1], [1, 1])[0]) < 1e-30
    assert abs(pg.prob(dU, [1, 1], [2, 0])[0] - 0.5) < 1e-15
    p, per = pg.prob(dU, [0, 0], [0, 0])
    assert p == 1.0 and per == 1.0


def test_prob_rejects_bad_patterns(pg):
    from paper_1606_05836_gb300 import PermError
    dU = to_dev(S.haar_unitary(4, 33))
    with pytest.raises(PermError):
        pg.prob(dU, [1, 0, 0, 0], [0, 0, 1, 1])   # photon numbers differ
    with pytest.raises(PermError):
        pg.prob(dU, [-1, 1, 0, 0], [0, 0, 0, 0])
