"""Pins of the boson-sampling oracle (oracle/sampler.py) against what the
mathematics fixes: closed-form minors, the permutation-sum definition, the exact
output distribution Eq. (1) of arXiv 1606.05836, Hong-Ou-Mandel bunching and
deterministic permutation unitaries.  A wrong column order, a dropped factor in
the step weights or a wrong choice rule fails at least one of them."""
import math

import numpy as np
import pytest

import oracle
import synthetic as S
from oracle import sampler as OS


def all_patterns(m, n):
    out = []

    def rec(prefix, left):
        if len(prefix) == m - 1:
            out.append(tuple(prefix + [left]))
            return
        for x in range(left + 1):
            rec(prefix + [x], left - x)

    rec([], n)
    return out


@pytest.mark.parametrize("k", [1, 2, 5, 9, 12])
def test_row_minors_rank_one_closed_form(k):
    """M = u v^T ((k-1) x k): Per(M without column j) = (k-1)! prod u prod_{l != j} v_l."""
    g = np.random.default_rng(1000 + k)
    u = g.normal(size=k - 1) + 1j * g.normal(size=k - 1)
    v = g.normal(size=k) + 1j * g.normal(size=k)
    M = np.outer(u, v)
    got = OS.row_minors(M)
    for j in range(k):
        want = math.factorial(k - 1) * np.prod(u) * np.prod(np.delete(v, j))
        assert abs(got[j] - want) <= 1e-12 * abs(want), (k, j)


@pytest.mark.parametrize("k", [2, 4, 7])
def test_row_minors_laplace_against_definition(k):
    """sum_j x_j m_j = Per([M; x]) by the permutation sum (independent of the minors)."""
    g = np.random.default_rng(77 + k)
    M = g.normal(size=(k - 1, k)) + 1j * g.normal(size=(k - 1, k))
    x = g.normal(size=k) + 1j * g.normal(size=k)
    lhs = np.dot(x, OS.row_minors(M))
    full = np.vstack([M, x[None, :]])
    rhs = oracle.perm_def(full)
    assert abs(lhs - rhs.hi) <= 1e-12 * abs(rhs.hi)


def test_row_minors_rejects_wrong_shape():
    with pytest.raises(ValueError):
        OS.row_minors(np.zeros((3, 3), dtype=complex))


def test_choose_rule_on_hand_cases():
    w = [0.0, 1.0, 0.0, 3.0]
    assert OS.choose(w, 0.0) == 1          # zero-weight modes are never drawn
    assert OS.choose(w, 0.2499) == 1
    assert OS.choose(w, 0.25) == 3         # running sum must exceed u W strictly
    assert OS.choose(w, 0.999999) == 3
    assert OS.choose([0.0, 0.0], 0.5) == -1
    assert OS.choose([2.0, 0.0], 1.0 - 2.0 ** -53) == 0


@pytest.mark.parametrize("m,n,seed", [(2, 2, 1), (4, 2, 2), (5, 3, 3), (4, 3, 4)])
def test_chain_distribution_equals_eq1(m, n, seed):
    """The chain over (alpha, r_1..r_n) reproduces Eq. (1) for every output pattern."""
    U = S.haar_unitary(m, seed)
    inputs = list(range(n))
    dist = OS.chain_distribution(U, inputs)
    s = [1] * n + [0] * (m - n)
    total = 0.0
    for t in all_patterns(m, n):
        want, _ = oracle.prob(U, s, list(t))
        got = dist.get(t, 0.0)
        assert abs(got - want) <= 1e-12, (t, got, want)
        total += got
    assert abs(total - 1.0) <= 1e-12


def test_chain_distribution_inputs_not_first_modes():
    U = S.haar_unitary(5, 9)
    inputs = [4, 1, 2]
    dist = OS.chain_distribution(U, inputs)
    s = [0, 1, 1, 0, 1]
    for t in all_patterns(5, 3):
        want, _ = oracle.prob(U, s, list(t))
        assert abs(dist.get(t, 0.0) - want) <= 1e-12


def test_hong_ou_mandel_bunching():
    """50:50 beam splitter, one photon per input: (1,1) never occurs, (2,0) and (0,2) at 1/2."""
    U = np.array([[1, 1], [1, -1]], dtype=complex) / math.sqrt(2)
    dist = OS.chain_distribution(U, [0, 1])
    assert dist.get((1, 1), 0.0) <= 1e-15
    assert abs(dist[(2, 0)] - 0.5) <= 1e-15 and abs(dist[(0, 2)] - 0.5) <= 1e-15
    for seed in range(20):
        g = np.random.default_rng(seed)
        r, _ = OS.sample(U, [0, 1], g.permutation(2), g.random(2))
        assert r[0] == r[1]


def test_permutation_unitary_is_deterministic():
    """U a permutation matrix: the photon in input mode i leaves in mode pi(i), drawn in alpha order."""
    m, n = 7, 4
    pi = [3, 0, 6, 1, 5, 2, 4]
    U = np.zeros((m, m), dtype=complex)
    for i in range(m):
        U[i, pi[i]] = 1.0  # Eq. (1) convention: row = input mode, column = output mode
    inputs = [2, 5, 0, 6]
    g = np.random.default_rng(5)
    for _ in range(5):
        alpha = g.permutation(n)
        r, _ = OS.sample(U, inputs, alpha, g.random(n))
        assert r == [pi[inputs[a]] for a in alpha]


def test_monte_carlo_histogram_matches_eq1():
    """Draws with seeded (alpha, u) follow Eq. (1): chi-square over the patterns of m=4, n=2."""
    m, n = 4, 2
    U = S.haar_unitary(m, 21)
    g = np.random.default_rng(123)
    counts = {}
    N = 3000
    for _ in range(N):
        r, _ = OS.sample(U, [0, 1], g.permutation(n), g.random(n))
        t = OS.pattern(r, m)
        counts[t] = counts.get(t, 0) + 1
    chi2, dof = 0.0, 0
    for t in all_patterns(m, n):
        p, _ = oracle.prob(U, [1, 1, 0, 0], list(t))
        e = N * p
        if e >= 5:
            chi2 += (counts.get(t, 0) - e) ** 2 / e
            dof += 1
    # 9 patterns, 8 degrees of freedom at most: P(chi2 > 35) < 3e-5
    assert dof >= 5 and chi2 < 35.0, (chi2, dof)


def test_sample_rejects_bad_draws():
    U = S.haar_unitary(4, 1)
    with pytest.raises(ValueError):
        OS.sample(U, [0, 1], [0, 0], [0.1, 0.2])
    with pytest.raises(ValueError):
        OS.sample(U, [1, 1], [0, 1], [0.1, 0.2])
