"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here retypes the oracle's formulas: each check compares the oracle with
a value printed in arXiv 1606.05836 (the all-r "theory" columns of the Supp.
precision tables, the (1+i)^45 result of the 13,000-node run), a closed form
(n!, derangements, diagonal, rank-one, block-diagonal products), a brute-force
count on tiny inputs, an exact-integer evaluation, or an identity the permanent
satisfies (Laplace expansion, multilinearity, invariances, sum of Eq. (1)
probabilities = 1).  A dropped term, a wrong sign or index, or a transposed
operand in oracle.c fails at least one of them.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synthetic as S
from conftest import read_tsv


def qrel(a, b):
    """Relative difference of two oracle results carried as hi + lo."""
    return abs((a.hi - b.hi) + (a.lo - b.lo)) / abs(a.hi)


def closed_allr(n, r):
    return (r ** n) * math.factorial(n)


def exact_allr(n, r_re, r_im):
    """r^n * n! exactly with Fractions (r given as decimal strings)."""
    re, im = Fraction(r_re), Fraction(r_im)
    pr, pi = Fraction(1), Fraction(0)
    for _ in range(n):
        pr, pi = pr * re - pi * im, pr * im + pi * re
    f = math.factorial(n)
    return pr * f, pi * f


# --------------------------------------------------------------------------
# Paper-printed values
# --------------------------------------------------------------------------

def test_allr_closed_form_matches_paper_tables():
    """r^n n! reproduces every printed theory value (Supp. all-r tables)."""
    rows = read_tsv("allr_theory.tsv")
    assert len(rows) >= 40
    for row in rows:
        n = int(row["n"])
        er, ei = exact_allr(n, row["r_re"], row["r_im"])
        mag = math.hypot(float(er), float(ei))
        tol = 5.0 * 10.0 ** (-int(row["digits"])) * mag
        assert abs(float(er) - float(row["theory_re"])) <= tol, row
        assert abs(float(ei) - float(row["theory_im"])) <= tol, row


@pytest.mark.parametrize("n,r", [(17, 1.0), (17, 0.2), (17, 1 + 1j), (18, 10 + 10j), (18, 0.1)])
def test_oracle_allr_paper_sizes(n, r):
    """Ryser (S1) and Glynn (S2) oracles give r^n n! on the paper's all-r matrices."""
    A = S.all_r(n, r)
    want = closed_allr(n, r)
    for f in (oracle.ryser, oracle.glynn):
        got = f(A)
        assert got.rel_err(want) < 1e-14, (f.__name__, got, want)


def test_oracle_allr_exact_quad_agreement():
    """At n = 20, r = 0.2 the two quad evaluations agree far below FP64 rounding."""
    A = S.all_r(20, 0.2)
    g, r = oracle.glynn(A), oracle.ryser(A)
    want = closed_allr(20, 0.2)
    assert g.rel_err(want) < 1e-14 and r.rel_err(want) < 1e-14
    assert abs((g.hi - r.hi) + (g.lo - r.lo)) < 1e-22 * abs(want)


def test_worked_examples_fixed_values():
    ex = {row["name"]: row for row in read_tsv("worked_examples.tsv")}
    ones = S.all_r(12, 1.0)
    jmi = S.ones_minus_identity(12)
    assert oracle.ryser_int(np.ones((12, 12), dtype=np.int64)) == int(ex["ones"]["value_re"])
    assert oracle.ryser_int((np.ones((12, 12)) - np.eye(12)).astype(np.int64)) == int(
        ex["ones_minus_identity"]["value_re"])
    assert oracle.glynn(ones).hi == complex(479001600, 0)
    assert oracle.ryser(jmi).hi == complex(176214841, 0)
    assert oracle.glynn(jmi).hi == complex(176214841, 0)


def test_diag_1pi_n45_paper_run():
    """The paper's 13,000-node run: Per(diag(1+i)_45) = (1+i)^45.

    Every Glynn term of a diagonal matrix equals prod d_i (delta_i^2 = 1), so a
    partial sum over any index range is (count) x (1+i)^45; for Ryser only the
    full subset contributes, whose Gray index is the inverse Gray code of 2^45-1.
    """
    row = {r["name"]: r for r in read_tsv("worked_examples.tsv")}["diag_1pi"]
    n = int(row["n"])
    want = complex(float(row["value_re"]), float(row["value_im"]))
    assert want == (1 + 1j) ** 45
    A = S.diagonal([1 + 1j] * n)
    for kb, ke in [(0, 7), (123456789, 123456789 + 5), ((1 << 44) - 3, 1 << 44)]:
        got = oracle.glynn_range(A, kb, ke, gray=True, threads=1)
        assert got.rel_err((ke - kb) * want) < 1e-30
    full = (1 << n) - 1
    k_star, g = 0, full
    while g:  # inverse reflected Gray code: prefix XOR of the shifts
        k_star ^= g
        g >>= 1
    assert k_star ^ (k_star >> 1) == full
    got = oracle.ryser_range(A, k_star - 3, k_star + 3, gray=True, threads=1)
    assert got.rel_err((-1) ** n * want) < 1e-30  # the oracle's range sum excludes (-1)^n
    got0 = oracle.ryser_range(A, k_star + 1, k_star + 9, gray=True, threads=1)
    assert got0.hi == 0


# --------------------------------------------------------------------------
# Brute force and exact integers
# --------------------------------------------------------------------------

def matching_count(B):
    n = B.shape[0]
    return sum(all(B[i, p[i]] for i in range(n)) for p in itertools.permutations(range(n)))


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7])
def test_bruteforce_perfect_matchings(n):
    for seed in range(3):
        B = S.bernoulli01(n, seed + 10 * n)
        cnt = matching_count(B)
        assert oracle.ryser_int(B) == cnt
        Bc = B.astype(np.complex128)
        assert oracle.perm_def(Bc).hi == cnt
        assert oracle.ryser(Bc).hi == cnt
        assert oracle.glynn(Bc).hi == cnt


def test_ryser_int_against_quad_bernoulli():
    for n, seed in [(14, 1), (16, 2), (18, 3)]:
        B = S.bernoulli01(n, seed)
        exact = oracle.ryser_int(B)
        q = oracle.ryser(B.astype(np.complex128))
        g = oracle.glynn(B.astype(np.complex128))
        assert q.hi.real + q.lo.real == pytest.approx(exact, abs=0.5) and q.hi.imag == 0
        assert float(exact) == g.hi.real


def test_ryser_int_signed_and_large():
    # negative entries and a permanent beyond 2^64: all-(-3) 20x20 = 3^20 20!
    A = np.full((20, 20), -3, dtype=np.int64)
    assert oracle.ryser_int(A) == 3 ** 20 * math.factorial(20)
    A = np.full((21, 21), -3, dtype=np.int64)
    assert oracle.ryser_int(A) == -(3 ** 21) * math.factorial(21)


# --------------------------------------------------------------------------
# Closed forms
# --------------------------------------------------------------------------

def test_n0_n1():
    assert oracle.perm_def(np.zeros((0, 0))).hi == 1
    assert oracle.ryser(np.zeros((0, 0))).hi == 1
    assert oracle.glynn(np.zeros((0, 0))).hi == 1
    a = np.array([[0.3 - 2.5j]])
    for f in (oracle.perm_def, oracle.ryser, oracle.glynn):
        assert f(a).hi == 0.3 - 2.5j


def test_diagonal_product():
    d = S.circular_gaussian((10,), 5)
    want = np.prod(d)
    A = S.diagonal(d)
    for f in (oracle.perm_def, oracle.ryser, oracle.glynn):
        assert f(A).rel_err(want) < 1e-14
    P, Q = S.random_permutations(10, 3)  # a permuted diagonal is still prod d
    assert oracle.ryser(A[P][:, Q]).rel_err(want) < 1e-14


@pytest.mark.parametrize("n", [8, 15])
def test_rank_one(n):
    A, u, v = S.rank_one(n, 11)
    want = math.factorial(n) * np.prod(u) * np.prod(v)
    fs = [oracle.ryser, oracle.glynn] + ([oracle.perm_def] if n <= 10 else [])
    for f in fs:
        assert f(A).rel_err(want) < 1e-12


def test_block_diagonal_product():
    B1, B2 = S.gaussian(7, 21, 1.0), S.gaussian(8, 22, 1.0)
    A = np.zeros((15, 15), dtype=np.complex128)
    A[:7, :7], A[7:, 7:] = B1, B2
    P, Q = S.random_permutations(15, 4)
    A = A[P][:, Q]
    want = oracle.perm_def(B1).hi * oracle.ryser(B2).hi
    assert oracle.ryser(A).rel_err(want) < 1e-13
    assert oracle.glynn(A).rel_err(want) < 1e-13


# --------------------------------------------------------------------------
# Identities of the permanent
# --------------------------------------------------------------------------

def test_laplace_expansion_rows_and_columns():
    A = S.gaussian(9, 31, 1.0)
    M = oracle.minors(A)
    p = oracle.perm_def(A)
    for i in (0, 4, 8):
        assert p.rel_err(np.sum(A[i, :] * M[i, :])) < 1e-13
        assert p.rel_err(np.sum(A[:, i] * M[:, i])) < 1e-13
    # one minor directly: remove row 2, column 5
    sub = np.delete(np.delete(A, 2, axis=0), 5, axis=1)
    assert abs(M[2, 5] - oracle.perm_def(sub).hi) <= 1e-14 * abs(M[2, 5])


def test_multilinear_in_a_row():
    A = S.gaussian(12, 41, 1.0)
    x, y = S.circular_gaussian((12,), 42), S.circular_gaussian((12,), 43)
    al, be = 0.7 - 0.2j, -1.3 + 0.5j
    Ax, Ay, Az = A.copy(), A.copy(), A.copy()
    Ax[5], Ay[5], Az[5] = x, y, al * x + be * y
    lhs = oracle.glynn(Az).hi
    rhs = al * oracle.glynn(Ax).hi + be * oracle.ryser(Ay).hi
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), abs(rhs))


def test_invariances():
    A = S.gaussian(12, 51, 1.0)
    p = oracle.ryser(A)
    P, Q = S.random_permutations(12, 52)
    assert qrel(p, oracle.ryser(A.T)) < 1e-24
    assert qrel(p, oracle.glynn(A[P][:, Q])) < 1e-24
    d1, d2 = S.circular_gaussian((12,), 53), S.circular_gaussian((12,), 54)
    scaled = (d1[:, None] * A) * d2[None, :]
    want = np.prod(d1) * np.prod(d2) * p.hi
    assert oracle.glynn(scaled).rel_err(want) < 1e-13


# --------------------------------------------------------------------------
# Range partial sums (used to check sampled GPU partial sums at large n)
# --------------------------------------------------------------------------

def test_ranges_partition_and_scaling():
    n = 13
    A = S.gaussian(n, 61)
    full_g = oracle.glynn(A)
    cuts = [0, 1, 777, 2048, 3001, 1 << (n - 1)]
    parts = [oracle.glynn_range(A, a, b, gray=True) for a, b in zip(cuts[:-1], cuts[1:])]
    tot = sum(p.hi for p in parts) / 2 ** (n - 1)
    assert full_g.rel_err(tot) < 1e-14
    full_r = oracle.ryser(A)
    cuts = [1, 5, 4096, 5000, 1 << n]
    parts = [oracle.ryser_range(A, a, b, gray=True) for a, b in zip(cuts[:-1], cuts[1:])]
    tot = (-1) ** n * sum(p.hi for p in parts)
    assert full_r.rel_err(tot) < 1e-14


def test_gray_block_maps_to_binary_block():
    """Reflected Gray code maps the aligned block [a 2^b, (a+1) 2^b) onto [g(a) 2^b, (g(a)+1) 2^b)."""
    n, b = 12, 5
    A = S.gaussian(n, 71, 1.0)
    for a in (0, 3, 17, 40):
        ga = a ^ (a >> 1)
        gs = oracle.glynn_range(A, a << b, (a + 1) << b, gray=True)
        bs = oracle.glynn_range(A, ga << b, (ga + 1) << b, gray=False)
        assert qrel(gs, bs) < 1e-25
        rs = oracle.ryser_range(A, a << b, (a + 1) << b, gray=True)
        rb = oracle.ryser_range(A, ga << b, (ga + 1) << b, gray=False)
        assert abs(rs.hi - rb.hi) <= 1e-25 * max(abs(rs.hi), 1e-300)


def test_row_sum_convention_single_column():
    """A matrix whose only nonzero column is the first: each Glynn term is
    (prod delta) prod_i x_i because delta_1 = +1 (row sums, Eq. S2); with column
    sums every term would vanish.  Under the Gray mapping the sign alternates with
    the parity of the index (parity of popcount(k ^ k>>1) = k & 1)."""
    n = 10
    x = S.circular_gaussian((n,), 81)
    A = np.zeros((n, n), dtype=np.complex128)
    A[:, 0] = x
    px = np.prod(x)
    for kb, ke in [(0, 1), (0, 2), (3, 10), (5, 400)]:
        evens = sum(1 for k in range(kb, ke) if k % 2 == 0)
        odds = (ke - kb) - evens
        got = oracle.glynn_range(A, kb, ke, gray=True)
        want = (evens - odds) * px
        assert abs(got.hi - want) <= 1e-14 * abs(px) * (ke - kb)
    # Ryser: a term is nonzero iff column 0 is in S; full Per of this matrix is 0
    assert abs(oracle.ryser(A).hi) <= 1e-15 * abs(px)
    # with column 0 the only column, each subset containing it contributes (-1)^{|S|} prod x
    got = oracle.ryser_range(A, 1, 2, gray=False)  # S = {0}
    assert got.rel_err(-px) < 1e-14


# --------------------------------------------------------------------------
# Eq. (1) probabilities
# --------------------------------------------------------------------------

def all_patterns(m, n):
    for c in itertools.combinations_with_replacement(range(m), n):
        t = np.zeros(m, dtype=np.int32)
        for j in c:
            t[j] += 1
        yield t


def test_prob_hong_ou_mandel():
    U = np.array([[1, 1], [1, -1]], dtype=np.complex128) / math.sqrt(2)
    s = [1, 1]
    p11, _ = oracle.prob(U, s, [1, 1])
    p20, _ = oracle.prob(U, s, [2, 0])
    p02, _ = oracle.prob(U, s, [0, 2])
    assert abs(p11) < 1e-30
    assert p20 == pytest.approx(0.5, abs=1e-15) and p02 == pytest.approx(0.5, abs=1e-15)


def test_prob_single_photon():
    U = S.haar_unitary(4, 91)
    for i in range(4):
        for j in range(4):
            s = np.eye(4, dtype=np.int32)[i]
            t = np.eye(4, dtype=np.int32)[j]
            p, _ = oracle.prob(U, s, t)
            assert p == pytest.approx(abs(U[i, j]) ** 2, rel=1e-14)


@pytest.mark.parametrize("s", [[1, 1, 1, 0, 0], [2, 1, 0, 0, 0], [0, 0, 3, 0, 1]])
def test_prob_sums_to_one(s):
    U = S.haar_unitary(5, 92)
    n = sum(s)
    total = sum(oracle.prob(U, s, t)[0] for t in all_patterns(5, n))
    assert total == pytest.approx(1.0, abs=1e-13)


def test_prob_orientation_rows_are_inputs():
    """Row r of U_ST is input mode i, column c is output mode j: a non-symmetric U
    gives different probabilities for (s,t) and (t,s) unless transposed."""
    U = S.haar_unitary(4, 93)
    s, t = [1, 1, 0, 0], [0, 1, 0, 1]
    p, per = oracle.prob(U, s, t)
    sub = U[np.ix_([0, 1], [1, 3])]
    assert per.rel_err(sub[0, 0] * sub[1, 1] + sub[0, 1] * sub[1, 0]) < 1e-14
    p_t, _ = oracle.prob(U.T, t, s)
    assert p == pytest.approx(p_t, rel=1e-13)


# --------------------------------------------------------------------------
# Gray-order quad Glynn (the O(n 2^n) evaluation used for larger references)
# --------------------------------------------------------------------------

def test_glynn_gray_pins():
    # closed forms of the paper's all-r tables and a diagonal
    A = S.all_r(18, 0.2)
    assert oracle.glynn_gray(A).rel_err(closed_allr(18, 0.2)) < 1e-14
    d = S.circular_gaussian((13,), 6)
    assert oracle.glynn_gray(S.diagonal(d)).rel_err(np.prod(d)) < 1e-14
    # the derangement number of the worked example, exactly
    assert oracle.glynn_gray(S.ones_minus_identity(12)).hi == 176214841
    # agreement with the direct-sum evaluation far below FP64 rounding, any thread split
    B = S.gaussian(15, 7, 1.0)
    ref = oracle.glynn(B)
    for threads in (1, 3, 8):
        assert qrel(ref, oracle.glynn_gray(B, threads=threads)) < 1e-28
    # exact integer counts of 0/1 matrices
    C = S.bernoulli01(16, 9)
    assert oracle.glynn_gray(C.astype(np.complex128)).hi == oracle.ryser_int(C)


# --------------------------------------------------------------------------
# FP64 Gray-order sums with double-double accumulation (the oracle for n = 29-40)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 5, 12, 17, 20])
def test_f64dd_glynn_against_quad(n):
    """FP64 terms + double-double sum agree with the quad Gray-order evaluation to
    FP64 rounding (the products' relative error, ~n eps, is all that is left)."""
    A = S.gaussian(n, 50 + n)
    q = oracle.glynn_gray(A)
    assert qrel(q, oracle.glynn_f64dd(A)) < 1e-13
    # any thread split gives the same value to double-double rounding
    assert qrel(oracle.glynn_f64dd(A, threads=1), oracle.glynn_f64dd(A, threads=5)) < 1e-28


@pytest.mark.parametrize("n", [2, 5, 12, 17, 20])
def test_f64dd_ryser_against_quad(n):
    """Ryser in FP64 loses digits to cancellation (the paper's finding), but its
    Gray-order FP64 sum still tracks the quad value at these sizes."""
    A = S.gaussian(n, 60 + n)
    q = oracle.ryser_range(A, 0, 1 << n, gray=True)
    f = oracle.ryser_f64dd_range(A, 0, 1 << n)
    assert abs((f.hi - q.hi) + (f.lo - q.lo)) <= 1e-9 * abs(q.hi)


def test_f64dd_exact_on_small_integers():
    """0/1 and other small-integer matrices at n = 12: every row sum, product and
    partial sum is an integer below 2^53, so both FP64 sums are exact."""
    for seed in range(4):
        B = S.bernoulli01(12, seed)
        want = oracle.ryser_int(B)
        Bc = B.astype(np.complex128)
        g = oracle.glynn_f64dd(Bc)
        assert g.hi == want and g.lo == 0
        r = oracle.ryser_f64dd_range(Bc, 0, 1 << 12)
        assert r.hi == want and r.lo == 0  # (-1)^12 = 1
    ex = {r["name"]: r for r in read_tsv("worked_examples.tsv")}
    assert oracle.glynn_f64dd(S.all_r(12, 1.0)).hi == float(ex["ones"]["value_re"])
    assert oracle.glynn_f64dd(S.ones_minus_identity(12)).hi == float(ex["ones_minus_identity"]["value_re"])
    d = [1, 0]  # derangement numbers, D(n) = (n - 1)(D(n-1) + D(n-2))
    for k in range(2, 12):
        d.append((k - 1) * (d[-1] + d[-2]))
    r = oracle.ryser_f64dd_range(S.ones_minus_identity(11), 0, 1 << 11)
    assert -r.hi == d[11]  # (-1)^11 is outside the range sum


def test_f64dd_paper_diag_1pi_n45_range():
    """The paper's 45 x 45 diag(1+i) run: every Glynn term is (1+i)^45, exactly
    representable, so a range sum is the count times (1+i)^45 with no rounding;
    the range straddles the top of the 2^44 index space and crosses piece starts."""
    n = 45
    A = S.diagonal([1 + 1j] * n)
    w = (1 + 1j) ** 45
    for kb, ke in [(0, 1000), ((1 << 44) - 12345, 1 << 44), (777, 777), (63, 65)]:
        got = oracle.glynn_f64dd_range(A, kb, ke, threads=3)
        assert got.hi == (ke - kb) * w and got.lo == 0


def test_f64dd_range_additivity_across_pieces():
    """Cutting the range at arbitrary points (inside pieces, at piece starts, empty
    pieces) gives the same total to double-double rounding: a piece boundary
    restarts the row sums but changes no term."""
    A = S.gaussian(15, 77, 1.0)
    total = 1 << 14
    full = oracle.glynn_f64dd_range(A, 0, total, threads=2)
    cuts = [0, 1, 63, 64, 65, 1000, 4096, 4097, 9999, total]
    parts = [oracle.glynn_f64dd_range(A, a, b, threads=2) for a, b in zip(cuts[:-1], cuts[1:])]
    s = sum((p.hi for p in parts), 0j) + sum((p.lo for p in parts), 0j)
    scale = float(np.sum(np.abs([p.hi for p in parts])))
    assert abs(s - full.hi - full.lo) <= 1e-15 * scale
    # and the full Glynn range over 2^(n-1) matches the normalised permanent
    assert qrel(oracle.glynn(A), oracle.glynn_f64dd(A)) < 1e-13
    R = oracle.ryser_f64dd_range(A, 0, 1 << 15, threads=2)
    rparts = [oracle.ryser_f64dd_range(A, a, b, threads=2) for a, b in [(0, 5), (5, 6000), (6000, 1 << 15)]]
    rs = sum((p.hi + p.lo for p in rparts), 0j)
    assert abs(rs - (R.hi + R.lo)) <= 1e-15 * float(np.sum(np.abs([p.hi for p in rparts])))


def test_f64dd_closed_forms_n24():
    """Rank-one u v^T (n! prod u prod v), a permuted block-diagonal matrix (product of
    the blocks' quad permanents) and the paper's all-r values at n = 24."""
    A, u, v = S.rank_one(24, 601)
    want = math.factorial(24) * np.prod(u) * np.prod(v)
    assert abs(oracle.glynn_f64dd(A).hi - want) <= 1e-11 * abs(want)
    B1, B2 = S.gaussian(12, 911), S.gaussian(12, 912)
    Z = np.zeros((24, 24), dtype=np.complex128)
    Z[:12, :12], Z[12:, 12:] = B1, B2
    P, Q = S.random_permutations(24, 913)
    want = oracle.glynn(B1).hi * oracle.ryser(B2).hi
    assert oracle.glynn_f64dd(Z[P][:, Q]).rel_err(want) < 1e-13
    assert oracle.glynn_f64dd(S.all_r(24, 1 + 1j)).rel_err(closed_allr(24, 1 + 1j)) < 1e-13


def test_f64dd_allones_precision_within_paper_band():
    """FP64 BB/FG on all-ones (the paper's precision tables): the error against n!
    stays at or below the printed BB/FG errors (double-double accumulation only
    removes the summation part of the paper's error)."""
    paper = {int(r["n"]): float(r["bbfg_relerr"]) for r in read_tsv("precision_allones.tsv")}
    for n in (20, 24, 26):
        g = oracle.glynn_f64dd(S.all_r(n, 1.0))
        exact = math.factorial(n)
        err = abs(Fraction(g.hi.real) + Fraction(g.lo.real) - exact) / exact
        assert float(err) <= 10 * paper[n] + 1e-15, (n, float(err), paper[n])


def test_f64dd_ones_noise_against_stored_quad():
    """The heavy-cancellation input of the precision ladder (all-ones + 1e-3
    Gaussian) at n = 24 against its stored quad Gray-order value."""
    row = [r for r in read_tsv("ladder_refs.tsv") if r["kind"] == "ones_noise" and int(r["n"]) == 24][0]
    A = S.ones_plus_noise(24, 0)
    f = oracle.glynn_f64dd(A)
    hi = complex(float(row["re_hi"]), float(row["im_hi"]))
    lo = complex(float(row["re_lo"]), float(row["im_lo"]))
    assert abs((f.hi - hi) + (f.lo - lo)) <= 1e-11 * abs(hi)


def _large_ref(kind, n, seed):
    rows = [r for r in read_tsv("large_refs.tsv") if r["kind"] == kind and int(r["n"]) == n and int(r["seed"]) == seed]
    assert rows, "no stored reference for %s n=%d seed=%d (tests/golden/make_large_refs.py)" % (kind, n, seed)
    r = rows[0]
    return r["sha"], complex(float(r["re_hi"]) + float(r["re_lo"]), float(r["im_hi"]) + float(r["im_lo"]))


def test_f64dd_against_quad_at_n32_stored():
    """At n = 32 the quad oracle takes ~50 min per matrix, so its values of the
    benchmark's Gaussian inputs are stored (make_sweep_refs.py); the FP64 /
    double-double evaluations of the same inputs (make_large_refs.py) agree with
    them far inside the 1e-10 bar."""
    quad = {int(r["seed"]): r for r in read_tsv("sweep_refs.tsv") if r["oracle"] == "glynn_gray" and r["n"] == "32"}
    assert sorted(quad) == [0, 1, 2]
    for seed, q in quad.items():
        sha, fv = _large_ref("gaussian", 32, seed)
        assert q["sha"] == sha
        qv = complex(float(q["re_hi"]) + float(q["re_lo"]), float(q["im_hi"]) + float(q["im_lo"]))
        assert abs(qv - fv) <= 1e-12 * abs(qv), seed


def test_f64dd_block_diagonal_n36_stored():
    """n = 36: the stored FP64 / double-double value of a permuted block-diagonal
    matrix equals the product of its two n = 18 block permanents from the quad
    oracle (Per(diag(B1, B2)) = Per(B1) Per(B2), invariant under row and column
    permutations)."""
    import importlib.util
    import os
    from conftest import GOLDEN
    spec = importlib.util.spec_from_file_location("make_large_refs", os.path.join(GOLDEN, "make_large_refs.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    sha, got = _large_ref("block_diag", 36, 36036)
    assert mod.digest(mod.make_input("block_diag", 36, 36036)) == sha
    B1, B2 = mod.block_diag_blocks(36, 36036)
    want = oracle.glynn_gray(B1).hi * oracle.glynn_gray(B2).hi
    assert abs(got - want) <= 1e-12 * abs(want)


@pytest.mark.slow
def test_f64dd_n32_recomputed_against_stored_quad():
    """One full n = 32 evaluation (2^31 FP64 terms, ~40 s on 8 cores) of the
    benchmark's seed-0 input against its stored quad value."""
    import hashlib
    row = [r for r in read_tsv("sweep_refs.tsv") if r["oracle"] == "glynn_gray" and r["n"] == "32" and r["seed"] == "0"]
    A = S.gaussian(32, 0)
    assert hashlib.sha256(np.ascontiguousarray(A).tobytes()).hexdigest()[:16] == row[0]["sha"]
    f = oracle.glynn_f64dd(A)
    q = row[0]
    qv = complex(float(q["re_hi"]) + float(q["re_lo"]), float(q["im_hi"]) + float(q["im_lo"]))
    assert abs((f.hi + f.lo) - qv) <= 1e-12 * abs(qv)
