"""GPU parity of the row minors (perm_row_minors) and of the boson-sampling
draws (boson_sample), through the C ABI, against oracle/sampler.py."""
import math

import numpy as np
import pytest

import oracle
import synthetic as S
from gpu_util import REL_TOL
from oracle import sampler as OS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    import paper_1606_05836_gb300 as pg
    from paper_1606_05836_gb300 import build
    build.build()
    pg.library()
    return pg


def dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x)).cuda()


def close_vec(got, want, tol=REL_TOL):
    scale = np.max(np.abs(want))
    for j in range(len(want)):
        ref = max(abs(want[j]), 1e-3 * scale)
        assert abs(got[j] - want[j]) <= tol * ref, (j, got[j], want[j])


# --------------------------------------------------------------------------
# row minors
# --------------------------------------------------------------------------

@pytest.mark.parametrize("k", [2, 3, 5, 9, 16, 21])
@pytest.mark.parametrize("opts", [{}, {"grid": 3, "chunk_log2": 3}, {"prec": "fp64_df"}, {"prec": "fp32x2"},
                                  {"prec": "fp32x2", "grid": 5, "chunk_log2": 4}])
def test_row_minors_vs_oracle(pg, k, opts):
    M = S.circular_gaussian((k - 1, k), 4000 + k, 1.0 / k)
    got = pg.row_minors(dev(M), **opts).cpu().numpy()
    close_vec(got, OS.row_minors(M))


def test_row_minors_k1_and_zero_row(pg):
    import torch
    got = pg.row_minors(torch.zeros(0, 1, dtype=torch.complex128, device="cuda")).cpu().numpy()
    assert got.tolist() == [1.0]
    M = S.circular_gaussian((9, 10), 5, 0.1)
    M[4, :] = 0.0
    assert np.all(pg.row_minors(dev(M)).cpu().numpy() == 0.0)


def test_row_minors_batch(pg):
    k, B = 12, 5
    Ms = np.stack([S.circular_gaussian((k - 1, k), 60 + b, 1.0 / k) for b in range(B)])
    got = pg.row_minors(dev(Ms)).cpu().numpy()
    for b in range(B):
        close_vec(got[b], OS.row_minors(Ms[b]))


@pytest.mark.parametrize("k", [24, 32])
@pytest.mark.parametrize("prec", ["fp64", "fp64_df", "fp32x2"])
def test_row_minors_rank_one_full_size(pg, k, prec):
    """M = u v^T: m_j = (k-1)! prod u prod_{l != j} v_l (closed form at the largest size)."""
    g = np.random.default_rng(k)
    u = (g.normal(size=k - 1) + 1j * g.normal(size=k - 1)) / k
    v = (g.normal(size=k) + 1j * g.normal(size=k)) / 2
    got = pg.row_minors(dev(np.outer(u, v)), prec=prec).cpu().numpy()
    pu = np.prod(u) * math.factorial(k - 1)
    want = np.array([pu * np.prod(np.delete(v, j)) for j in range(k)])
    # all k minors are sums over the same 2^(k-1) terms, so their rounding errors
    # have one common size: the bound is normwise (a minor with a large |v_j|
    # excluded is small and carries the same absolute error)
    scale = np.max(np.abs(want))
    tol = 1e-9 if prec == "fp32x2" else REL_TOL  # R4's stated bound on extreme cancellation
    for j in range(k):
        assert abs(got[j] - want[j]) <= tol * scale, (j, got[j], want[j])


# --------------------------------------------------------------------------
# draws
# --------------------------------------------------------------------------

def draws(seed, nsamples, n):
    return S.sampler_draws(n, nsamples, seed)


def check_against_oracle(U, inputs, alpha, u, got):
    """Equal draws, or a first difference at a near-tie of the oracle's running sums."""
    near_ties = 0
    for s in range(alpha.shape[0]):
        want, margins = OS.sample(U, inputs, alpha[s], u[s])
        if list(got[s]) == want:
            continue
        k = next(i for i in range(len(want)) if got[s][i] != want[i])
        assert margins[k] < 1e-9, (s, k, list(got[s]), want, margins[k])
        near_ties += 1
    assert near_ties <= 1


@pytest.mark.parametrize("m,n,ns", [(8, 4, 40), (30, 8, 16), (64, 12, 6), (120, 16, 3), (1000, 16, 2)])
@pytest.mark.parametrize("prec", ["fp64", "fp64_df", "fp32x2"])
def test_draws_match_oracle(pg, m, n, ns, prec):
    U = S.haar_unitary(m, 100 + m)
    g = np.random.default_rng(m)
    inputs = sorted(g.choice(m, size=n, replace=False).tolist())
    alpha, u = draws(7 * m + n, ns, n)
    got = pg.boson_sample(dev(U), inputs, dev(alpha), dev(u), prec=prec).cpu().numpy()
    check_against_oracle(U, inputs, alpha, u, got)


def test_draw_histogram_matches_eq1(pg):
    """20,000 draws of 3 photons in 5 modes: chi-square against Eq. (1) (oracle.prob)."""
    m, n, N = 5, 3, 20000
    U = S.haar_unitary(m, 33)
    alpha, u = draws(99, N, n)
    got = pg.boson_sample(dev(U), [0, 1, 2], dev(alpha), dev(u)).cpu().numpy()
    assert (got >= 0).all()
    counts = {}
    for r in got:
        t = OS.pattern(r, m)
        counts[t] = counts.get(t, 0) + 1
    chi2, dof = 0.0, 0
    from test_sampler_oracle import all_patterns
    for t in all_patterns(m, n):
        p, _ = oracle.prob(U, [1, 1, 1, 0, 0], list(t))
        e = N * p
        if e >= 5:
            chi2 += (counts.get(t, 0) - e) ** 2 / e
            dof += 1
    # 35 patterns: for <= 34 degrees of freedom P(chi2 > 80) < 1e-5
    assert dof >= 20 and chi2 < 80.0, (chi2, dof)


@pytest.mark.parametrize("prec", ["fp64", "fp64_df", "fp32x2"])
def test_hong_ou_mandel_32_photons(pg, prec):
    """16 beam splitters side by side, one photon in every mode: every pair bunches."""
    m = n = 32
    U = np.zeros((m, m), dtype=complex)
    for p in range(16):
        U[2 * p:2 * p + 2, 2 * p:2 * p + 2] = np.array([[1, 1], [1, -1]]) / math.sqrt(2)
    alpha, u = draws(3232, 2, n)
    got = pg.boson_sample(dev(U), list(range(n)), dev(alpha), dev(u), prec=prec).cpu().numpy()
    for r in got:
        t = OS.pattern(r, m)
        assert all(t[2 * p] + t[2 * p + 1] == 2 and t[2 * p] != 1 for p in range(16)), t


def test_permutation_unitary_24_photons(pg):
    m, n = 40, 24
    g = np.random.default_rng(4)
    pi = g.permutation(m)
    U = np.zeros((m, m), dtype=complex)
    U[np.arange(m), pi] = np.exp(1j * g.random(m))
    inputs = sorted(g.choice(m, size=n, replace=False).tolist())
    alpha, u = draws(24, 2, n)
    got = pg.boson_sample(dev(U), inputs, dev(alpha), dev(u)).cpu().numpy()
    for s in range(2):
        assert list(got[s]) == [pi[inputs[a]] for a in alpha[s]]


def test_invalid_draw_inputs_mark_only_that_draw(pg):
    m, n = 10, 4
    U = S.haar_unitary(m, 8)
    alpha, u = draws(5, 4, n)
    alpha[1] = [0, 0, 1, 2]      # not a permutation
    u[2, 3] = 1.0                # outside [0, 1)
    got = pg.boson_sample(dev(U), [1, 3, 5, 7], dev(alpha), dev(u)).cpu().numpy()
    assert (got[1] == -1).all() and (got[2] == -1).all()
    for s in (0, 3):
        want, _ = OS.sample(U, [1, 3, 5, 7], alpha[s], u[s])
        assert list(got[s]) == want


def test_host_argument_errors(pg):
    from paper_1606_05836_gb300 import PermError
    U = dev(S.haar_unitary(6, 1))
    alpha, u = draws(1, 2, 3)
    with pytest.raises(PermError):
        pg.boson_sample(U, [1, 1, 2], dev(alpha), dev(u))  # repeated input mode
    with pytest.raises(PermError):
        pg.boson_sample(U, [0, 1, 6], dev(alpha), dev(u))  # mode out of range
    with pytest.raises(ValueError):
        pg.BosonSampler(U, list(range(33)), 1)


def test_graph_replay_matches_run(pg):
    import torch
    m, n, ns = 50, 10, 8
    U = dev(S.haar_unitary(m, 12))
    alpha, u = draws(77, ns, n)
    smp = pg.BosonSampler(U, list(range(0, 2 * n, 2)), ns)
    first = smp.run(dev(alpha), dev(u)).clone()
    smp.capture()
    smp.out.fill_(-7)
    again = smp.replay().clone()
    torch.cuda.synchronize()
    assert torch.equal(first, again)
    alpha2, u2 = draws(78, ns, n)
    smp.load(dev(alpha2), dev(u2))
    third = smp.replay().cpu().numpy()
    check_against_oracle(S.haar_unitary(m, 12), list(range(0, 2 * n, 2)), alpha2, u2, third)


@pytest.mark.parametrize("m,n,ns", [(5, 1, 30), (6, 6, 12), (2, 2, 40)])
def test_draw_edge_sizes_match_oracle(pg, m, n, ns):
    """One photon (weights |U[in, l]|^2 only), every mode occupied (m = n), the
    smallest interferometer: equal draws to the oracle's."""
    U = S.haar_unitary(m, 50 + m + n)
    inputs = list(range(m - n, m))
    alpha, u = draws(60 + m + n, ns, n)
    got = pg.boson_sample(dev(U), inputs, dev(alpha), dev(u)).cpu().numpy()
    check_against_oracle(U, inputs, alpha, u, got)
    assert (got >= 0).all() and (got < m).all()


def test_identity_photon_order_and_row_minors_batch_of_one(pg):
    """alpha = identity for every draw is valid; a batch of one matrix equals the unbatched call."""
    import numpy as np_
    m, n, ns = 12, 5, 6
    U = S.haar_unitary(m, 77)
    alpha = np_.tile(np_.arange(n, dtype=np_.int32), (ns, 1))
    _, u = draws(78, ns, n)
    got = pg.boson_sample(dev(U), [1, 3, 5, 7, 9], dev(alpha), dev(u)).cpu().numpy()
    check_against_oracle(U, [1, 3, 5, 7, 9], alpha, u, got)
    M = S.circular_gaussian((8, 9), 79, 1.0 / 9)
    one = pg.row_minors(dev(M)).cpu().numpy()
    batch = pg.row_minors(dev(M[None, :, :])).cpu().numpy()
    assert np_.array_equal(one, batch[0])
