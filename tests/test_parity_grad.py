"""GPU parity of the adjoint (perm_grad) through the C ABI: minors against the
oracle's minor permanents, central finite differences of |Per|^2, the Laplace
(Euler) identities at the full sizes n = 24 and 32, and the autograd Function."""
import numpy as np
import pytest

import oracle
import synthetic as S
from gpu_util import REL_TOL, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    import paper_1606_05836_gb300 as pg
    from paper_1606_05836_gb300 import build
    build.build()
    pg.library()
    return pg


def normwise(M, W):
    return float(np.max(np.abs(M - W)) / np.max(np.abs(W)))


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 12, 14, 16, 17])
def test_minors_vs_oracle(pg, n):
    """All n^2 minors against the oracle's minor permanents; from n = 16 on the
    kernel prefetches the H column that the next Gray step flips."""
    A = S.gaussian(n, 900 + n, 1.0)
    per, abs2, M, G = pg.grad(to_dev(A), minor=True, grad_abs2=True)
    want_p = oracle.ryser(A) if n > 0 else None
    assert want_p.rel_err(complex(per.cpu().item())) < REL_TOL
    # |Per|^2 and 2 Per conj(M) combine two computed factors: twice the bar
    assert abs(abs2.item() - abs(want_p.hi) ** 2) <= 2 * REL_TOL * abs(want_p.hi) ** 2
    if n == 1:
        assert complex(M.cpu()[0, 0].item()) == 1.0
        return
    W = oracle.minors(A)
    assert normwise(M.cpu().numpy(), W) < REL_TOL
    Gw = 2 * want_p.hi * np.conj(W)
    assert normwise(G.cpu().numpy(), Gw) < 2 * REL_TOL


def test_minors_sampled_n20(pg):
    A = S.gaussian(20, 920)
    _, _, M, _ = pg.grad(to_dev(A))
    M = M.cpu().numpy()
    for i, j in [(0, 0), (3, 17), (19, 19), (11, 4)]:
        sub = np.delete(np.delete(A, i, axis=0), j, axis=1)
        want = oracle.ryser(sub)
        assert want.rel_err(M[i, j]) < REL_TOL


@pytest.mark.parametrize("n", [6, 12])
def test_finite_differences_abs2(pg, n):
    """Central differences (h = 1e-6) of |Per|^2 in Re a_ij and Im a_ij, Per from
    the quad oracle, against d|Per|^2/dRe a + i d|Per|^2/dIm a."""
    A = S.gaussian(n, 930 + n, 1.0)
    _, _, _, G = pg.grad(to_dev(A), minor=False, grad_abs2=True)
    G = G.cpu().numpy()
    h = 1e-6
    for i, j in [(0, 0), (n - 1, 1), (n // 2, n - 1)]:
        for unit in (1.0, 1j):
            Ap, Am = A.copy(), A.copy()
            Ap[i, j] += h * unit
            Am[i, j] -= h * unit
            fp = abs(oracle.glynn(Ap).hi) ** 2
            fm = abs(oracle.glynn(Am).hi) ** 2
            fd = (fp - fm) / (2 * h)
            got = G[i, j].real if unit == 1.0 else G[i, j].imag
            assert abs(got - fd) <= 1e-6 * np.max(np.abs(G)), (i, j, unit, got, fd)


@pytest.mark.parametrize("n", [24, 32])
def test_laplace_identity_full_size(pg, n):
    """sum_j a_ij dPer/da_ij = Per for every row i (and every column): the
    property check at the configured adjoint sizes, where no minor oracle runs."""
    A = S.gaussian(n, 940 + n)
    per, _, M, _ = pg.grad(to_dev(A))
    M = M.cpu().numpy()
    P = complex(per.cpu().item())
    rows = np.sum(A * M, axis=1)
    cols = np.sum(A * M, axis=0)
    assert np.max(np.abs(rows - P)) <= REL_TOL * abs(P) * 10
    assert np.max(np.abs(cols - P)) <= REL_TOL * abs(P) * 10
    single = complex(pg.glynn(to_dev(A)).cpu().item())
    assert abs(P - single) <= REL_TOL * abs(single)


def test_batch_matches_single_items(pg):
    mats = np.stack([S.gaussian(10, 950 + b, 1.0) for b in range(6)])
    per, abs2, M, _ = pg.grad(to_dev(mats))
    for b in range(6):
        pb, _, Mb, _ = pg.grad(to_dev(mats[b]))
        assert complex(per[b].cpu().item()) == complex(pb.cpu().item())
        assert np.array_equal(M[b].cpu().numpy(), Mb.cpu().numpy())
    W = oracle.minors(mats[3])
    assert normwise(M[3].cpu().numpy(), W) < REL_TOL


def test_autograd_function(pg):
    import torch
    A = S.gaussian(9, 960, 1.0)
    t = to_dev(A).requires_grad_(True)
    y = pg.PermAbs2.apply(t)
    y.backward()
    P = oracle.ryser(A).hi
    W = oracle.minors(A)
    assert abs(y.item() - abs(P) ** 2) <= 2 * REL_TOL * abs(P) ** 2
    assert normwise(t.grad.cpu().numpy(), 2 * P * np.conj(W)) < 2 * REL_TOL
    # batched, with a non-trivial upstream gradient
    mats = to_dev(np.stack([S.gaussian(7, 970 + b, 1.0) for b in range(3)])).requires_grad_(True)
    w = torch.tensor([0.5, -2.0, 3.0], dtype=torch.float64, device="cuda")
    (pg.PermAbs2.apply(mats) * w).sum().backward()
    for b in range(3):
        Ab = mats[b].detach().cpu().numpy()
        want = w[b].item() * 2 * oracle.ryser(Ab).hi * np.conj(oracle.minors(Ab))
        assert normwise(mats.grad[b].cpu().numpy(), want) < 2 * REL_TOL


@pytest.mark.parametrize("n", [1, 2, 3, 8, 14, 17])
def test_minors_vs_oracle_double_float_products(pg, n):
    """The R3 adjoint (prefix / suffix / q products in double-float on the FP32
    pipe, row sums and accumulators FP64) against the oracle's minors: the same
    1e-10 bar as the FP64 adjoint."""
    A = S.gaussian(n, 980 + n, 1.0)
    per, abs2, M, G = pg.grad(to_dev(A), minor=True, grad_abs2=True, prec="fp64_df")
    want_p = oracle.ryser(A)
    assert want_p.rel_err(complex(per.cpu().item())) < REL_TOL
    if n == 1:
        assert complex(M.cpu()[0, 0].item()) == 1.0
        return
    W = oracle.minors(A)
    assert normwise(M.cpu().numpy(), W) < REL_TOL
    assert normwise(G.cpu().numpy(), 2 * want_p.hi * np.conj(W)) < 2 * REL_TOL


@pytest.mark.parametrize("n", [24, 32])
def test_double_float_products_full_size(pg, n):
    """R3 adjoint at the configured sizes: the Laplace identities, and agreement
    with the FP64 adjoint's minors (normwise) and permanent."""
    A = S.gaussian(n, 990 + n)
    dA = to_dev(A)
    per, _, M, _ = pg.grad(dA, prec="fp64_df")
    per0, _, M0, _ = pg.grad(dA)
    M, M0 = M.cpu().numpy(), M0.cpu().numpy()
    P = complex(per.cpu().item())
    assert np.max(np.abs(np.sum(A * M, axis=1) - P)) <= REL_TOL * abs(P) * 10
    assert normwise(M, M0) < REL_TOL
    assert abs(P - complex(per0.cpu().item())) <= REL_TOL * abs(P)


def test_grad_rejects_other_precisions(pg):
    with pytest.raises(ValueError):
        pg.grad(to_dev(S.gaussian(4, 1, 1.0)), prec="fp32x2")
    import ctypes
    from paper_1606_05836_gb300._native import Opts, load
    o = Opts(2, 0, 0, 0, 0)
    assert load().perm_grad_workspace_size(4, ctypes.byref(o)) == 0
