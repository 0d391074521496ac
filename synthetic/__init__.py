"""Seeded synthetic inputs shared by the oracle tests, the GPU parity tests and bench.py.

This module only *builds input matrices*; it holds none of the permanent's
arithmetic.  Every generator takes an explicit seed and uses
``numpy.random.default_rng(seed)``.

Input recipe (stand-ins for the paper's matrices, which were MATLAB-generated and
are not published, arXiv 1606.05836 Supp. tables of random-unitary,
random-derived and special-derived results):

* Haar unitary (m x m): QR of an i.i.d. circular complex Gaussian (Ginibre)
  matrix, the phases of R's diagonal folded into Q (Mezzadri's construction).
* Collision-free n-photon submatrix of an m = n^2 mode Haar unitary: entries
  i.i.d. circular complex Gaussian with variance 1/n^2 (``gaussian``).
* Cancellation-heavy stand-in for the "special-derived" class: all-ones plus
  1e-3 x circular Gaussian (``ones_plus_noise``).
* 0/1 Bernoulli(1/2) matrices (``bernoulli01``), whose permanents are exact
  integer perfect-matching counts.
* Batched output patterns of one unitary (``batch_patterns``): n uniform in a
  range, rows drawn without replacement, columns without replacement for 80 % of
  the items and with at least one repeat (a photon collision) for the rest.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def circular_gaussian(shape, seed: int, var: float = 1.0) -> np.ndarray:
    """i.i.d. complex entries with E|z|^2 = var, real and imaginary parts N(0, var/2)."""
    g = rng(seed)
    re = g.standard_normal(shape)
    im = g.standard_normal(shape)
    return (re + 1j * im) * np.sqrt(var / 2.0)


def haar_unitary(m: int, seed: int) -> np.ndarray:
    """Haar-random m x m unitary: Q of QR(Ginibre), times diag(r_ii / |r_ii|)."""
    Z = circular_gaussian((m, m), seed, 1.0)
    Q, R = np.linalg.qr(Z)
    d = np.diag(R)
    ph = d / np.abs(d)
    return np.ascontiguousarray(Q * ph[None, :])


def haar_block(n: int, m: int, seed: int) -> np.ndarray:
    """Top-left n x n block of an m x m Haar unitary."""
    return np.ascontiguousarray(haar_unitary(m, seed)[:n, :n])


def gaussian(n: int, seed: int, var: float | None = None) -> np.ndarray:
    """n x n circular Gaussian, variance 1/n^2 by default."""
    if var is None:
        var = 1.0 / (n * n)
    return np.ascontiguousarray(circular_gaussian((n, n), seed, var))


def ones_plus_noise(n: int, seed: int, eps: float = 1e-3) -> np.ndarray:
    return np.ascontiguousarray(np.ones((n, n), dtype=np.complex128) + eps * circular_gaussian((n, n), seed, 1.0))


def bernoulli01(n: int, seed: int, p: float = 0.5) -> np.ndarray:
    """0/1 matrix (int64) with i.i.d. Bernoulli(p) entries."""
    return (rng(seed).random((n, n)) < p).astype(np.int64)


def all_r(n: int, r: complex) -> np.ndarray:
    return np.full((n, n), r, dtype=np.complex128)


def ones_minus_identity(n: int) -> np.ndarray:
    return np.ones((n, n), dtype=np.complex128) - np.eye(n, dtype=np.complex128)


def diagonal(d) -> np.ndarray:
    d = np.asarray(d, dtype=np.complex128)
    return np.diag(d)


def rank_one(n: int, seed: int) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """(u v^T, u, v) with u, v circular Gaussian of unit variance."""
    u = circular_gaussian((n,), seed, 1.0)
    v = circular_gaussian((n,), seed + 7919, 1.0)
    return np.ascontiguousarray(np.outer(u, v)), u, v


def random_permutations(n: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    g = rng(seed)
    return g.permutation(n), g.permutation(n)


def batch_patterns(U: np.ndarray, count: int, n_lo: int, n_hi: int, seed: int, collision_frac: float = 0.2):
    """Output patterns of one m x m unitary U.

    Returns (mats, ns, s_rows, t_cols, collide): ``mats[k]`` is the n_k x n_k
    submatrix with rows ``s_rows[k]`` (distinct input modes, one photon each) and
    columns ``t_cols[k]`` (output modes, repeated for collisions, ascending).
    """
    m = U.shape[0]
    g = rng(seed)
    mats, ns, rows_l, cols_l, collide = [], [], [], [], []
    for _ in range(count):
        n = int(g.integers(n_lo, n_hi + 1))
        rows = np.sort(g.choice(m, size=n, replace=False))
        c = bool(g.random() < collision_frac) and n >= 2
        if c:
            while True:
                cols = np.sort(g.choice(m, size=n, replace=True))
                if len(np.unique(cols)) < n:
                    break
                # force a repeat: copy one column index onto another slot
                i, j = g.choice(n, size=2, replace=False)
                cols[i] = cols[j]
                cols = np.sort(cols)
                break
        else:
            cols = np.sort(g.choice(m, size=n, replace=False))
        mats.append(np.ascontiguousarray(U[np.ix_(rows, cols)]))
        ns.append(n)
        rows_l.append(rows)
        cols_l.append(cols)
        collide.append(c)
    return mats, np.array(ns, dtype=np.int32), rows_l, cols_l, np.array(collide)


def sampler_draws(n: int, count: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Random inputs of ``count`` boson-sampling draws of n photons: int32 photon
    orders (each row a uniform permutation of 0..n-1) and float64 uniforms in [0, 1)."""
    g = rng(seed)
    alpha = np.stack([g.permutation(n) for _ in range(count)]).astype(np.int32)
    u = g.random((count, n))
    return alpha, u
