"""Boson-sampling draws on top of the permanent oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s ``cpu_baseline`` /
``--impl reference`` leg may import this module; the GPU product path never
imports or executes it, and it shares no code with ``paper_1606_05836_gb300``.

arXiv 1606.05836 gives the output distribution of boson sampling as Eq. (1),
Pr[S -> T] = |Per(U_ST)|^2 / (prod s_i! prod t_j!), and bounds the cost of one
draw by that of one permanent (Section 1).  This module draws from Eq. (1) with
the chain rule of P. Clifford and R. Clifford ("The classical complexity of
boson sampling", SODA 2018), restated from the published method:

* A[l, j] = U[inputs[alpha_j], l] (one photon in each of n distinct input
  modes; Eq. (1) takes the rows of U for the input modes and its columns for
  the output modes), the photons taken in the order of a uniformly random
  permutation alpha;
* for k = 1..n, every output mode l gets the weight
  w_k(l) = |Per(A[(r_1, .., r_{k-1}, l), (0, .., k-1)])|^2, evaluated by the
  Laplace expansion along the new last row,
  Per = sum_j A[l, j] Per(A[(r_1..r_{k-1}), (0..k-1) without j])
  (:func:`row_minors` gives the k permanents of the (k-1) x k matrix);
* r_k is the first l whose running sum of w_k exceeds u_k * sum_l w_k(l).

The random draws (alpha, u_1..u_n) are inputs, so the GPU sampler and this
oracle make the same decisions on the same draws.  Conventions fixed here:
running sums in mode order; if rounding leaves u W at or above every running
sum, the last mode of positive weight is taken; a step whose total weight is
zero or not finite ends the draw and marks it failed (-1 from then on).

Parity pins (tests/test_sampler_oracle.py): closed-form minors of rank-one
matrices, the Laplace identity against the permutation-sum definition, the
exact output distribution of the chain (enumerated over alpha and every draw
sequence) equal to Eq. (1), Hong-Ou-Mandel bunching, permutation-matrix
unitaries (deterministic outputs) and a Monte-Carlo histogram.
"""
from __future__ import annotations

import itertools
import math
from collections import defaultdict

import numpy as np

from . import perm_def, ryser


def row_minors(M) -> np.ndarray:
    """m_j = Per(M without column j) for a (k-1) x k matrix M, j = 0..k-1.

    Each minor is a square permanent: the permutation-sum definition up to
    order 8, Supp. Eq. (S1) in quad precision above.  k = 1 gives [1] (the
    permanent of the empty matrix).
    """
    M = np.asarray(M, dtype=np.complex128)
    if M.ndim != 2 or M.shape[1] != M.shape[0] + 1:
        raise ValueError("row_minors wants a (k-1) x k matrix, got %r" % (M.shape,))
    k = M.shape[1]
    if k == 1:
        return np.ones(1, dtype=np.complex128)
    out = np.empty(k, dtype=np.complex128)
    for j in range(k):
        sub = np.ascontiguousarray(np.delete(M, j, axis=1))
        q = perm_def(sub) if k - 1 <= 8 else ryser(sub)
        out[j] = q.hi + q.lo
    return out


def step_weights(A, r_prefix, k: int) -> np.ndarray:
    """w_k(l) = |sum_j A[l, j] Per(A[r_prefix, 0..k-1 without j])|^2 for every l.

    ``A`` is m x n with its columns already in the random order; ``r_prefix``
    holds r_1..r_{k-1}.
    """
    A = np.asarray(A, dtype=np.complex128)
    r_prefix = list(r_prefix)
    if len(r_prefix) != k - 1:
        raise ValueError("step %d needs %d earlier draws" % (k, k - 1))
    minors = row_minors(A[r_prefix, :k]) if k > 1 else np.ones(1, dtype=np.complex128)
    amp = A[:, :k] @ minors
    return amp.real * amp.real + amp.imag * amp.imag


def choose(w, u: float) -> int:
    """The first l with (w_0 + .. + w_l) > u W, W = sum of w; -1 if W is not > 0."""
    w = np.asarray(w, dtype=np.float64)
    c = np.cumsum(w)
    W = c[-1] if len(c) else 0.0
    if not (W > 0.0) or not math.isfinite(W):
        return -1
    x = u * W
    l = int(np.searchsorted(c, x, side="right"))
    if l >= len(w):
        l = int(np.nonzero(w > 0.0)[0][-1])
    return l


def choice_margin(w, u: float) -> float:
    """Distance of u W from the nearest running sum, relative to W (ties are 0)."""
    c = np.cumsum(np.asarray(w, dtype=np.float64))
    W = c[-1]
    return float(np.min(np.abs(c - u * W)) / W) if W > 0 else 0.0


def _columns(U, inputs, alpha):
    U = np.asarray(U, dtype=np.complex128)
    inputs = [int(x) for x in inputs]
    alpha = [int(x) for x in alpha]
    n = len(inputs)
    if sorted(alpha) != list(range(n)):
        raise ValueError("alpha must be a permutation of 0..n-1")
    if len(set(inputs)) != n:
        raise ValueError("input modes must be distinct")
    return np.ascontiguousarray(U[[inputs[a] for a in alpha], :].T)


def sample(U, inputs, alpha, u):
    """One draw: (r_1..r_n, per-step margins) for the random inputs alpha, u."""
    A = _columns(U, inputs, alpha)
    n = A.shape[1]
    r, margins = [], []
    for k in range(1, n + 1):
        w = step_weights(A, r, k)
        l = choose(w, float(u[k - 1]))
        if l < 0:
            return [-1] * n, margins
        margins.append(choice_margin(w, float(u[k - 1])))
        r.append(l)
    return r, margins


def pattern(r, m: int):
    """Output occupation vector t (length m) of a draw sequence."""
    t = [0] * m
    for x in r:
        t[x] += 1
    return tuple(t)


def chain_distribution(U, inputs):
    """Exact distribution of the output pattern produced by the chain.

    Enumerates every column order alpha (probability 1/n!) and every draw
    sequence, multiplying the step probabilities w_k(r_k) / W_k.  Tiny cases
    only (n! m^n leaves).
    """
    U = np.asarray(U, dtype=np.complex128)
    m, n = U.shape[0], len(inputs)
    dist = defaultdict(float)
    perms = list(itertools.permutations(range(n)))
    for alpha in perms:
        A = _columns(U, inputs, alpha)

        def walk(prefix, p):
            k = len(prefix) + 1
            if k > n:
                dist[pattern(prefix, m)] += p / len(perms)
                return
            w = step_weights(A, prefix, k)
            W = float(np.sum(w))
            if W <= 0.0:
                return
            for l in range(m):
                if w[l] > 0.0:
                    walk(prefix + [l], p * w[l] / W)

        walk([], 1.0)
    return dict(dist)
