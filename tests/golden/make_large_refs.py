"""Writes large_refs.tsv: oracle permanents of inputs at n = 32-40.

At these sizes the quad-precision oracle is too slow (about 50 minutes per
n = 32 matrix on 8 cores, 16x more per +4 in n), so the references come from
``oracle.glynn_f64dd``: Eq. (S2) in reflected-Gray order with FP64 row sums and
products and double-double accumulation (minutes at n = 36, hours at n = 40 on
8 cores).  Its agreement with the quad oracle is pinned in
tests/test_oracle_pins.py (n <= 28 directly; n = 32 against the stored quad
values of sweep_refs.tsv; n = 36 on a block-diagonal matrix whose permanent is
the product of two quad-oracle block permanents).

Inputs (module ``synthetic``):
  gaussian    the benchmark sweep's matrices, i.i.d. circular Gaussian, variance 1/n^2
  ones_noise  all-ones + 1e-3 Gaussian (the precision ladder's cancellation input)
  bernoulli   0/1 entries, Bernoulli(1/2)
  block_diag  diag(B1, B2) with Gaussian blocks of n/2 (seeds s, s+1), rows and
              columns permuted (seed s+2)
Each row carries the SHA-256 prefix of the input (complex128 bytes), so a test
can tell that it regenerated the same matrix.  References come from ``oracle``
only.  Rows already present are kept; missing ones are computed in CASES order
and appended one by one.

Usage: python tests/golden/make_large_refs.py [kind:n:seed ...]
"""
import hashlib
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synthetic as S  # noqa: E402

OUT = os.path.join(HERE, "large_refs.tsv")
HEADER = ("# FP64 / double-double Gray-order Glynn (oracle.glynn_f64dd) of inputs at n = 32-40.\n"
          "# value = re_hi + re_lo + i (im_hi + im_lo); sha = SHA-256 prefix of the input; seconds = host time.\n"
          "kind\tn\tseed\tsha\tre_hi\tre_lo\tim_hi\tim_lo\toracle\tseconds\n")

CASES = ([("gaussian", 32, s) for s in (0, 1, 2)] + [("ones_noise", 32, 0), ("bernoulli", 32, 0)]
         + [("gaussian", 36, s) for s in (0, 1, 2)] + [("block_diag", 36, 36036)]
         + [("ones_noise", 36, 0), ("bernoulli", 36, 0)] + [("gaussian", 40, 0)])


def make_input(kind, n, seed):
    if kind == "gaussian":
        return S.gaussian(n, seed)
    if kind == "ones_noise":
        return S.ones_plus_noise(n, seed)
    if kind == "bernoulli":
        return S.bernoulli01(n, seed).astype(np.complex128)
    if kind == "block_diag":
        h = n // 2
        A = np.zeros((n, n), dtype=np.complex128)
        A[:h, :h], A[h:, h:] = block_diag_blocks(n, seed)
        P, Q = S.random_permutations(n, seed + 2)
        return np.ascontiguousarray(A[P][:, Q])
    raise ValueError(kind)


def block_diag_blocks(n, seed):
    h = n // 2
    return S.gaussian(h, seed), S.gaussian(n - h, seed + 1)


def digest(A):
    return hashlib.sha256(np.ascontiguousarray(A, dtype=np.complex128).tobytes()).hexdigest()[:16]


def main(cases):
    have = set()
    if os.path.exists(OUT):
        for line in open(OUT):
            if line[:1].isalpha() and not line.startswith("kind"):
                f = line.split("\t")
                have.add((f[0], int(f[1]), int(f[2])))
    else:
        with open(OUT, "w") as fh:
            fh.write(HEADER)
    for kind, n, seed in cases:
        if (kind, n, seed) in have:
            continue
        A = make_input(kind, n, seed)
        t0 = time.time()
        q = oracle.glynn_f64dd(A)
        dt = time.time() - t0
        with open(OUT, "a") as fh:
            fh.write("%s\t%d\t%d\t%s\t%r\t%r\t%r\t%r\tglynn_f64dd\t%.0f\n" % (
                kind, n, seed, digest(A), q.hi.real, q.lo.real, q.hi.imag, q.lo.imag, dt))
            fh.flush()
        print(kind, n, seed, q.hi, "%.0f s" % dt, flush=True)


if __name__ == "__main__":
    args = [a.split(":") for a in sys.argv[1:]]
    main([(k, int(n), int(s)) for k, n, s in args] or CASES)
