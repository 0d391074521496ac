"""Writes ladder_refs.tsv: oracle reference permanents of the precision-ladder inputs.

Inputs (module ``synthetic``): Gaussian var 1/n^2, all-ones + 1e-3 Gaussian, and
0/1 Bernoulli(1/2), n = 16, 24, 28, seed 0.  References come from ``oracle``
only: the quad-precision Gray-order Glynn evaluation (Eq. (S2)) for the complex
inputs and the exact int128 Ryser evaluation (Eq. (S1)) for the 0/1 inputs.
Each row carries the SHA-256 of the input matrix (complex128 bytes) so a test can
tell that it regenerated the same input.

Usage: python tests/golden/make_ladder_refs.py   (a few minutes on 8 cores)
"""
import hashlib
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synthetic as S  # noqa: E402

CASES = [(kind, n, 0) for n in (16, 24, 28) for kind in ("gaussian", "ones_noise", "bernoulli")]


def make_input(kind, n, seed):
    if kind == "gaussian":
        return S.gaussian(n, seed)
    if kind == "ones_noise":
        return S.ones_plus_noise(n, seed)
    return S.bernoulli01(n, seed).astype(np.complex128)


def digest(A):
    return hashlib.sha256(np.ascontiguousarray(A, dtype=np.complex128).tobytes()).hexdigest()[:16]


def main():
    rows = []
    for kind, n, seed in CASES:
        A = make_input(kind, n, seed)
        if kind == "bernoulli":
            v = oracle.ryser_int(A.real.astype(np.int64))
            hi = float(v)
            lo = float(v - int(hi))
            ref = (hi, lo, 0.0, 0.0, "ryser_int")
        else:
            q = oracle.glynn_gray(A)
            ref = (q.hi.real, q.lo.real, q.hi.imag, q.lo.imag, "glynn_gray")
        rows.append((kind, n, seed, digest(A)) + ref)
        print(kind, n, ref, flush=True)
    with open(os.path.join(HERE, "ladder_refs.tsv"), "w") as f:
        f.write("# Oracle references for the precision ladder (written by make_ladder_refs.py).\n")
        f.write("# value = re_hi + re_lo + i (im_hi + im_lo); sha = SHA-256 prefix of the input.\n")
        f.write("kind\tn\tseed\tsha\tre_hi\tre_lo\tim_hi\tim_lo\toracle\n")
        for r in rows:
            f.write("%s\t%d\t%d\t%s\t%r\t%r\t%r\t%r\t%s\n" % r)


if __name__ == "__main__":
    main()
