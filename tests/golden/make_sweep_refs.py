"""Writes sweep_refs.tsv: oracle permanents of the benchmark sweep's largest inputs.

The sweep times one complex128 Gaussian matrix (variance 1/n^2) per (n, seed),
seeds 0, 1, 2 (module ``synthetic``, platform-independent generator).  At n = 32
the quad-precision Gray-order Glynn evaluation (Eq. (S2), ``oracle.glynn_gray``)
takes tens of minutes per matrix on a CPU host, too long for a test, so its
values are stored here with the SHA-256 of the input.  References come from
``oracle`` only.

Usage: python tests/golden/make_sweep_refs.py [seed ...]   (about an hour per seed on 8 cores)
Rows already present are kept; new seeds are appended.
"""
import hashlib
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synthetic as S  # noqa: E402

OUT = os.path.join(HERE, "sweep_refs.tsv")
HEADER = ("# Quad-precision Gray-order Glynn (oracle.glynn_gray) of the sweep's n = 32 inputs.\n"
          "# value = re_hi + re_lo + i (im_hi + im_lo); sha = SHA-256 prefix of the input.\n"
          "n\tseed\tsha\tre_hi\tre_lo\tim_hi\tim_lo\toracle\n")


def digest(A):
    return hashlib.sha256(np.ascontiguousarray(A, dtype=np.complex128).tobytes()).hexdigest()[:16]


def main(seeds):
    have = set()
    if os.path.exists(OUT):
        for line in open(OUT):
            if line[:1].isdigit():
                f = line.split("\t")
                have.add((int(f[0]), int(f[1])))
    else:
        with open(OUT, "w") as fh:
            fh.write(HEADER)
    for seed in seeds:
        n = 32
        if (n, seed) in have:
            continue
        A = S.gaussian(n, seed)
        q = oracle.glynn_gray(A)
        with open(OUT, "a") as fh:
            fh.write("%d\t%d\t%s\t%r\t%r\t%r\t%r\tglynn_gray\n" % (n, seed, digest(A), q.hi.real, q.lo.real,
                                                                   q.hi.imag, q.lo.imag))
            fh.flush()


if __name__ == "__main__":
    main([int(x) for x in sys.argv[1:]] or [0, 1, 2])
