"""Writes bench_refs.json: oracle values that bench.py compares its GPU results with.

bench.py itself never runs the oracle outside its CPU-baseline leg; the parity
figures it reports next to the timed forms come from this file.  Inputs are the
ones bench.py builds (module ``synthetic``), each stored with the SHA-256 of the
input so bench.py can tell that it regenerated the same input:

* glynn_gaussian_n20: Per of the n = 20 Gaussian (seed 0), quad Glynn (Eq. (S2));
* batched_items: the first 8 items with n <= 14 of the 4096-item batch (one Haar
  1000 x 1000 unitary, seed 0; patterns seed 1), quad Glynn, stored with the
  matrices themselves (a Haar unitary comes out of a LAPACK QR, whose last bits
  differ between machines, so bench.py runs these stored matrices);
* sampler_m30_n8: 4 draws of 8 photons (modes 0..7) of a Haar 30 x 30 unitary
  (seed 3, stored) with the draw inputs of seed 6, by oracle/sampler.py.

Usage: python tests/golden/make_bench_refs.py   (about a minute)
"""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synthetic as S  # noqa: E402
from oracle import sampler as OS  # noqa: E402


def digest(A):
    return hashlib.sha256(np.ascontiguousarray(A).tobytes()).hexdigest()[:16]


def flat(A):
    """Row-major [re, im, re, im, ...] of a complex matrix (exact decimal round trip)."""
    return np.ascontiguousarray(A, dtype=np.complex128).view(np.float64).ravel().tolist()


def qc(q):
    return [q.hi.real, q.lo.real, q.hi.imag, q.lo.imag]


def main():
    out = {}
    A20 = S.gaussian(20, 0)
    out["glynn_gaussian_n20"] = {"sha": digest(A20), "value": qc(oracle.glynn(A20))}
    U = S.haar_unitary(1000, 0)
    mats, ns, _, _, _ = S.batch_patterns(U, 4096, 8, 24, 1)
    small = [i for i in range(len(mats)) if ns[i] <= 14][:8]
    out["batched_items"] = [{"index": i, "n": int(ns[i]), "sha": digest(mats[i]), "value": qc(oracle.glynn(mats[i])),
                             "matrix": flat(mats[i])} for i in small]
    U30 = S.haar_unitary(30, 3)
    alpha, u = S.sampler_draws(8, 4, 6)
    out["sampler_m30_n8"] = {"sha_U": digest(U30), "U": flat(U30), "sha_alpha": digest(alpha), "sha_u": digest(u),
                             "draws": [OS.sample(U30, list(range(8)), alpha[i], u[i])[0] for i in range(4)]}
    with open(os.path.join(HERE, "bench_refs.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
