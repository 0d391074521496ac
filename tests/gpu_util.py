"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np

# Parity bar for FP64 results against the quad / exact oracle (relative error).
REL_TOL = 1e-10


def to_dev(A):
    import torch
    return torch.as_tensor(np.ascontiguousarray(A, dtype=np.complex128)).cuda()


def val(t) -> complex:
    return complex(t.cpu().item())


def pair(t) -> tuple[complex, complex]:
    """(hi, lo) of a range partial sum."""
    v = t.cpu().numpy()
    return complex(v[0]), complex(v[1])


def rel(x: complex, want) -> float:
    """|x - want| / |want|, want an oracle QC or a number."""
    if hasattr(want, "hi"):
        return want.rel_err(x)
    return abs(complex(x) - complex(want)) / abs(complex(want))


def row_scale(A) -> float:
    """prod_i ||row_i||_2: the size of a typical term, a scale for partial sums."""
    return float(np.prod(np.linalg.norm(np.asarray(A), axis=1)))
