"""Build libperm.so (the C-ABI library) for sm_103a with nvcc.

Translation units are compiled in parallel (the forward kernels are split into
size groups) and linked into ``paper_1606_05836_gb300/lib/libperm.so``.  Objects
are rebuilt only when a source or header is newer than the object.

Usage: ``python -m paper_1606_05836_gb300.build [-j JOBS] [--force]``.
"""
from __future__ import annotations

import argparse
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIBDIR, "libperm.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]

# Translation units compiled several times with different -D values (so their
# template instances build in parallel).
MULTI = {
    "fwd_inst.cu": ["-DPERM_PART=%d" % p for p in range(8)],
    "batched_inst.cu": ["-DPERM_PREC=%d" % p for p in range(5)],
    "grad_inst.cu": ["-DPERM_PART=%d" % p for p in range(4)],
    "minors_inst.cu": ["-DPERM_PART=%d" % p for p in range(4)],
}


def _nvcc() -> str:
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libperm")


def _headers() -> list[str]:
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return hs


def _units() -> list[tuple[str, str, list[str]]]:
    """(source, object, extra flags) for every translation unit."""
    units = []
    for f in sorted(os.listdir(CSRC)):
        if not f.endswith(".cu"):
            continue
        if f in MULTI:
            for i, d in enumerate(MULTI[f]):
                units.append((os.path.join(CSRC, f), os.path.join(BUILD, "%s_%d.o" % (f[:-3], i)), [d]))
        else:
            units.append((os.path.join(CSRC, f), os.path.join(BUILD, f[:-3] + ".o"), []))
    return units


def _stale(obj: str, deps: list[str]) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(jobs: int | None = None, force: bool = False, verbose: bool = False) -> str:
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    headers = _headers()
    units = _units()
    todo = [u for u in units if force or _stale(u[1], [u[0]] + headers)]

    def compile_one(u):
        src, obj, extra = u
        cmd = [nvcc] + NVFLAGS + extra + ["-c", src, "-o", obj + ".tmp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
        os.replace(obj + ".tmp", obj)
        if verbose:
            print("compiled", os.path.relpath(obj, ROOT), flush=True)

    if todo:
        jobs = jobs or max(1, min(len(todo), os.cpu_count() or 4))
        with ThreadPoolExecutor(max_workers=jobs) as ex:
            list(ex.map(compile_one, todo))
    objs = [u[1] for u in units]
    if force or todo or _stale(LIB, objs):
        cmd = [nvcc] + ARCH + ["-shared", "-o", LIB + ".tmp"] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
        os.replace(LIB + ".tmp", LIB)
        if verbose:
            print("linked", os.path.relpath(LIB, ROOT), flush=True)
    return LIB


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("-j", "--jobs", type=int, default=None)
    ap.add_argument("--force", action="store_true")
    a = ap.parse_args()
    print(build(a.jobs, a.force, verbose=True))


if __name__ == "__main__":
    main()
