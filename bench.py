#!/usr/bin/env python3
"""Throughput benchmark of the GB300 permanent engine.

Workload: the plain single-permanent sweep — complex128 n x n matrices with
i.i.d. circular Gaussian entries of variance 1/n^2 (the collision-free n-photon
submatrix of an m = n^2 mode Haar unitary), Glynn Gray-code sums in FP64, one
matrix per launch.  One step = one permanent per n with the seed cycling 0, 1, 2
over the steps.  Metric: Gray-code terms per second (2^(n-1) per permanent) of
the form that meets the 1e-10 bar, device-timed with CUDA events, inputs
resident in HBM; the L2 (129 MB) is flushed between steps by writing 256 MB.
Ryser (2^n terms; FP64 Ryser loses digits to cancellation, the paper's finding)
is timed on the same inputs after the sweep and reported apart with its error
(``by_method``); ``--kinds glynn,ryser`` puts it back into the timed steps.

The JSON line also carries: the end-to-end rate through the C ABI from pinned
host buffers (copies inside the timed region); the roofline of the dominant
kernel against the FP64 peak measured on the same GPU by the DFMA probe
(``perm_fp64_fma_probe``; the peak derived from SM count x 4 FP64 flop/clk/SM x
max SM clock beside it); Glynn and Ryser apart (terms/s, error of the timed n = 32
results against stored quad-oracle values); the SM clocks sampled during the
timed region; the CPU oracle's FP64 Gray-order Glynn (double-double sum) on full
permanents at n = 20-32 on all host cores (rank 0, N = 1); and the other forms
(precision rungs, batch, adjoint, collisions, row minors, draws, and single
Glynn permanents at n = 20, 36 and 40 against stored oracle values).

``--impl reference`` times the CPU oracle (the only reference implementation of
this method here: FP64 Gray-order Glynn / Ryser partial sums with double-double
accumulation) on the same workload, one bounded sample per item and step.

Multi-GPU (torchrun): every rank runs the same sweep on its own GPU — the
permanents are independent problems, so there is no data-path collective; the
step time is the max over ranks and ``value`` counts the terms of all ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gray-code terms/s (plain FP64 Glynn permanents, <= 1e-10 vs the oracle)"
UNIT = "terms/s"
L2_FLUSH_BYTES = 256 << 20


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n-list", default="24,28,32", help="matrix sizes of the sweep")
    ap.add_argument("--kinds", default="glynn",
                    help="methods of the timed sweep (Ryser, which misses the 1e-10 bar in FP64, is timed "
                         "and reported apart in by_method)")
    ap.add_argument("--prec", default="fp64", choices=["fp64", "fp64_dd", "fp32p_dd", "fp64_df", "fp32x2"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="target CPU time of the oracle baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the batched / compensated / adjoint forms")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the single n = 36 and n = 40 Glynn launches (about 3.7 minutes together)")
    ap.add_argument("--form", choices=["sweep", "batched", "adjoint", "sampler", "shard", "range"], default="sweep",
                    help="sweep = the metric above (default); batched / adjoint / sampler time only that "
                         "form (for profiling) and print its own JSON line; shard = one Glynn permanent "
                         "of --shard-n split over the ranks' Gray ranges with one exchange of partials; range = "
                         "one Glynn partial sum over the first 2^--range-log2 Gray indices at n = --range-n "
                         "(a shard-sized unit of a large permanent, for profiling)")
    ap.add_argument("--shard-n", type=int, default=36)
    ap.add_argument("--range-n", type=int, default=40,
                    help="--form range: size of the matrix whose first 2^--range-log2 Gray terms are summed")
    ap.add_argument("--range-log2", type=int, default=30)
    ap.add_argument("--batched-count", type=int, default=4096)
    ap.add_argument("--adjoint-n", type=int, default=24)
    ap.add_argument("--adjoint-batch", type=int, default=64)
    ap.add_argument("--adjoint-prec", default="fp64", choices=["fp64", "fp64_df"])
    ap.add_argument("--sampler-m", type=int, default=1000)
    ap.add_argument("--sampler-n", type=int, default=24)
    ap.add_argument("--sampler-count", type=int, default=16)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def terms_of(kind: str, n: int) -> int:
    return 2 ** (n - 1) if kind == "glynn" else 2 ** n


def flops_per_term(n: int) -> int:
    # update 2n + product 6(n-1) + accumulate 2 (FP64 flops per Gray-code term)
    return 8 * n - 4


def workload(args):
    ns = [int(x) for x in args.n_list.split(",") if x]
    kinds = [k for k in args.kinds.split(",") if k]
    return ns, kinds


def step_items(ns, kinds, step):
    seed = step % 3
    return [(k, n, seed) for n in ns for k in kinds]


def config_dict(args, ns, kinds, world):
    return {
        "workload": "plain single-permanent sweep: complex128 Gaussian var 1/n^2, n=%s, %s, %s, "
                    "seed cycling 0,1,2 over steps, one matrix per launch" % (
                        ",".join(map(str, ns)), "+".join(kinds), args.prec),
        "n": ns,
        "methods": kinds,
        "precision_rung": args.prec,
        "l2": "flushed between steps (256 MB write); inputs 16 n^2 bytes",
        "parallelism": "independent permanents per GPU (x%d)" % world,
    }


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = []
        for line in out.splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                rows.append(dict(sm=float(p[1]), smax=float(p[2]), power=float(p[3]), hw=p[5], hwt=p[6], swt=p[7],
                                 swp=p[8]))
            except ValueError:
                continue
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"), ("swt", "sw_thermal_slowdown"),
                              ("swp", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max(r["power"] for r in rows)}


# ---------------------------------------------------------------------------
# DRAM traffic of the dominant kernel, from a committed ncu summary
# ---------------------------------------------------------------------------
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "fwd_kernel_traffic.json")
KERNEL_SOURCES = ("common.cuh", "fwd_kernel.cuh", "fwd_inst.cu")


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1606_05836_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(n: int):
    """dram read+write bytes per launch of fwd_kernel<n> from the ncu capture,
    or None when there is none or the kernel sources changed since it was taken."""
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("source_sha256") != kernel_source_hash() or int(rec.get("n", -1)) != n:
        return None
    return rec.get("dram_bytes_per_launch")


# ---------------------------------------------------------------------------
# the oracle on the host cores
# ---------------------------------------------------------------------------
def oracle_sample_fn(kind):
    """The oracle's FP64 Gray-order partial sum (double-double accumulation) for a method."""
    import oracle
    return oracle.glynn_f64dd_range if kind == "glynn" else oracle.ryser_f64dd_range


def oracle_full_rate(ns, seconds: float, threads: int):
    """Oracle FP64 Glynn terms/s on full permanents of the sweep's seed-0 inputs:
    every n of ``ns`` once, then again from the smallest while the total stays
    below ``seconds``."""
    import oracle
    import synthetic as S

    done, spent, runs = 0, 0.0, []
    for n in sorted(ns):
        A = S.gaussian(n, 0)
        t0 = time.perf_counter()
        oracle.glynn_f64dd(A, threads=threads)
        dt = time.perf_counter() - t0
        done += 2 ** (n - 1)
        spent += dt
        runs.append((n, dt))
        if spent > seconds:
            break
    return done / spent, runs, spent


def quad_ryser_times(ns, threads: int):
    """Seconds of the quad-precision Ryser oracle (Eq. (S1), subsets in binary
    order with the row sums of every subset formed afresh, as the paper's
    Algorithm 1 does) on the sweep's seed-0 Gaussian inputs."""
    import oracle
    import synthetic as S

    out = {}
    for n in ns:
        A = S.gaussian(n, 0)
        t0 = time.perf_counter()
        oracle.ryser(A, threads=threads)
        out[str(n)] = time.perf_counter() - t0
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    ns, kinds = workload(args)
    threads = os.cpu_count() or 1
    per_step = max(args.cpu_seconds, 1.0) / 3.0
    import synthetic as S

    mats = {(n, seed): S.gaussian(n, seed) for n in ns for seed in range(3)}

    def one_step(step, sample):
        items = step_items(ns, kinds, step)
        t0 = time.perf_counter()
        done = 0
        for kind, n, seed in items:
            cnt = min(sample, terms_of(kind, n))
            oracle_sample_fn(kind)(mats[(n, seed)], 0, cnt, threads=threads)
            done += cnt
        return done, time.perf_counter() - t0

    # calibrate one bounded sample per item (the first terms in Gray order) so
    # that a step costs about per_step seconds
    sample = 1 << 16
    while True:
        d, t = one_step(0, sample)
        if t > per_step / 4 or sample >= (1 << 40):
            break
        sample *= 2
    sample = max(1, int(sample * per_step / max(t, 1e-6)))

    for w in range(args.warmup):
        one_step(w, sample)
    tot_terms, tot_t = 0, 0.0
    for s in range(args.steps):
        d, t = one_step(s, sample)
        tot_terms += d
        tot_t += t
    value = tot_terms / tot_t
    sample_desc = ("oracle FP64 Gray-order partial sums (double-double accumulation), first %d terms of each "
                   "(method, n) item per step, %d threads" % (sample, threads))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64 (oracle, dd sum)",
        "data": "synthetic", "config": config_dict(args, ns, kinds, 1),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample_desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# the other forms, each against the plain form on the same GPU
# ---------------------------------------------------------------------------
def measure_forms(dev, plain_rate, peak_fp64, large=True):
    """The other forms of the method on the same GPU: precision rungs, the batched
    form (graph replay), the adjoint, photon collisions, row minors and
    boson-sampling draws, each with its parity figure.  A failing section is
    reported as "<name>_error" instead of ending the run."""
    import math

    import numpy as np
    import torch

    import paper_1606_05836_gb300 as pg
    import synthetic as S
    from paper_1606_05836_gb300 import batch as B

    refs = bench_refs()

    def timed(fn, reps=1):
        best = None
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize(dev)
            t = e0.elapsed_time(e1) / 1e3
            best = t if best is None else min(best, t)
        return best

    forms = {}
    ctx = {"base": plain_rate}

    def ladder():
        # precision ladder: rates at n = 32 (Gaussian var 1/n^2), errors at n = 20 vs a stored oracle value
        A32 = torch.as_tensor(S.gaussian(32, 0)).to(dev)
        A20h = S.gaussian(20, 0)
        A20 = torch.as_tensor(A20h).to(dev)
        r20 = refs["glynn_gaussian_n20"]
        rungs = {}
        for prec in ("fp64", "fp64_dd", "fp32p_dd", "fp64_df", "fp32x2"):
            pg.glynn(A32, prec=prec)
            t = timed(lambda: pg.glynn(A32, prec=prec))
            err = ref_rel_err(r20, A20h, complex(pg.glynn(A20, prec=prec).cpu().item()))
            rungs[prec] = {"terms_per_s": 2 ** 31 / t, "vs_plain_glynn": None, "rel_err_n20_vs_oracle": err}
        ctx["base"] = rungs["fp64"]["terms_per_s"]
        for prec, v in rungs.items():
            v["vs_plain_glynn"] = v["terms_per_s"] / ctx["base"]
            forms["glynn_n32_" + prec] = v

    def batched():
        # 4096 output patterns of one Haar 1000 x 1000 unitary, n in 8..24, 20 % collisions
        U = S.haar_unitary(1000, 0)
        ctx["U"] = U
        mats, ns, rows, cols, collide = S.batch_patterns(U, 4096, 8, 24, 1)
        scale = [1.0 / float(np.prod([math.factorial(int(x)) for x in np.bincount(c)])) for c in cols]
        bp = B.BatchedPermanents(mats, method="glynn", scale=scale)
        tuned = bp.autotune(candidates=[(9, 128), (11, 64), (11, 128), (13, 128)], reps=2)
        bp.capture()
        bp.replay()
        t = timed(bp.replay, reps=3)
        terms = int(sum(2 ** (int(n) - 1) for n in ns))
        # sampled parity of the batched kernel: the 8 stored items (n <= 14) of this batch, with their oracle values
        items = refs["batched_items"]
        pick = [unflat(r["matrix"], r["n"], r["n"]) for r in items]

        def sampled_err(prec):
            per8, _ = pg.batched(pick, method="glynn", prec=prec)
            per8 = per8.cpu().numpy()
            return max(ref_rel_err(r, pick[i], complex(per8[i])) for i, r in enumerate(items))

        walked = [walked_terms(A) for A in mats]
        wflops = sum(flops_per_term(int(A.shape[0])) * w for A, w in zip(mats, walked))
        forms["batched_4096_n8-24"] = {"terms_per_s": terms / t, "perms_per_s": len(mats) / t, "s_per_replay": t,
                                       "walked_terms_per_s": sum(walked) / t, "tflops_walked": wflops / t / 1e12,
                                       "frac_of_fp64_peak": wflops / t / peak_fp64,
                                       "vs_plain_glynn": terms / t / ctx["base"],
                                       "collision_items": int(collide.sum()),
                                       "tuned": {"unit_log2": tuned["unit_log2"], "block": tuned["block"]},
                                       "max_rel_err_sampled_vs_oracle": sampled_err("fp64")}
        # the same batch in R3 (FP64 row sums, double-float products) and R4 (double-float walk)
        for prec in ("fp64_df", "fp32x2"):
            # each rung gets its own tuned shape (the autotuner's cache is keyed by precision)
            bpx = B.BatchedPermanents(mats, method="glynn", scale=scale, prec=prec)
            tuned_x = bpx.autotune(candidates=[(9, 128), (11, 64), (11, 128), (13, 128)], reps=2)
            bpx.capture()
            bpx.replay()
            tx = timed(bpx.replay, reps=3)
            forms["batched_4096_n8-24_" + prec] = {"terms_per_s": terms / tx, "perms_per_s": len(mats) / tx,
                                                  "s_per_replay": tx, "vs_fp64_batch": t / tx,
                                                  "tuned": {"unit_log2": tuned_x["unit_log2"],
                                                            "block": tuned_x["block"]},
                                                  "max_rel_err_sampled_vs_oracle": sampled_err(prec)}

    def adjoint():
        # batch of 64 Gaussian matrices at n = 24
        G = torch.as_tensor(np.stack([S.gaussian(24, b) for b in range(64)])).to(dev)
        pg.grad(G[:1])
        tg = timed(lambda: pg.grad(G))
        tf = timed(lambda: [pg.glynn(G[b]) for b in range(64)])
        _, _, M, _ = pg.grad(G[:1])
        A0 = G[0].cpu().numpy()
        P0 = complex(pg.glynn(G[0]).cpu().item())
        lap = float(np.max(np.abs(np.sum(A0 * M[0].cpu().numpy(), axis=1) - P0)) / abs(P0))
        forms["adjoint_64_n24"] = {"terms_per_s": 64 * 2 ** 23 / tg, "s": tg, "cost_vs_plain_same_batch": tg / tf,
                                   "laplace_identity_rel_err": lap}
        # the same batch with the products in double-float (R3)
        pg.grad(G[:1], prec="fp64_df")
        tr3 = timed(lambda: pg.grad(G, prec="fp64_df"))
        _, _, M3, _ = pg.grad(G[:1], prec="fp64_df")
        forms["adjoint_64_n24_fp64_df"] = {
            "terms_per_s": 64 * 2 ** 23 / tr3, "s": tr3, "vs_fp64_adjoint": tg / tr3,
            "minors_normwise_diff_vs_fp64": float(np.max(np.abs(M3[0].cpu().numpy() - M[0].cpu().numpy()))
                                                  / np.max(np.abs(M[0].cpu().numpy())))}
        # the same batch through the autograd Function: |Per|^2 forward, gradient backward
        Gr = G.clone().requires_grad_(True)

        def through_autograd():
            pg.PermAbs2.apply(Gr).sum().backward()

        ta = timed(through_autograd)
        forms["adjoint_64_n24"]["autograd_s"] = ta
        # n = 32, the configured batch of 64 (about 2 minutes; --no-large times 2)
        nb = 64 if large else 2
        G32 = torch.as_tensor(np.stack([S.gaussian(32, b) for b in range(nb)])).to(dev)
        tg32 = timed(lambda: pg.grad(G32))
        tf32 = timed(lambda: [pg.glynn(G32[b]) for b in range(min(nb, 8))]) * nb / min(nb, 8)
        _, _, M32, _ = pg.grad(G32[:1])
        A32 = G32[0].cpu().numpy()
        P32 = complex(pg.glynn(G32[0]).cpu().item())
        lap32 = float(np.max(np.abs(np.sum(A32 * M32[0].cpu().numpy(), axis=1) - P32)) / abs(P32))
        forms["adjoint_%d_n32" % nb] = {"terms_per_s": nb * 2 ** 31 / tg32, "s": tg32,
                                        "cost_vs_plain_same_batch": tg32 / tf32,
                                        "laplace_identity_rel_err": lap32}

    def collisions():
        # n = 28: the multiplicity expansion against the plain kernel on the expanded matrix
        coll = {}
        for mult in ([2, 1, 1, 1], [2, 2, 2, 1], [3, 2, 2, 2, 2, 1]):
            mult = mult + [1] * (28 - sum(mult))
            Bh = S.circular_gaussian((28, len(mult)), 2800 + len(mult), 1.0 / 28)
            dB = torch.as_tensor(Bh).to(dev)
            dE = torch.as_tensor(np.ascontiguousarray(np.repeat(Bh, mult, axis=1))).to(dev)
            pg.glynn_mult(dB, mult)
            tm = timed(lambda: pg.glynn_mult(dB, mult), reps=2)
            tp = timed(lambda: pg.glynn(dE), reps=2)
            a, b = complex(pg.glynn_mult(dB, mult).cpu().item()), complex(pg.glynn(dE).cpu().item())
            key = "+".join(str(m) for m in mult if m > 1)
            coll[key] = {"s": tm, "speedup_vs_expanded": tp / tm, "rel_diff_vs_expanded": abs(a - b) / abs(b)}
        forms["collisions_n28"] = coll

    def minors():
        # row minors of a 31 x 32 matrix in one pass, against the forward kernel at n = 32
        M32 = torch.as_tensor(S.circular_gaussian((31, 32), 0, 1.0 / 32)).to(dev)
        for rp in ("fp64", "fp64_df", "fp32x2"):
            pg.row_minors(M32, prec=rp)
            tmr = timed(lambda: pg.row_minors(M32, prec=rp))
            key = "row_minors_k32" + ("" if rp == "fp64" else "_" + rp)
            forms[key] = {"terms_per_s": 2 ** 31 / tmr, "s": tmr, "cost_vs_glynn_n32": tmr * ctx["base"] / 2 ** 31}

    def sampler():
        # 16 draws of 24 photons in the 1000-mode unitary (one graph replay per batch)
        U = ctx["U"] if "U" in ctx else S.haar_unitary(1000, 0)
        n, ns = 24, 16
        A24 = torch.as_tensor(S.gaussian(24, 0)).to(dev)
        pg.glynn(A24)
        t24 = timed(lambda: pg.glynn(A24), reps=2)
        # sampled parity: 4 draws of 8 photons in 30 modes against the oracle's stored draws
        rs = refs["sampler_m30_n8"]
        U30 = unflat(rs["U"], 30, 30)
        for rp in ("fp64", "fp64_df", "fp32x2"):
            smp, _, _ = sampler_case(pg, U, n, ns, 5, dev, prec=rp)
            smp.capture()
            smp.replay()
            ts = timed(smp.replay, reps=2)
            s30, _, _ = sampler_case(pg, U30, 8, 4, 6, dev, prec=rp)
            got = s30.run().cpu().numpy()
            same = "%d/4" % sum(int(list(got[i]) == rs["draws"][i]) for i in range(4))
            key = "boson_sample_m1000_n24_x16" + ("" if rp == "fp64" else "_" + rp)
            forms[key] = {"draws_per_s": ns / ts, "s_per_replay": ts, "terms_per_s": ns * (2 ** n - 2) / ts,
                          "cost_per_draw_in_glynn_n24": ts / ns / t24, "launches_per_replay": 2 * n - 1,
                          "draws_equal_oracle_m30_n8": same}

    def single_sizes():
        # one FP64 Glynn permanent per launch across the metric's n = 20-40 (the
        # sweep's seed-0 Gaussian inputs), each against a stored oracle value; the
        # error is that of the timed launch's own result (a second n = 40 pass
        # would cost minutes)
        for n in ([20, 36, 40] if large else [20]):
            Ah = S.gaussian(n, 0)
            dA = torch.as_tensor(Ah).to(dev)
            held = {}

            def run():
                held["out"] = pg.glynn(dA)

            if n == 20:
                ref = refs["glynn_gaussian_n20"]
                run()
                reps = 50
                t = timed(lambda: [run() for _ in range(reps)]) / reps
                src = "quad Glynn (bench_refs.json)"
            else:
                r = large_ref("gaussian", n, 0)
                ref = {"sha": r[0], "value": list(r[1])} if r else None
                pg.glynn_range(dA, 0, 1 << 16)  # loads the n-sized kernel without a full pass
                t = timed(run)
                src = "FP64 + double-double Glynn (large_refs.tsv)"
            got = complex(held["out"].cpu().item())
            fl = flops_per_term(n) * 2 ** (n - 1) / t
            forms["glynn_single_n%d" % n] = {
                "terms_per_s": 2 ** (n - 1) / t, "s": t, "tflops": fl / 1e12, "frac_of_fp64_peak": fl / peak_fp64,
                "rel_err_vs_oracle": ref_rel_err(ref, Ah, got) if ref else None, "oracle": src}

    for name, fn in (("glynn_n32", ladder), ("batched_4096_n8-24", batched), ("adjoint", adjoint),
                     ("collisions_n28", collisions), ("row_minors_k32", minors),
                     ("boson_sample_m1000_n24_x16", sampler), ("glynn_single", single_sizes)):
        try:
            fn()
        except Exception as e:  # one form failing must not take the bench line down
            forms[name + "_error"] = "%s: %s" % (type(e).__name__, e)
    return forms


def walked_terms(A) -> int:
    """Gray indices the batched Glynn walk visits for matrix A: 2^(n-1), or with
    repeated columns the multiplicity expansion's classes x 2^free (the delta = +1
    copy taken from a singleton column if there is one, else from the smallest
    group)."""
    import numpy as np

    n = A.shape[0]
    _, counts = np.unique(np.ascontiguousarray(A.T).view(np.complex128).reshape(n, n), axis=0,
                          return_counts=True)
    counts = sorted(int(c) for c in counts)
    if max(counts) == 1:
        return 2 ** (n - 1)
    singles = counts.count(1)
    groups = [c for c in counts if c > 1]
    classes = 1
    if singles:
        for m in groups:
            classes *= m + 1
        return classes * 2 ** (singles - 1)
    smallest = groups[0]
    classes = smallest
    for m in groups[1:]:
        classes *= m + 1
    return classes


def bench_refs():
    """Oracle values for the forms' parity figures, written by tests/golden/make_bench_refs.py."""
    with open(os.path.join(ROOT, "tests", "golden", "bench_refs.json")) as f:
        return json.load(f)


def input_digest(A) -> str:
    import hashlib

    import numpy as np
    return hashlib.sha256(np.ascontiguousarray(A).tobytes()).hexdigest()[:16]


def unflat(v, rows: int, cols: int):
    import numpy as np
    return np.asarray(v, dtype=np.float64).view(np.complex128).reshape(rows, cols)


def ref_rel_err(ref, A, got: complex):
    """|got - P| / |P| against a stored oracle value; None if the input was not regenerated bit for bit."""
    if ref["sha"] != input_digest(A):
        return None
    rh, rl, ih, il = ref["value"]
    d = complex((got.real - rh) - rl, (got.imag - ih) - il)
    return abs(d) / abs(complex(rh + rl, ih + il))


def sampler_case(pg, U, n, ns, seed, dev, prec="fp64"):
    """A BosonSampler on U (numpy) with photons in modes 0..n-1 and seeded draws loaded."""
    import torch

    import synthetic as S

    alpha, uu = S.sampler_draws(n, ns, seed)
    smp = pg.BosonSampler(torch.as_tensor(U).to(dev), list(range(n)), ns, prec=prec)
    smp.load(torch.as_tensor(alpha).to(dev), torch.as_tensor(uu).to(dev))
    return smp, alpha, uu


def ryser_pass(ryser, dmat, ns, flush, stream, prec):
    """FP64 Ryser on the sweep's inputs (every n, seeds 0-2; 2^n terms each), one
    launch per matrix timed with CUDA events after an L2 flush, and the error of
    its n = max results against the stored quad-oracle values."""
    import torch

    nmax = max(ns)
    per_kind = {"ryser": [0, 0.0]}
    results = {}
    for n in ns:
        ryser(dmat[(n, 0)], prec=prec)
        for seed in range(3):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            out = ryser(dmat[(n, seed)], prec=prec)
            b.record(stream)
            torch.cuda.synchronize()
            per_kind["ryser"][0] += 2 ** n
            per_kind["ryser"][1] += a.elapsed_time(b)
            results[("ryser", n, seed)] = out
    r = method_rates(per_kind, results, nmax)["ryser"]
    r["timed"] = "one launch per (n, seed), n = %s, seeds 0-2, outside the timed sweep" % ",".join(map(str, ns))
    return r


def fp64_peak(dev, gpu_index: int, sms: int):
    """FP64 peak measured on this GPU: the DFMA probe (perm_fp64_fma_probe, 4 x SMs
    blocks of 256 threads, 4 independent FMA chains per thread), best of 8
    launches timed with CUDA events, SM clocks sampled meanwhile.  None if the
    probe fails (the derived peak is used then)."""
    import torch

    import paper_1606_05836_gb300 as pg

    grid, block, iters = 4 * sms, 256, 1 << 16
    try:
        pg.fp64_fma_probe(256, grid, block, dev)
        torch.cuda.synchronize(dev)
        clk = ClockSampler(gpu_index)
        clk.start()
        best, fmas = None, 0
        for _ in range(8):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fmas = pg.fp64_fma_probe(iters, grid, block, dev)
            e1.record()
            torch.cuda.synchronize(dev)
            t = e0.elapsed_time(e1) / 1e3
            best = t if best is None else min(best, t)
        c = clk.stop()
    except Exception:  # the probe is a diagnostic: fall back to the derived peak
        return None
    return {"flops_per_s": 2.0 * fmas / best, "dfma_per_s": fmas / best, "s_per_launch": best,
            "grid": grid, "block": block, "iters": iters, "chains": 4,
            "sm_mhz": c["sm_mhz"] if c else None, "reasons": c["reasons"] if c else None}


def sweep_refs():
    """{(n, seed): (sha, (re_hi, re_lo, im_hi, im_lo))} of the quad-oracle values of
    the sweep's inputs (tests/golden/sweep_refs.tsv, written by make_sweep_refs.py)."""
    out = {}
    path = os.path.join(ROOT, "tests", "golden", "sweep_refs.tsv")
    with open(path) as f:
        for line in f:
            p = line.rstrip("\n").split("\t")
            if not p[0].isdigit() or p[7] != "glynn_gray":
                continue
            out[(int(p[0]), int(p[1]))] = (p[2], tuple(float(x) for x in p[3:7]))
    return out


def large_ref(kind: str, n: int, seed: int):
    """(sha, (re_hi, re_lo, im_hi, im_lo)) of tests/golden/large_refs.tsv (FP64 /
    double-double oracle, make_large_refs.py), or None if not stored."""
    path = os.path.join(ROOT, "tests", "golden", "large_refs.tsv")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        for line in f:
            p = line.rstrip("\n").split("\t")
            if len(p) >= 8 and p[0] == kind and p[1] == str(n) and p[2] == str(seed):
                return p[3], tuple(float(x) for x in p[4:8])
    return None


def method_rates(per_kind, results, nmax: int):
    """Glynn and Ryser apart: terms/s over all their timed launches, and the error
    of their timed n = nmax results against the stored quad-oracle values."""
    import synthetic as S

    refs = sweep_refs()
    bars = {"glynn": "1e-10 (FP64 Glynn)",
            "ryser": "none: FP64 Ryser loses digits to cancellation (the paper's finding; stated ~1e-6 at n = 32)"}
    out = {}
    for kind, (terms, ms) in per_kind.items():
        errs = {}
        for (k, n, seed), t in results.items():
            if k != kind or n != nmax or (n, seed) not in refs:
                continue
            sha, v = refs[(n, seed)]
            e = ref_rel_err({"sha": sha, "value": list(v)}, S.gaussian(n, seed), complex(t.cpu().item()))
            if e is not None:
                errs["n%d_seed%d" % (n, seed)] = e
        out[kind] = {"terms_per_s": terms / (ms / 1e3) if ms > 0 else None, "launches_ms": ms,
                     "rel_err_vs_quad_oracle": errs, "max_rel_err": max(errs.values()) if errs else None,
                     "bar": bars.get(kind)}
    return out


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch

    import paper_1606_05836_gb300 as pg
    import synthetic as S

    rank, world, local = dist_env()
    if world != args.gpus:
        raise SystemExit("--gpus %d but WORLD_SIZE=%d" % (args.gpus, world))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    pg.library()
    ns, kinds = workload(args)
    fn = {"glynn": pg.glynn, "ryser": pg.ryser}
    host = {(n, seed): S.gaussian(n, seed) for n in ns for seed in range(3)}
    dmat = {key: torch.as_tensor(a).to(dev) for key, a in host.items()}
    pinned = {key: torch.as_tensor(a).pin_memory() for key, a in host.items()}
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    nmax = max(ns)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        if world == 1:
            return x
        import torch.distributed as dist
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    # warm-up (also compiles nothing: the library is prebuilt; first calls set attributes)
    for w in range(args.warmup):
        for kind, n, seed in step_items(ns, kinds, w):
            fn[kind](dmat[(n, seed)], prec=args.prec)
    torch.cuda.synchronize(dev)

    # ---- device-timed steps ----
    sampler = ClockSampler(local) if rank == 0 else None
    barrier()
    torch.cuda.synchronize(dev)
    if sampler:
        sampler.start()
    step_ms = []
    dom = []  # (flops, ms) of the dominant kernel's launches
    per_kind = {k: [0, 0.0] for k in kinds}  # terms, ms of every launch of the method
    results = {}  # (kind, n, seed) -> the permanent the timed launch returned
    terms_total = 0
    launches = 0
    for s in range(args.steps):
        flush.zero_()
        items = step_items(ns, kinds, s)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in items]
        outs = []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for (kind, n, seed), (a, b) in zip(items, ev):
            a.record(stream)
            outs.append(fn[kind](dmat[(n, seed)], prec=args.prec))
            b.record(stream)
            terms_total += terms_of(kind, n)
            launches += 1
        e1.record(stream)
        torch.cuda.synchronize(dev)
        step_ms.append(e0.elapsed_time(e1))
        for (kind, n, seed), (a, b), out in zip(items, ev, outs):
            ms = a.elapsed_time(b)
            per_kind[kind][0] += terms_of(kind, n)
            per_kind[kind][1] += ms
            results[(kind, n, seed)] = out
            if n == nmax:
                dom.append((flops_per_term(n) * terms_of(kind, n), ms))
    torch.cuda.synchronize(dev)
    clocks = sampler.stop() if sampler else None
    t_dev = max_over_ranks(sum(step_ms) / 1e3)
    barrier()

    # ---- end-to-end steps: pinned host -> device, compute, result -> host ----
    e2e = None
    if not args.no_e2e:
        out_host = torch.empty(1, dtype=torch.complex128).pin_memory()
        h2d = d2h = 0
        e2e_ms = []
        e2e_terms = 0
        barrier()
        torch.cuda.synchronize(dev)
        for s in range(args.steps):
            flush.zero_()
            items = step_items(ns, kinds, s)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h2d = d2h = 0
            for kind, n, seed in items:
                src = pinned[(n, seed)]
                dA = src.to(dev, non_blocking=True)
                r = fn[kind](dA, prec=args.prec)
                out_host.copy_(r.reshape(1), non_blocking=True)
                h2d += src.numel() * src.element_size()
                d2h += out_host.numel() * out_host.element_size()
                e2e_terms += terms_of(kind, n)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            e2e_ms.append(e0.elapsed_time(e1))
        t_e2e = max_over_ranks(sum(e2e_ms) / 1e3)
        e2e = {"value": world * e2e_terms / t_e2e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    if rank != 0:
        return 0

    value = world * terms_total / t_dev
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except (OSError, ValueError):
        pass
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    sm_max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    # GB300: 2 FP64 FMA lanes per clock per SM (0.5 per sub-partition) = 4 flop/clk/SM
    peak_derived = sms * 4 * sm_max_mhz * 1e6
    probe = fp64_peak(dev, local, sms)
    peak_fp64 = probe["flops_per_s"] if probe else peak_derived
    achieved = sum(f for f, _ in dom) / (sum(ms for _, ms in dom) / 1e3) if dom else None
    traffic = measured_traffic(nmax)
    roofline = {
        "bound": "alu", "pipe": "fp64",
        "kernel": "fwd_kernel<N=%d> (%s, %s)" % (nmax, "+".join(kinds), args.prec),
        "achieved": achieved / 1e12 if achieved else None, "peak": peak_fp64 / 1e12, "unit": "TFLOP/s",
        "frac": (achieved / peak_fp64) if achieved else None,
        "peak_source": ("measured: FP64 FMA probe (perm_fp64_fma_probe), %.0f MHz median SM clock during it"
                        % probe["sm_mhz"] if probe else
                        "derived: %d SMs x 4 FP64 flop/clk/SM x %.0f MHz" % (sms, sm_max_mhz)),
        "peak_derived": peak_derived / 1e12,
        "frac_of_derived": (achieved / peak_derived) if achieved else None,
        "peak_probe": probe,
        "flops_per_term": "8n-4 (2n update + 6(n-1) product + 2 accumulate)",
        "traffic": traffic,
    }
    by_method = method_rates(per_kind, results, nmax)
    if "ryser" not in kinds and not args.no_forms:
        by_method["ryser"] = ryser_pass(fn["ryser"], dmat, ns, flush, stream, args.prec)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        rate, runs, dt = oracle_full_rate([20, 24, 28, 32], args.cpu_seconds, threads)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "oracle FP64 Gray-order Glynn with double-double accumulation (glynn_f64dd), full "
                         "permanents of the sweep's seed-0 Gaussian inputs at n = %s, %.1f s on %d threads"
                         % (",".join(str(n) for n, _ in runs), dt, threads),
               "per_n_terms_per_s": {str(n): 2 ** (n - 1) / t for n, t in runs}}
        nlast, tlast = runs[-1]
        cpu["extrapolated_s_per_permanent"] = {
            str(n): tlast * 2.0 ** (n - nlast) for n in (36, 40) if n > nlast}
        cpu["extrapolated_note"] = "x2 per +1 in n from the n = %d time (not measured)" % nlast
        cpu["quad_ryser_s"] = quad_ryser_times([20, 22], threads)
    forms = None
    if world == 1 and not args.no_forms:
        forms = measure_forms(dev, value, peak_fp64, not args.no_large)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sum(step_ms) / len(step_ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.prec != "fp32p_dd" else "f64+f32",
        "data": "synthetic", "config": config_dict(args, ns, kinds, world), "roofline": roofline,
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks, "by_method": by_method,
        "forms": forms,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_single_form(args):
    """Time one form on its own (used for profiling runs); prints its JSON line."""
    import numpy as np
    import torch

    import paper_1606_05836_gb300 as pg
    import synthetic as S

    dev = torch.device("cuda", 0)
    if args.form == "range":
        n, L = args.range_n, args.range_log2
        dA = torch.as_tensor(S.gaussian(n, 0)).to(dev)
        for _ in range(args.warmup):
            pg.glynn_range(dA, 0, 1 << 12)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            pg.glynn_range(dA, 0, 1 << L)
        e1.record()
        torch.cuda.synchronize(dev)
        t = e0.elapsed_time(e1) / 1e3 / max(args.steps, 1)
        print(json.dumps({"form": "range", "n": n, "terms": 1 << L, "steps": args.steps, "s": t,
                          "terms_per_s": (1 << L) / t, "tflops": (8 * n - 4) * (1 << L) / t / 1e12}), flush=True)
    elif args.form == "sampler":
        m, n, ns = args.sampler_m, args.sampler_n, args.sampler_count
        smp, _, _ = sampler_case(pg, S.haar_unitary(m, 0), n, ns, 5, dev)
        for _ in range(args.warmup):
            smp.run()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            smp.run()
        e1.record()
        torch.cuda.synchronize(dev)
        t = e0.elapsed_time(e1) / 1e3
        print(json.dumps({"form": "sampler", "m": m, "n": n, "count": ns, "steps": args.steps,
                          "draws_per_s": args.steps * ns / t}), flush=True)
    elif args.form == "adjoint":
        n, b = args.adjoint_n, args.adjoint_batch
        G = torch.as_tensor(np.stack([S.gaussian(n, i) for i in range(b)])).to(dev)
        for _ in range(args.warmup):
            pg.grad(G[:1], prec=args.adjoint_prec)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            pg.grad(G, prec=args.adjoint_prec)
        e1.record()
        torch.cuda.synchronize(dev)
        t = e0.elapsed_time(e1) / 1e3
        print(json.dumps({"form": "adjoint", "n": n, "batch": b, "steps": args.steps, "prec": args.adjoint_prec,
                          "terms_per_s": args.steps * b * 2 ** (n - 1) / t}), flush=True)
    else:
        import math

        from paper_1606_05836_gb300 import batch as B
        U = S.haar_unitary(1000, 0)
        mats, ns, rows, cols, collide = S.batch_patterns(U, args.batched_count, 8, 24, 1)
        scale = [1.0 / float(np.prod([math.factorial(int(x)) for x in np.bincount(c)])) for c in cols]
        bp = B.BatchedPermanents(mats, method="glynn", scale=scale)
        for _ in range(args.warmup):
            bp.run()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            bp.run()
        e1.record()
        torch.cuda.synchronize(dev)
        t = e0.elapsed_time(e1) / 1e3
        terms = int(sum(2 ** (int(n) - 1) for n in ns))
        print(json.dumps({"form": "batched", "count": len(mats), "steps": args.steps,
                          "terms_per_s": args.steps * terms / t}), flush=True)
    return 0


def run_shard(args):
    """One Glynn permanent (the sweep's seed-0 Gaussian input of size --shard-n)
    split over the ranks as Algorithm 2 splits its iteration range: each rank one
    contiguous Gray range on its own GPU (perm_glynn_range), then one all-gather of
    the 32-byte partials and perm_combine_partials on every rank.  Timed from a
    barrier to the combined result on every rank (max over ranks); prints one JSON
    line on rank 0 with the rate and the error against the stored oracle value."""
    import torch

    import paper_1606_05836_gb300 as pg  # noqa: F401  (loads the library)
    import synthetic as S
    from paper_1606_05836_gb300 import shard

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    n = args.shard_n
    Ah = S.gaussian(n, 0)
    dA = torch.as_tensor(Ah).to(dev)
    fn = shard.gpu_partial_fn(dA, "glynn")
    fn(0, 1 << 12)  # loads the kernel
    times, per = [], None
    for _ in range(max(1, args.steps)):
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        per = shard.sharded_permanent(n, "glynn", fn, rank, world)
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        if world > 1:
            t = torch.tensor([dt], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t.item())
        times.append(dt)
    if rank == 0:
        r = large_ref("gaussian", n, 0)
        err = ref_rel_err({"sha": r[0], "value": list(r[1])}, Ah, per) if r else None
        t = min(times)
        print(json.dumps({"form": "shard", "n": n, "n_gpus": world, "steps": len(times), "s": t,
                          "terms_per_s": 2 ** (n - 1) / t, "exchange": "all-gather of 32-byte partials" if world > 1
                          else "none (one rank)", "rel_err_vs_oracle": err, "scaling": "strong"}), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.form == "shard":
        return run_shard(args)
    if args.form != "sweep":
        return run_single_form(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
