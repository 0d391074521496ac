"""Checkpointed long runs: interruption and resume, several ranks' logs, a torn
last line, and logs of another problem rejected.  The partials come from the
oracle on the CPU (and from the GPU range kernel in the gpu test)."""
import json

import pytest

import oracle
import synthetic as S
from paper_1606_05836_gb300 import longrun


def oracle_partial(A, method):
    f = oracle.glynn_range if method == "glynn" else oracle.ryser_range

    def fn(kb, ke):
        r = f(A, kb, ke, gray=True, threads=2)
        return r.hi, r.lo

    return fn


@pytest.mark.parametrize("method", ["glynn", "ryser"])
def test_interrupt_and_resume(tmp_path, method):
    A = S.gaussian(11, 3)
    log = str(tmp_path / "run.jsonl")
    fn = oracle_partial(A, method)
    total = longrun.n_chunks(11, method, 6)
    assert longrun.run(A, log, fn, method=method, chunk_log2=6, max_chunks=3) == 3
    assert longrun.combine(A, [log], method=method, chunk_log2=6) is None  # incomplete
    assert longrun.run(A, log, fn, method=method, chunk_log2=6) == total - 3  # resumes, skips done chunks
    assert longrun.run(A, log, fn, method=method, chunk_log2=6) == 0
    per = longrun.combine(A, [log], method=method, chunk_log2=6)
    assert oracle.ryser(A).rel_err(per) < 1e-13


def test_two_ranks_and_torn_line(tmp_path):
    A = S.gaussian(12, 4)
    logs = [str(tmp_path / ("r%d.jsonl" % r)) for r in range(2)]
    fn = oracle_partial(A, "glynn")
    for r in range(2):
        longrun.run(A, logs[r], fn, chunk_log2=5, rank=r, world=2)
    with open(logs[1], "a") as f:
        f.write('{"key": "truncated')  # an interrupted write
    per = longrun.combine(A, logs, chunk_log2=5)
    assert oracle.ryser(A).rel_err(per) < 1e-13


@pytest.mark.parametrize("method", ["glynn", "ryser"])
def test_resume_after_torn_write(tmp_path, method):
    """An interrupted run leaves a torn record at the end of its log; the resumed
    run recomputes only that chunk and the ones never started, appends parsable
    records after the fragment, and the combined result matches the oracle."""
    A = S.gaussian(11, 8)
    log = str(tmp_path / "run.jsonl")
    calls = []

    def fn(kb, ke):
        calls.append((kb, ke))
        return oracle_partial(A, method)(kb, ke)

    total = longrun.n_chunks(11, method, 6)
    assert longrun.run(A, log, fn, method=method, chunk_log2=6, max_chunks=3) == 3
    with open(log) as f:
        lines = f.read().splitlines()
    # the third record was cut short by the interruption
    with open(log, "w") as f:
        f.write("\n".join(lines[:2]) + "\n" + lines[2][:25])
    calls.clear()
    assert longrun.run(A, log, fn, method=method, chunk_log2=6) == total - 2
    assert len(calls) == len(set(calls)) == total - 2  # no chunk computed twice
    assert longrun.run(A, log, fn, method=method, chunk_log2=6) == 0
    per = longrun.combine(A, [log], method=method, chunk_log2=6)
    assert per is not None and oracle.ryser(A).rel_err(per) < 1e-13


def test_log_of_another_problem_is_rejected(tmp_path):
    A, B = S.gaussian(9, 5), S.gaussian(9, 6)
    log = str(tmp_path / "run.jsonl")
    longrun.run(A, log, oracle_partial(A, "glynn"), chunk_log2=4, max_chunks=1)
    with pytest.raises(ValueError):
        longrun.run(B, log, oracle_partial(B, "glynn"), chunk_log2=4)
    rec = json.loads(open(log).readline())
    assert rec["k_end"] - rec["k_begin"] == 16


@pytest.mark.gpu
def test_gpu_checkpointed_run_matches_single_launch(tmp_path):
    import torch
    import paper_1606_05836_gb300 as pg
    A = S.gaussian(26, 7)
    log = str(tmp_path / "gpu.jsonl")
    longrun.gpu_run(A, log, chunk_log2=20, max_chunks=5)
    longrun.gpu_run(A, log, chunk_log2=20)
    per = longrun.combine(A, [log], chunk_log2=20)
    single = complex(pg.glynn(torch.as_tensor(A).cuda()).cpu().item())
    assert abs(per - single) <= 1e-12 * abs(single)
