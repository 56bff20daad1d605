"""The multi-process path of bench.py on CPU: two gloo ranks (one process per
GPU on a GPU machine, where the backend is NCCL).  Every rank runs its own product
(weak scaling, no collective on the data path); the job's step time is the
slowest rank's, the whole-job value counts every rank's work, and only rank 0
prints (the reference arm's other ranks exit without work)."""
import io
import multiprocessing as mp
import os
import socket
import sys
import argparse
import contextlib

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, _ = bench._init_dist()
    assert bench._backend() == "gloo"
    ms = bench._max_over_ranks(10.0 + 3.0 * r, w)          # rank 1 is the slow one
    bench._barrier(w)
    value = bench._job_value(2.0e12, ms, w)
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        args = argparse.Namespace(steps=1, warmup=0, gpus=w, ref_sample=64, shape="", dtype="bf16")
        rc = bench.run_reference(args) if r != 0 else 0    # rank 0 would run the oracle: skipped here
    q.put((r, w, ms, value, rc, out.getvalue()))
    dist.destroy_process_group()


def test_two_rank_timing_and_output():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, ms, value, rc, printed in res:
        assert w == 2
        assert ms == pytest.approx(13.0)                     # max over ranks
        assert value == pytest.approx(2 * 2.0e12 / 13.0e-3 / 1e12)
        if r == 1:
            assert rc == 0 and printed == ""                 # non-zero ranks print nothing


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._max_over_ranks(4.5, 1) == 4.5
    assert bench._job_value(1e12, 1.0, 1) == pytest.approx(1000.0)


def test_reference_arm_prints_the_contract_line():
    # the reference arm (the FP64 oracle on the host cores) on a tiny sample of the
    # square workload: one JSON line with the keys the measurement contract names
    import json
    sys.path.insert(0, ROOT)
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        os.environ.pop(k, None)
    out = io.StringIO()
    args = argparse.Namespace(steps=1, warmup=0, gpus=1, ref_sample=8, shape="", dtype="bf16")
    with contextlib.redirect_stdout(out):
        assert bench.run_reference(args) == 0
    lines = [l for l in out.getvalue().splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"].startswith("square") and d["config"]["m"] == 16384
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
