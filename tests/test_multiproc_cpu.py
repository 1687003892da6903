"""The multi-rank path of the benchmark on CPU (gloo, world size 2): every
rank runs its own replica of the frame, the job's time is the slowest rank's
(max over ranks), the whole-job rate counts every rank's frames, and only
rank 0 runs the oracle's reference arm."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, os.environ["LS_ROOT"])
import bench
ws, rank, local = bench.dist_setup(None, backend="gloo")
# rank r pretends its timed steps took 10 + 5 r ms in total
slowest = bench.max_over_ranks(10.0 + 5.0 * rank, ws, device="cpu")
bench.barrier(ws)
print(json.dumps({"rank": rank, "ws": ws, "slowest": slowest, "rate": bench.job_rate(ws, slowest)}), flush=True)
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run_ranks(code, ws=2, extra_env=None, timeout=120):
    port = _free_port()
    procs = []
    for r in range(ws):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(ws), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), LS_ROOT=ROOT, CUDA_VISIBLE_DEVICES="")
        env.update(extra_env or {})
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=timeout)
        except subprocess.TimeoutExpired:
            p.kill()
            raise
        assert p.returncode == 0, e
        outs.append(o)
    return outs


def test_slowest_rank_sets_the_job_time_and_rates_add_up():
    outs = _run_ranks(WORKER)
    lines = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    assert sorted(l["rank"] for l in lines) == [0, 1]
    for l in lines:
        assert l["ws"] == 2
        assert l["slowest"] == 15.0  # max over ranks, seen by every rank
        assert l["rate"] == pytest.approx(2 * 1e3 / 15.0)


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    env = {k: os.environ.pop(k) for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK") if k in os.environ}
    try:
        assert bench.dist_setup(None, backend="gloo") == (1, 0, 0)
        assert bench.max_over_ranks(7.5, 1) == 7.5
        assert bench.job_rate(1, 2.0) == 500.0
    finally:
        os.environ.update(env)


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the other ranks exit at once without output."""
    code = ("import os, sys; sys.path.insert(0, os.environ['LS_ROOT']); import bench, argparse; "
            "a = argparse.Namespace(steps=1, warmup=0); sys.exit(bench.run_reference(a))")
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", LS_ROOT=ROOT)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
