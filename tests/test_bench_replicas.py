"""The multi-GPU path of bench.py: independent replicas, one per rank, whose
timings are combined on the host (max over ranks, units of all ranks).  Run
here as two gloo ranks on the CPU; no GPU and no data-path collective."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_RANK_PROG = r"""
import json, os, sys
sys.path.insert(0, os.environ["TT_ROOT"])
import torch.distributed as dist
import bench
world, rank, local = bench.dist_setup()
dist.init_process_group("gloo")
# rank r took (r + 1) seconds for its 5 steps: the job's time is the slowest
value, tmax = bench.job_throughput(world, 5, float(rank + 1), dist, "cpu")
m = bench.max_over_ranks(-3.0 * rank, dist, "cpu")
dist.barrier()
dist.destroy_process_group()
print(json.dumps({"rank": rank, "world": world, "local": local, "value": value, "tmax": tmax, "m": m}))
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _launch(world, argv, timeout=120):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, WORLD_SIZE=str(world), RANK=str(r), LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), TT_ROOT=ROOT, CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen(argv, env=env, cwd=ROOT, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                      text=True))
    outs = []
    try:
        for p in procs:
            o, e = p.communicate(timeout=timeout)
            outs.append((p.returncode, o, e))
    finally:
        for p in procs:
            if p.poll() is None:
                p.kill()
    return outs


def test_dist_setup_defaults(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_setup() == (1, 0, 0)
    assert bench.max_over_ranks(2.5) == 2.5
    assert bench.job_throughput(1, 10, 2.0) == (5.0, 2.0)


def test_two_gloo_ranks_take_the_slowest_replica():
    pytest.importorskip("torch.distributed")
    outs = _launch(2, [sys.executable, "-c", _RANK_PROG])
    res = []
    for rc, o, e in outs:
        assert rc == 0, e[-2000:]
        res.append(json.loads(o.strip().splitlines()[-1]))
    for r in res:
        assert r["world"] == 2 and r["local"] == r["rank"]
        # max over ranks on every rank; units of both ranks over that time
        assert r["tmax"] == 2.0
        assert r["value"] == pytest.approx(2 * 5 / 2.0)
        assert r["m"] == 0.0


def test_reference_arm_runs_on_rank_zero_only():
    # rank 1 of a two-rank launch exits at once with no output (no process
    # group is needed: the reference arm has no collective)
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1", CUDA_VISIBLE_DEVICES="")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=120)
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""
