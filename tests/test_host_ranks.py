"""CPU tests of the multi-rank host logic of bench.py (world_size 2, gloo).

Under torchrun every rank runs an independent replica of the scene path (the
method has no exchange step between scenes), so the only cross-rank work is
the timing: the job's time is the slowest rank's, and the whole-job rate
counts every rank's scenes.  These tests run that reduction as two gloo
ranks on the host, check that the reference arm does no work on ranks
other than 0, and check the JSON line the reference arm prints.
"""
import os
import socket
import subprocess
import sys
import types

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_RANK_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, os.environ["TEST_ROOT"])
import torch.distributed as dist
import bench
rank = int(os.environ["RANK"])
world = int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", rank=rank, world_size=world)
mine = [0.25, 0.75][rank]            # this rank's timed seconds
slowest = bench.max_over_ranks(mine, dist)
steps = 10
out = {"rank": rank, "slowest": slowest, "rate": bench.whole_job_rate(world, steps, slowest)}
dist.barrier()
dist.destroy_process_group()
print(json.dumps(out), flush=True)
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_single_rank_reduction_is_the_identity():
    assert bench.max_over_ranks(1.5) == 1.5
    assert bench.whole_job_rate(1, 200, 0.25) == 800.0


def test_two_gloo_ranks_take_the_slowest_time_and_count_both_replicas():
    import json

    pytest.importorskip("torch.distributed")
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), TEST_ROOT=ROOT, CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", _RANK_SCRIPT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=120)
        except subprocess.TimeoutExpired:
            for q in procs:
                q.kill()
            raise
        assert p.returncode == 0, e
        outs.append(json.loads(o.strip().splitlines()[-1]))
    assert sorted(o["rank"] for o in outs) == [0, 1]
    for o in outs:
        # both ranks see the slower replica's time, and the job's rate is
        # 2 ranks x 10 scenes over it
        assert o["slowest"] == 0.75
        assert o["rate"] == pytest.approx(2 * 10 / 0.75, rel=0, abs=1e-12)


def test_reference_arm_runs_on_rank_0_only(capsys):
    args = types.SimpleNamespace(steps=1, warmup=0, gpus=2)
    bench.run_reference(args, rank=1)  # returns before any oracle work
    assert capsys.readouterr().out == ""


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` times the FP64 oracle on the host cores
    (one full plume scene per step) and prints one JSON line whose metric,
    unit and direction are the GPU arm's, with its own CPU-baseline record
    and an end-to-end record that moves no bytes to or from a device."""
    import json

    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT,
                       env=dict(os.environ, CUDA_VISIBLE_DEVICES=""))
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["unit"] == "scenes/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["steps"] == 1 and d["warmup"] == 0 and d["dtype"] == "f64" and d["data"] == "synthetic"
    assert d["config"]["workload"] == bench.WORKLOAD
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
