"""Host logic of bench.py on CPU: with two gloo ranks, replicas draw distinct problems,
the job time is the slowest rank's and the reference arm runs on rank 0 only; and the
roofline object's fields and arithmetic."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
rank = int(os.environ["RANK"]); world = int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo")
mine = [120.0, 300.0][rank]
mx = bench.max_over_ranks(mine, dist)
ms, val = bench.job_seconds_per_solve(mx, 3, world)
p = bench._workload(300, rank)
dist.barrier()
print(json.dumps({"rank": rank, "max": mx, "ms": ms, "val": val, "x0": float(p.X[0, 0])}))
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_take_the_slowest_replica(tmp_path):
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER, ROOT], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for pr in procs:
        o, e = pr.communicate(timeout=120)
        assert pr.returncode == 0, e
        outs.append(json.loads(o.strip().splitlines()[-1]))
    for o in outs:
        assert o["max"] == 300.0
        assert o["ms"] == pytest.approx(100.0)
        assert o["val"] == pytest.approx(0.05)      # 2 solves per 100 ms step
    assert outs[0]["x0"] != outs[1]["x0"]           # each replica solves its own problem


def test_single_rank_aggregation_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.job_seconds_per_solve(30.0, 3, 1) == (10.0, 0.01)


def test_reference_arm_is_rank0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_roofline_fields_and_arithmetic():
    # the roofline object of the bench line: achieved = n^2 pairs / average launch time,
    # peak = min(FMA-pipe rate / FMA ops per pair, MUFU rate) from unit counts and the clock
    sys.path.insert(0, ROOT)
    import bench

    class P:  # the mixture workload's shape without drawing its points
        n, d, nrhs = 100000, 8, 1

    clocks = {"sm_max_mhz": 2070.0}
    r = bench.roofline(P, kms=1620.0, kcnt=1000, clocks=clocks, precision=1, sms=152)
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in r
    assert r["bound"] == "alu" and r["unit"] == "Gpair/s"
    mufu = 152 * 32 * 2070e6 / 1e9
    assert r["peak"] == pytest.approx(mufu)
    assert r["achieved"] == pytest.approx(1e10 / 1.62e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    # the ncu DRAM bytes of the current kernel, or None until they have been captured
    assert r["traffic"] == bench.MEASURED_TRAFFIC.get((1, 100000, 8))
    r0 = bench.roofline(P, kms=3780.0, kcnt=1000, clocks=clocks, precision=0, sms=152)
    assert r0["peak"] == pytest.approx(152 * 128 * 2070e6 / 10 / 1e9)   # d + 1 + nrhs FMA ops
    assert r0["traffic"] is None                                        # not captured for this form
