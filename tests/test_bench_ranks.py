"""Multi-rank host logic of bench.py, on CPU with the gloo backend: two ranks
agree on the slowest rank's time, the whole-job value counts every rank's
work over that time, and the reference arm runs on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_CODE = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
dist.init_process_group("gloo")
import bench
r = dist.get_rank()
t = bench.job_time_ms(10.0 + 5.0 * r, dist, "cpu")
v = bench.job_value(dist.get_world_size(), 3.0e9, 4, t)
dist.barrier()
dist.destroy_process_group()
print(json.dumps({"rank": r, "t": t, "v": v}))
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_take_the_slowest_time():
    pytest.importorskip("torch")
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(r),
                   WORLD_SIZE="2", LOCAL_RANK=str(r))
        procs.append(subprocess.Popen([sys.executable, "-c", RANK_CODE, ROOT], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        assert o["t"] == 15.0                        # max over ranks of 10 and 15 ms
        # 2 ranks x 3e9 flops x 4 steps in 15 ms
        assert abs(o["v"] - 2 * 3.0e9 * 4 / 15e-3 / 1e12) < 1e-12


def test_single_process_time_is_its_own():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_time_ms(7.5, None, "cpu") == 7.5
    assert abs(bench.job_value(1, 1.0e12, 2, 1000.0) - 2.0) < 1e-12


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""
