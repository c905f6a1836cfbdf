"""The multi-process side of bench.py on CPU: world size 2 over gloo (one
process per rank, as torchrun launches them), the whole-job aggregation
(max time over ranks, summed work), and the reference arm printing on rank 0
only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


WORKER = r"""
import os, sys, json
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
ms = 10.0 * (rank + 1)
work = 100 + rank
t_max, work_all, e2e = bench.aggregate(ms, work, world, "cpu", op_max_seconds=0.5 + rank)
print(json.dumps({"rank": rank, "t_max": t_max, "work": work_all, "e2e": e2e,
                  "value": work_all / (t_max / 1e3)}), flush=True)
dist.barrier()
dist.destroy_process_group()
"""


def test_aggregate_over_two_gloo_ranks(tmp_path):
    pytest.importorskip("torch")
    script = tmp_path / "worker.py"
    script.write_text(WORKER)
    port = free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                   WORLD_SIZE="2", LOCAL_RANK=str(rank))
        procs.append(subprocess.Popen([sys.executable, str(script), ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        assert o["t_max"] == 20.0           # the slower rank's time
        assert o["work"] == 201             # both ranks' work
        assert o["e2e"] == 1.5
        assert abs(o["value"] - 201 / 0.020) < 1e-9


def test_reference_arm_prints_on_rank_zero_only():
    out = {}
    for rank in (0, 1):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank))
        p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                            "--warmup", "0", "--cpu-sample", "4", "--chi", "16", "--n-sites", "32"],
                           env=env, capture_output=True, text=True, timeout=600)
        assert p.returncode == 0, p.stderr
        out[rank] = p.stdout.strip()
    assert out[1] == ""
    line = json.loads(out[0].splitlines()[-1])
    assert line["impl"] == "reference" and line["cpu_baseline"]["kind"] == "oracle"
    assert line["value"] > 0 and line["e2e"]["h2d_bytes_per_step"] == 0
    # the same workload description as the GPU arm's line (bench.headline_config)
    sys.path.insert(0, ROOT)
    import bench
    import argparse
    args = argparse.Namespace(n_sites=32, chi=16, g=1, gpus=1)
    assert line["config"] == bench.headline_config(args, 1)
