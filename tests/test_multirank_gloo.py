"""The multi-rank path of the benchmark on CPU ranks (gloo, world size 2): the job time is
the slowest rank's, the value counts every rank's block (weak scaling), each rank draws its
own block, and under torchrun only rank 0 of the reference arm prints."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [12.5, 20.0][rank]
    t = bench.reduce_max_time(local, world)
    out[rank] = (t, bench.job_value(1360.0, world, t), bench.rank_block_seed(2002, rank))
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_max_and_weak_scaling_value():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    (t0, v0, s0), (t1, v1, s1) = out[0], out[1]
    assert t0 == t1 == 20.0                      # slowest rank
    assert abs(v0 - 2 * 1360.0 / 0.020) < 1e-6   # both ranks' applies
    assert s0 != s1                              # independent blocks


@pytest.mark.slow
def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
