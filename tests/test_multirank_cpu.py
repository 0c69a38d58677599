"""The replicas path (N > 1) of bench.py on CPU, with gloo ranks.

A single MPS does not shard within this scope: N GPUs run N independent
replicas, and the job's numbers are the slowest replica's time and the sum of
all replicas' work.  These tests run that arithmetic across two real
processes (gloo on 127.0.0.1), and the reference arm under torchrun, where
rank 0 alone works and prints.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    sys.path.insert(0, ROOT)
    import bench
    seconds = bench.max_over_ranks(1.0 + 0.5 * rank, ws, device="cpu")  # rank 1 is the slower replica
    q.put((rank, seconds, bench.job_value(50, ws, seconds)))
    dist.barrier()
    dist.destroy_process_group()


def test_slowest_replica_and_whole_job_value_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, seconds, value in got:
        assert seconds == 1.5          # max over ranks, the same on every rank
        assert value == 50 * 2 / 1.5   # all replicas' updates over the slowest time


def test_reference_arm_under_torchrun_prints_one_line_from_rank0():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [line for line in out.stdout.splitlines() if line.startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_side_measurement_records_a_failure():
    import bench

    def boom(x):
        raise RuntimeError(f"tebd_batch_step: non-finite singular values (status -7) {x}")
    assert bench.side_measurement(lambda x: {"ok": x}, 3) == {"ok": 3}
    assert bench.side_measurement(boom, 1) == {"error": "RuntimeError: tebd_batch_step: non-finite singular "
                                                         "values (status -7) 1"}
