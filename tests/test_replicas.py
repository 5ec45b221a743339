"""Multi-process checks (world_size 2, gloo, CPU) of the benchmark's
multi-GPU path, which runs independent replicas: every rank matches its own
instance, the whole-job work is the sum over ranks, the time is the slowest
rank's, and under a torchrun launch only rank 0 prints the JSON line."""
import json
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        units, t_ms = bench.replica_totals(100.0 * (rank + 1), 10.0 + 5 * rank, world, device="cpu")
        q.put((rank, units, t_ms, bench.replica_seed(7, rank)))
    finally:
        dist.destroy_process_group()


def test_replica_totals_sum_work_and_take_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_replica_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [(u, t) for _, u, t, _ in got] == [(300.0, 15.0), (300.0, 15.0)]
    assert got[0][3] != got[1][3]  # each replica has its own instance


def test_single_process_totals_pass_through():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_totals(5.0, 2.0, 1) == (5.0, 2.0)
    assert bench.replica_seed(3, 0) == 3


def test_reference_arm_under_torchrun_prints_once():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
           "--workload", "small"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-3000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
