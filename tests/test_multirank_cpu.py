"""world_size-2 gloo checks of bench.py's replica path helpers on CPU: the
max-over-ranks timing reduction and the barrier; and that the reference arm
prints only on rank 0."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    bench.barrier(ws)
    m = bench.allreduce_max(float(10 * (rank + 1)), ws)
    q.put((rank, m))
    dist.destroy_process_group()


def test_allreduce_max_and_barrier_gloo():
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
    assert got == [(0, 20.0), (1, 20.0)]


def test_reference_arm_rank1_silent():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1",
               MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    # rank 1 of the reference arm must exit 0 without work or output; it never
    # reaches the process-group rendezvous because the reference arm only
    # needs rank 0.
    code = ("import sys; sys.path.insert(0, %r); import bench; "
            "bench.run_reference(type('A', (), {'workload': 'cfg1', 'steps': 1, "
            "'warmup': 0, 'gpus': 2})(), 2, 1)" % ROOT)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_rank0_prints_json():
    import json
    code = ("import sys; sys.path.insert(0, %r); import bench; "
            "bench.run_reference(type('A', (), {'workload': 'cfg1', 'steps': 2, "
            "'warmup': 1, 'gpus': 1})(), 1, 0)" % ROOT)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "gates/s"
    assert line["cpu_baseline"]["kind"] == "oracle"
