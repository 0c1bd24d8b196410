"""The multi-rank plumbing of bench.py on CPU: two gloo ranks (replicas),
max-over-ranks timing, and only rank 0 printing the JSON line."""
import io
import json
import multiprocessing as mp
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, world, port):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})


def _max_child(rank, world, port, q):
    _env(rank, world, port)
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group(backend="gloo")
    v = bench.max_over_ranks(1.5 + rank, world)
    bench.barrier(world)
    dist.destroy_process_group()
    q.put((rank, v))


def _reference_child(rank, world, port, q):
    _env(rank, world, port)
    sys.path.insert(0, ROOT)
    import bench
    sys.argv = ["bench.py", "--impl", "reference", "--workload", "small_field", "--steps", "1", "--warmup", "0",
                "--gpus", str(world)]
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.main()
    q.put((rank, buf.getvalue()))


def _run(target, world=2, timeout=300):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=timeout) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return out


def test_max_over_ranks_two_gloo_ranks():
    out = _run(_max_child)
    assert out == {0: 2.5, 1: 2.5}


def test_reference_arm_prints_once_under_two_ranks():
    out = _run(_reference_child)
    assert out[1].strip() == ""
    line = json.loads(out[0].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["unit"] == "GB/s" and line["value"] > 0
