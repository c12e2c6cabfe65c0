"""Multi-process bookkeeping of bench.py on CPU (gloo, world size 2).

The lattice update does not shard here (replicas only): every rank
advances its own lattice and only the timing is reduced.  These tests run the
same Dist / aggregate_replicas code the GPU bench uses, with gloo ranks.
"""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    d = bench.Dist(backend="gloo")
    # rank r "took" 1 + r seconds for 10 steps of 1000 cells
    mlups, tmax = bench.aggregate_replicas(d, 1000.0, 10, 1.0 + rank)
    d.barrier()
    d.close()
    q.put((rank, mlups, tmax))


def test_replicas_aggregate_over_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    for rank, mlups, tmax in res:
        assert tmax == pytest.approx(2.0)                     # the slowest rank
        assert mlups == pytest.approx(2 * 1000 * 10 / 2.0 / 1e6)  # all ranks' updates / max time


def test_reference_arm_non_zero_rank_does_no_work(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0"]) == 0
    assert buf.getvalue() == ""


def test_reference_arm_line(monkeypatch):
    """The reference arm (the oracle on the host cores) prints one JSON line
    with the contract's keys."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.main(["--impl", "reference", "--steps", "2", "--warmup", "1", "--n", "32"]) == 0
    line = json.loads(buf.getvalue())
    assert line["impl"] == "reference" and line["unit"] == "MLUPS" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
