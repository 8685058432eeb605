"""Replica mode of bench.py on CPU: two gloo ranks (world_size 2) check the host-side logic that a
multi-GPU run relies on -- rank environment, barrier, max-over-ranks timing and the whole-job
value -- and that the reference arm prints on rank 0 only."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    r, w, lr = bench.dist_env()
    dist = bench.dist_init(w, "gloo")
    bench.dist_barrier(dist)
    my_ms = 10.0 * (r + 1)  # rank 1 is the slowest
    mx = bench.dist_max(dist, my_ms, "cpu")
    value = bench.replica_value(w, 1_000_000, mx)
    # the reference arm: only rank 0 runs and prints
    buf = io.StringIO()
    if r != 0:
        class A:
            pass
        with redirect_stdout(buf):
            bench.reference_arm(A())
    bench.dist_barrier(dist)
    out.put((r, w, lr, mx, value, buf.getvalue()))
    dist.destroy_process_group()


def test_two_gloo_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    assert all(r[3] == 20.0 for r in res)  # max over ranks
    assert all(r[4] == pytest.approx(2 * 1e6 / 0.020 / 1e9) for r in res)
    assert res[1][5] == ""  # rank 1 printed nothing for the reference arm
