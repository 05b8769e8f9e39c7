"""The multi-process path of bench.py (independent replicas, no data-path
collective): world-size-2 gloo ranks on the CPU exercise the barrier, the
max-over-ranks time and the whole-job aggregation."""
from __future__ import annotations

import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    class Args:
        impl = "ours"

    w, r, local, pg = bench.dist_setup(Args(), backend="gloo")
    bench.barrier(pg)
    my_ms = 100.0 + 50.0 * r  # rank 1 is the slow one
    mx = bench.max_over_ranks(pg, my_ms)
    value = bench.replica_value(w, 2.0 * 8192 ** 3, 10, mx)
    bench.barrier(pg)
    pg.destroy_process_group()
    q.put((r, w, mx, value))


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
    assert [r[0] for r in res] == [0, 1]
    assert all(r[1] == 2 and r[2] == 150.0 for r in res)  # both ranks see the slowest rank's time
    expect = 2 * 2.0 * 8192 ** 3 * 10 / 0.150 / 1e12
    assert all(abs(r[3] - expect) < 1e-9 * expect for r in res)
