"""The multi-rank path of the benchmark on CPU (gloo, world size 2).

Queries are independent problems: each rank searches a disjoint shard of the
query set and no collective touches the data path; the ranks only meet at a
barrier and in the max-over-ranks reduction of the timing.
"""

import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, n_total, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank), CUDA_VISIBLE_DEVICES="")
    import bench
    import torch.distributed as dist
    try:
        w, r, local = bench.dist_setup()
        lo, hi = bench.shard_rows(n_total, r, w)
        bench.barrier(w)
        t = bench.max_over_ranks(w, 0.5 + r)
        out.put((r, w, lo, hi, t, dist.get_backend()))
    finally:
        if dist.is_initialized():
            dist.destroy_process_group()


@pytest.mark.parametrize("n_total", [10, 7, 1])
def test_two_ranks_shard_queries_and_reduce_time(n_total):
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, n_total, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    assert all(r[5] == "gloo" for r in res)
    # disjoint, ordered shards that cover the set
    covered = []
    for r in res:
        covered += list(range(r[2], r[3]))
    assert covered == list(range(n_total))
    # every rank sees the slowest rank's time
    assert all(r[4] == 1.5 for r in res)


def test_single_rank_takes_everything():
    import bench
    assert bench.shard_rows(10, 0, 1) == (0, 10)
    assert bench.shard_rows(0, 0, 2) == (0, 0)
