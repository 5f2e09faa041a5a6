"""bench.py --gpus N runs independent replicas; the only cross-rank step is
the max of the timed totals over a gloo group (world size 2, on CPU)."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    r, w, local = bench.dist_env()
    dist = bench.init_dist(w)
    bench.barrier(dist)
    total = bench.max_over_ranks(dist, 1.5 + rank)   # rank 1 is the slower replica
    q.put((r, w, local, total))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_slowest_replica():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert all(o[3] == 2.5 for o in out)


def test_single_process_needs_no_group():
    import bench
    assert bench.init_dist(1) is None
    assert bench.max_over_ranks(None, 3.0) == 3.0
