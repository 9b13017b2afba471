"""The N > 1 path of bench.py on CPU: two gloo ranks, each with its own
problem, aggregated as the slowest rank's time and the sum of all pairs."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, _ = bench.dist_env()
    t, pairs = bench.reduce_over_ranks(1.0 + r, 100 * (r + 1), dist, "cpu")
    prob = bench.make_problem(r)
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, w, t, pairs, float(prob["mu1"][0, 0])))


def test_two_ranks_aggregate_on_cpu():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    # every rank sees the slowest time and the pairs of both ranks
    assert all(o[2] == 2.0 and o[3] == 300.0 for o in out)
    # the ranks work on different problems (seed + rank)
    assert out[0][4] != out[1][4]


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(2.5, 7, None, "cpu") == (2.5, 7.0)
