"""The multi-rank bookkeeping of the benchmark on two CPU processes (gloo):
balanced disjoint shards that cover every unit, the barrier, and the maximum of
the ranks' timings that sets the reported time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    from paper_1101_2254_gb300 import dist as gd
    w, r, _ = gd.env()
    gd.init(w)
    import torch.distributed as dist
    out = {}
    for count in (0, 1, 7, 4096, 65537):
        a, b = gd.shard(count, r, w)
        got = [None] * w
        dist.all_gather_object(got, (a, b))
        out[count] = got
    gd.barrier(w)
    out["max"] = gd.max_over_ranks(10.0 + 3.0 * r, w)
    gd.finalize(w)
    q.put((r, out))


def test_two_rank_shards_and_max_over_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world = 2
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        out = res[r]
        assert out["max"] == 13.0  # the slower rank's time on every rank
        for count in (0, 1, 7, 4096, 65537):
            spans = out[count]
            assert spans[0][0] == 0 and spans[-1][1] == count
            assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1


def test_single_rank_is_a_no_op():
    from paper_1101_2254_gb300 import dist as gd
    assert gd.shard(10, 0, 1) == (0, 10)
    assert gd.max_over_ranks(4.5, 1) == 4.5
    gd.barrier(1)
