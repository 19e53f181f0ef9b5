"""The N > 1 path of bench.py on the CPU: two ranks over gloo.

Each rank runs its own problems (weak scaling, no collective on the data
path); the JSON line's value is the points all ranks processed over the
slowest rank's time.  These tests drive the rank plumbing (process group,
barrier, max and sum reductions), the per-rank problem sets of the batched
workload and the aggregate rate with two CPU processes.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    g = bench.RankGroup(backend="gloo")
    assert (g.world, g.rank) == (world, rank)
    g.barrier()
    spec = bench.workload_spec("batch")
    spec["count"] = 6
    probs, shapes, dts, Ps = bench.batch_set(spec, g.rank)
    npts = sum(n * n for n, _ in shapes)
    seconds = 0.5 + rank                              # rank 1 is the slow one
    rate = bench.aggregate_rate(g, npts * 10, seconds)
    out.put((rank, [p.n for p in probs], npts, g.max(float(rank + 3)), g.sum(1.0), rate))
    g.barrier()
    g.close()


def test_two_ranks_over_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        rank, ns, npts, mx, sm, rate = out.get(timeout=120)
        res[rank] = (ns, npts, mx, sm, rate)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][0] != res[1][0]                     # each rank draws its own problems
    assert res[0][2] == res[1][2] == 4.0              # max over ranks
    assert res[0][3] == res[1][3] == 2.0              # sum over ranks
    total = (res[0][1] + res[1][1]) * 10
    for r in (0, 1):
        assert res[r][4] == pytest.approx(total / 1.5)   # all points over the slowest rank's time


def test_one_rank_is_the_identity(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    import bench
    g = bench.RankGroup()
    assert g.world == 1
    g.barrier()
    assert g.max(3.5) == 3.5 and g.sum(2.0) == 2.0
    assert bench.aggregate_rate(g, 100.0, 4.0) == 25.0
    g.close()
