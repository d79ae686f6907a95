"""Host logic of the multi-GPU (replica) bench path on CPU: two gloo ranks, barrier, max-over-ranks timing and
system sharding. The single-system evaluation does not shard; replicas and batched systems need no
data-path collective."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    d = bench.Dist()
    try:
        d.barrier()
        t = d.max(1.5 + rank)  # each rank's timed-region length; the job is as slow as its slowest rank
        mine = bench.shard(list(range(10)), d.rank, d.world)
        every = bench.gather_all(d, (rank, mine))
        # the batched leg's systems and the served request stream, split by rank
        from paper_2009_12617_gb300 import workloads as wl

        sizes = [s.n for s in bench.shard(wl.batch_systems(64, seed=4), d.rank, d.world)]
        arr_all, which_all, pool, arr, which = bench.serving_stream(4000, d.rank, d.world)
        served = [int(pool[w]) for w in which]
        q.put((rank, t, mine, every, sizes, served, arr.tolist(), which_all.tolist()))
    finally:
        d.close()


def test_two_gloo_ranks_max_and_shard():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [2.5, 2.5]
    assert out[0][2] == [0, 2, 4, 6, 8] and out[1][2] == [1, 3, 5, 7, 9]
    assert sorted(out[0][2] + out[1][2]) == list(range(10))
    assert out[0][3] == out[1][3] == [(0, [0, 2, 4, 6, 8]), (1, [1, 3, 5, 7, 9])]  # all_gather_object
    # every batch system evaluated by exactly one rank
    from paper_2009_12617_gb300 import workloads as wl

    allsizes = [s.n for s in wl.batch_systems(64, seed=4)]
    assert sorted(out[0][4] + out[1][4]) == sorted(allsizes) and len(out[0][4]) == len(out[1][4]) == 32
    # every request served by exactly one rank, in arrival order, for the system it asked for
    which_all = out[0][7]
    assert out[1][7] == which_all
    assert len(out[0][5]) + len(out[1][5]) == 4000
    assert [w for w in which_all if w % 2 == 0] == out[0][5] and [w for w in which_all if w % 2 == 1] == out[1][5]
    for o in out:
        assert o[6] == sorted(o[6])
