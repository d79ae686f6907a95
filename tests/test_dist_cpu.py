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
        q.put((rank, t, mine))
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
