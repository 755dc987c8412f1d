"""The multi-rank bench path on CPU: two gloo ranks (one process each, 127.0.0.1)
agree on the slowest rank's time, and the whole-job value of N independent
replicas is N x units / that time (weak scaling, no data-path collective)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as D
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    D.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = [120.0, 135.5][rank]
    ms = bench.max_over_ranks(ms_local)
    value = bench.replica_throughput(8_294_400, ms, world)
    D.barrier()
    D.destroy_process_group()
    q.put((rank, ms, value))


def test_two_gloo_ranks_agree_on_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=5) for _ in range(2))
    for rank, ms, value in res:
        assert ms == 135.5
        assert value == pytest.approx(2 * 8_294_400 / 0.1355 / 1e6)


def test_single_process_is_its_own_maximum():
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.replica_throughput(1_000_000, 10.0, 1) == pytest.approx(100.0)
