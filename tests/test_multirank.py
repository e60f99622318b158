"""The replica path of bench.py with world size 2 on CPU (gloo): pairs are
sharded round-robin with no data exchange, and only the timing (max over
ranks) and the converged-POI count (sum over ranks) cross ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q) -> None:
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        units = bench.shard(5, rank, world)
        ms, conv = bench.reduce_over_ranks(10.0 + rank, 100.0 * (rank + 1), torch.device("cpu"))
        q.put((rank, units, ms, conv))
    finally:
        tdist.destroy_process_group()


def test_two_ranks_shard_and_reduce():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    assert got[0][1] == [0, 2, 4] and got[1][1] == [1, 3]
    for _, _, ms, conv in got:
        assert ms == 11.0          # slowest rank
        assert conv == 300.0       # all ranks' converged POIs


def test_single_process_reduce_is_identity():
    import bench
    assert bench.reduce_over_ranks(7.5, 42, torch.device("cpu")) == (7.5, 42.0)
