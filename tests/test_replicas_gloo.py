"""The multi-rank path of bench.py on CPU: two gloo ranks, as torchrun would start
them.  The workload does not shard (replicas only): every rank times its own
solves, the job's time is the slowest rank's, and the rate counts every rank's
units."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, t_ms, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ws_env, rank_env = bench._dist()
    m = bench.max_over_ranks(t_ms[rank], ws_env, device="cpu")
    out.put((rank_env, ws_env, m, bench.replica_rate(5, m, ws_env)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    t_ms = [120.0, 80.0]
    procs = [mp.Process(target=_rank, args=(r, 2, port, t_ms, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [g[0] for g in got] == [0, 1] and all(g[1] == 2 for g in got)
    assert all(g[2] == 120.0 for g in got)                     # the slower rank's time on both
    assert all(abs(g[3] - 2 * 5 / 0.120) < 1e-9 for g in got)  # 10 solves in 120 ms


def test_one_rank_is_the_local_time():
    import bench
    assert bench.max_over_ranks(42.0, 1) == 42.0
    assert abs(bench.replica_rate(3, 1500.0, 1) - 2.0) < 1e-12
