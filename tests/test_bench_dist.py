"""Multi-rank host logic of the benchmark (replicas, weak scaling) on CPU:
two gloo ranks take the slowest rank's time, count every rank's queries, and
draw different query sets on the same graph."""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        import synth
        g = synth.gen_zipf_kg(2000, 20000, 4, 3, seed=5)
        S0, T0 = synth.queries_edge_biased(g, 16, seed=0)
        S, T = bench.rank_queries(g, S0, T0, rank, "medium")
        local_ms = 100.0 * (rank + 1)           # rank 1 is the slow one
        max_ms = bench.max_over_ranks(local_ms, ws, "cpu")
        rate = bench.job_rate(len(S), ws, 10, max_ms)
        allq = [None] * ws
        dist.all_gather_object(allq, (S.tolist(), T.tolist()))
        q.put((rank, max_ms, rate, allq))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_weak_scaling():
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, max_ms, rate, allq in res:
        assert max_ms == 200.0                              # the slowest rank's time on every rank
        assert rate == pytest.approx(16 * 2 * 10 / 0.2)     # all ranks' queries / that time
        (s0, t0), (s1, t1) = allq
        assert len(s0) == len(s1) == 16
        assert (s0, t0) != (s1, t1)                          # each replica its own queries
        assert all(a != b for a, b in zip(s1, t1))


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.job_rate(64, 1, 200, 1000.0) == 64 * 200
    import synth
    g = synth.gen_zipf_kg(500, 4000, 2, 2, seed=1)
    S, T = synth.queries_edge_biased(g, 8, seed=0)
    S2, T2 = bench.rank_queries(g, S, T, 0, "medium")
    assert np.array_equal(S, S2) and np.array_equal(T, T2)
