"""Host logic of the vertex-partitioned multi-GPU search, on CPU.

- Two and three gloo ranks exchange their partial lists with the module's
  all-gather: every rank receives every rank's lists, in rank order.
- Each rank's query options name its part.
- The decomposition itself, on the oracle: splitting the paths of a query by
  the hop-1 vertex (u % W), taking each part's K best and merging them gives
  the unpartitioned K best (the property Alg. 2's tree merge relies on).
The GPU search and merge of the parts are tested in test_gpu_partition.py.
"""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
from tests._graphs import path_tuples, random_kg  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        from paper_2406_07727_gb300 import partition
        nq, K = 5, 4
        # rank r's lists: bytes r*1000 + position, counts r + query
        out = (torch.arange(nq * K * 24, dtype=torch.int64) % 251 + rank).to(torch.uint8).reshape(nq, K * 24)
        n_out = torch.arange(nq, dtype=torch.int32) + rank
        parts, counts = partition.gather_parts(out, n_out)
        opts = partition.part_options({"prune": 1}, ws, rank)
        q.put((rank, parts.numpy(), counts.numpy(), opts))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2, 3])
def test_ranks_exchange_partial_lists(ws):
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
    nq, K = 5, 4
    for rank, parts, counts, opts in res:
        assert parts.shape == (ws, nq, K * 24) and counts.shape == (ws, nq)
        for r in range(ws):
            want = ((np.arange(nq * K * 24) % 251 + r) % 256).astype(np.uint8).reshape(nq, K * 24)
            assert np.array_equal(parts[r], want)
            assert np.array_equal(counts[r], np.arange(nq) + r)
        assert opts == {"prune": 1, "part_count": ws, "part_index": rank}


def test_single_rank_options_unchanged():
    from paper_2406_07727_gb300 import partition
    assert partition.part_options({"order": 1}, 1, 0) == {"order": 1}


@pytest.mark.parametrize("W", [2, 3, 5])
def test_partition_by_hop1_vertex_merges_to_the_full_result(W):
    """Every path has one hop-1 vertex u, so the parts u % W == r are disjoint
    and cover all paths; the K best of the union are the K best of the parts'
    K best (merged in the total order)."""
    rng = np.random.default_rng(W)
    for trial in range(4):
        g = random_kg(rng, 60, 900, 3, 4, dyadic=(trial % 2 == 0))
        s, t = int(rng.integers(0, 60)), int(rng.integers(0, 60))
        if s == t:
            continue
        _, _, n_paths = oracle.topk_paths(g, s, t, 1, with_counts=True)
        every = path_tuples(oracle.topk_paths(g, s, t, max(1, n_paths)))
        for K in (1, 7, 40):
            parts = [[p for p in every if p[1] % W == r][:K] for r in range(W)]
            assert sum(len(p) for p in [[x for x in every if x[1] % W == r] for r in range(W)]) == len(every)
            merged = sorted([p for part in parts for p in part], key=lambda p: (-p[0],) + p[1:])[:K]
            assert merged == every[:K]
