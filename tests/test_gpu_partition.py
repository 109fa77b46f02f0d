"""Vertex-partitioned search on the GPU through the C ABI.

The W parts of a batch (paths split by hop-1 vertex u % W) run one after the
other on one GPU -- independent launches, as on W GPUs -- and each part must
equal the oracle's K best of its own paths; the GPU tree merge of the parts
(mhr_merge_paths, Alg. 2) must equal the unpartitioned search byte for byte.
"""

import numpy as np
import pytest

import oracle
import synth
from tests._graphs import path_tuples, random_kg
from tests.test_gpu_parity import compare_query

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mhr():
    import paper_2406_07727_gb300 as m
    return m


def parts_of(m, G, S, T, K, W, opts=None):
    outs, cnts = [], []
    for r in range(W):
        o = dict(opts or {})
        o.update(part_count=W, part_index=r)
        out, n = m.mhr_topk_paths_batched(G, S, T, K, opts=o)
        outs.append(out)
        cnts.append(n)
    return np.stack(outs), np.stack(cnts)


@pytest.mark.parametrize("W", [2, 3, 4, 7])
@pytest.mark.parametrize("fn", ["transe", "distmult"])
def test_parts_match_oracle_and_merge_to_full(mhr, W, fn):
    rng = np.random.default_rng(10 * W + (fn == "distmult"))
    for trial in range(4):
        g = random_kg(rng, 150, 5000, 4, 16, dtype="bf16" if trial % 2 else "f32", dyadic=(trial == 3))
        S = rng.integers(0, g.n, 10).astype(np.uint32)
        T = rng.integers(0, g.n, 10).astype(np.uint32)
        K = int(rng.choice([1, 9, 60]))
        G = mhr.load_kg(g, score_fn=fn)
        try:
            full, n_full = mhr.mhr_topk_paths_batched(G, S, T, K)
            opts = {"prune": 1, "order": 1} if trial % 2 else None
            parts, counts = parts_of(mhr, G, S, T, K, W, opts)
            merged, n_merged = mhr.mhr_merge_paths(parts, counts, K)
        finally:
            G.close()
        assert np.array_equal(n_merged, n_full)
        for q in range(len(S)):
            if S[q] == T[q]:
                assert n_full[q] == -1 and (counts[:, q] == -1).all()
                continue
            assert merged[q][: n_merged[q]].tobytes() == full[q][: n_full[q]].tobytes(), (q, W)
            # each part: the oracle's K best among the paths whose u it owns
            _, _, n_paths = oracle.topk_paths(g, int(S[q]), int(T[q]), 1, fn=fn, with_counts=True)
            every = oracle.topk_paths(g, int(S[q]), int(T[q]), max(1, n_paths), fn=fn)
            for r in range(W):
                want = every[every["u"] % W == r][:K]
                compare_query(parts[r, q], int(counts[r, q]), want, ctx=(q, r, W))


def test_merge_device_tensors_and_one_part(mhr):
    import torch
    rng = np.random.default_rng(3)
    g = random_kg(rng, 200, 6000, 3, 8)
    S = rng.integers(0, g.n, 12).astype(np.uint32)
    T = rng.integers(0, g.n, 12).astype(np.uint32)
    K = 25
    G = mhr.load_kg(g)
    try:
        full, n_full = mhr.mhr_topk_paths_batched(G, S, T, K)
        parts, counts = parts_of(mhr, G, S, T, K, 3)
    finally:
        G.close()
    dparts = torch.from_numpy(parts.view(np.uint8).reshape(3, len(S), K * 24)).cuda()
    dcounts = torch.from_numpy(counts).cuda()
    out, n_out = mhr.mhr_merge_paths(dparts, dcounts, K)
    torch.cuda.synchronize()
    got = mhr.paths_from_device(out, K)
    dn = n_out.cpu().numpy()
    assert np.array_equal(dn, n_full)
    for q in range(len(S)):
        assert got[q][: dn[q]].tobytes() == full[q][: n_full[q]].tobytes()
    # one part: the list itself
    one, n_one = mhr.mhr_merge_paths(full[None], n_full[None], K)
    assert np.array_equal(n_one, n_full)
    for q in range(len(S)):
        assert one[q][: n_one[q]].tobytes() == full[q][: n_full[q]].tobytes()


def test_partition_argument_errors(mhr):
    rng = np.random.default_rng(4)
    g = random_kg(rng, 50, 400, 3, 4)
    G = mhr.load_kg(g)
    S = np.array([1], dtype=np.uint32)
    T = np.array([2], dtype=np.uint32)
    try:
        for o in ({"part_count": 3, "part_index": 3}, {"part_count": 2, "part_index": -1},
                  {"part_count": 0, "part_index": 1}, {"part_count": -2}):
            with pytest.raises(mhr.MhrError) as e:
                mhr.mhr_topk_paths_batched(G, S, T, 5, opts=o)
            assert e.value.status == mhr.MHR_EINVAL
    finally:
        G.close()
    with pytest.raises(mhr.MhrError):
        mhr.mhr_merge_paths(np.zeros((2, 1, 5), dtype=mhr.PATH_DTYPE), np.zeros((2, 1), np.int32), 0)


@pytest.mark.slow
def test_medium_workload_partitioned(mhr):
    """The medium workload (1M vertices, 20M edges, 64 queries, K = 100) in 4
    parts, pruned form: the merge equals the unpartitioned bytes."""
    g, S, T, K, spec = synth.workload("medium")
    G = mhr.load_kg(g)
    try:
        full, n_full, st = mhr.mhr_topk_paths_batched(G, S, T, K, opts={"prune": 0, "order": 0}, with_stats=True)
        outs, cnts, scanned = [], [], 0
        for r in range(4):
            out, n, sr = mhr.mhr_topk_paths_batched(G, S, T, K, opts={"prune": 1, "order": 1, "part_count": 4,
                                                                    "part_index": r}, with_stats=True)
            outs.append(out)
            cnts.append(n)
            scanned += sr["edges_scanned"]
        merged, n_merged = mhr.mhr_merge_paths(np.stack(outs), np.stack(cnts), K)
    finally:
        G.close()
    assert np.array_equal(n_merged, n_full)
    for q in range(len(S)):
        assert merged[q][: n_merged[q]].tobytes() == full[q][: n_full[q]].tobytes()
    assert scanned > 0
