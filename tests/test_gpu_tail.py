"""Tail prediction (Alg. 3 / Alg. 4) on the GPU vs the CPU oracle, element by
element, through the C ABI.

Bar: candidate ids and order bit-exact, scores bit-identical (the fp64
rescoring repeats the oracle's operation order).  Cases span the register-row
kernels (fp32 and bf16 rows, padded vector counts), the any-length kernel
(dims not a multiple of the 16-byte vector, dims above 1024), query batches
split over several launches, the one-pass and sampled two-pass forms, exact
ties (zero embeddings: every candidate in the band), survivor lists that
overflow their sized buffer (an adversarial candidate order), empty candidate
sets, K above the candidate count and at MHR_TAIL_K_MAX.
"""

import numpy as np
import pytest

import oracle
import synth
from tests._graphs import random_kg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mhr():
    import paper_2406_07727_gb300 as m
    return m


def compare(got, n_got, want, n_want, ctx=""):
    assert n_got.tolist() == n_want.tolist(), ctx
    for q in range(len(n_want)):
        k = int(n_want[q])
        g = [(float(x["score"]), int(x["v"])) for x in got[q][:k]]
        w = [(float(x["score"]), int(x["v"])) for x in want[q][:k]]
        assert [v for _, v in g] == [v for _, v in w], (ctx, q)
        assert [s for s, _ in g] == [s for s, _ in w], (ctx, q, "scores not bit-identical")


def run(m, g, H, Rq, K, cand_type, fn, stats=False):
    G = m.load_kg(g, score_fn=fn)
    try:
        res = m.mhr_tail_topk(G, H, Rq, K, cand_type=cand_type, with_stats=stats)
    finally:
        G.close()
    want, n_want = oracle.tail_topk(g, H, Rq, K, cand_type=cand_type, fn=fn)
    compare(res[0], res[1], want, n_want, ctx=(fn, K, cand_type))
    return res


def queries(rng, g, nq):
    return (rng.integers(0, g.n, size=nq).astype(np.uint32),
            rng.integers(0, g.R, size=nq).astype(np.uint16))


@pytest.mark.parametrize("fn", ["transe", "distmult"])
@pytest.mark.parametrize("cand_type", [-1, 0, 3])
@pytest.mark.parametrize("K", [1, 10, 100])
def test_tiny_workload(mhr, fn, cand_type, K):
    g = synth.workload("tiny")[0]
    rng = np.random.default_rng(K + 7 * (cand_type + 1))
    H, Rq = queries(rng, g, 5)
    run(mhr, g, H, Rq, K, cand_type, fn)


@pytest.mark.parametrize("fn", ["transe", "distmult"])
@pytest.mark.parametrize("dtype,d", [("f32", 8), ("f32", 12), ("f32", 10), ("f32", 128), ("f32", 256),
                                     ("f32", 1040), ("bf16", 8), ("bf16", 40), ("bf16", 20),
                                     ("bf16", 128)])
def test_row_formats(mhr, fn, dtype, d):
    # 8/12/128/256 fp32 and 8/40/128 bf16: register rows, two per lane group
    # (12: a padded vector count); 10 fp32, 20 bf16 (not whole 16-byte
    # vectors) and 1040 fp32 (above 512): the any-length kernel
    rng = np.random.default_rng(d)
    n = 12000 if d < 1000 else 3000
    g = random_kg(rng, n, 3 * n, 5, d, dtype=dtype, scale=0.3)
    H, Rq = queries(rng, g, 4)
    run(mhr, g, H, Rq, 20, -1, fn)
    run(mhr, g, H, Rq, 7, 1, fn)


def test_two_pass_and_many_queries(mhr):
    # 40000 candidates: sampled two-pass form; 300 queries at d = 64 span two
    # scan launches
    rng = np.random.default_rng(1)
    g = random_kg(rng, 40000, 80000, 9, 64, scale=0.25)
    H, Rq = queries(rng, g, 300)
    _, _, st = run(mhr, g, H, Rq, 50, -1, "transe", stats=True)
    M = max(8192, 32 * 50, 40000 // 256)
    assert st["edges_scanned"] == 300 * (40000 + M)
    assert st["rescored"] >= 300 * 50
    assert st["dense_queries"] == 0


@pytest.mark.parametrize("n,K", [(20000, 4096), (200000, 1000)])
def test_large_K(mhr, n, K):
    # dyadic bf16 rows: many exact ties at the K-th score; 200000 candidates
    # with K = 1000 take the sampled two-pass form
    rng = np.random.default_rng(K)
    g = random_kg(rng, n, 2 * n, 4, 16, dtype="bf16", dyadic=True)
    H, Rq = queries(rng, g, 3)
    run(mhr, g, H, Rq, K, -1, "transe")
    run(mhr, g, H, Rq, K, 2, "distmult")


def test_K_above_candidate_count(mhr):
    rng = np.random.default_rng(6)
    g = random_kg(rng, 9000, 20000, 4, 24, scale=0.3)
    H, Rq = queries(rng, g, 3)
    _, n_out = run(mhr, g, H, Rq, 4096, 2, "transe")
    assert n_out.tolist() == [int(np.sum(g.vtypes == 2))] * 3


def test_all_ties_overflow_and_large_band(mhr):
    # zero vertex embeddings: every candidate scores gamma - |w_r|_1; the
    # survivors overflow the sized buffer, the query is rescanned alone and the
    # band (every candidate) is larger than the shared-memory sort
    rng = np.random.default_rng(2)
    g = random_kg(rng, 20000, 30000, 3, 8, dyadic=True)
    g.vemb[:] = 0.0
    H, Rq = queries(rng, g, 2)
    _, _, st = run(mhr, g, H, Rq, 10, -1, "transe", stats=True)
    assert st["dense_queries"] == 2
    assert st["rescored"] == 2 * 20000
    run(mhr, g, H, Rq, 300, -1, "distmult")


def test_adversarial_candidate_order_rescans(mhr):
    # the strided sample (even positions) holds only far candidates, so its
    # threshold keeps every odd candidate and the sized buffer overflows
    rng = np.random.default_rng(3)
    n, d = 20000, 8
    g = random_kg(rng, n, 2 * n, 1, d)
    g.vtypes[:] = 0
    g.remb[:] = 0.0
    g.vemb[0::2] = 4.0
    g.vemb[1::2] = (rng.integers(-2, 3, size=(n // 2, d)) / 8.0).astype(np.float32)
    g.vemb[1] = 0.0
    H = np.array([1, 3], dtype=np.uint32)
    Rq = np.zeros(2, dtype=np.uint16)
    _, _, st = run(mhr, g, H, Rq, 1, -1, "transe", stats=True)
    assert st["dense_queries"] == 2


def test_device_memory_and_empty_type(mhr):
    import torch
    rng = np.random.default_rng(4)
    g = random_kg(rng, 15000, 30000, 6, 32, scale=0.3)
    H, Rq = queries(rng, g, 9)
    G = mhr.load_kg(g)
    try:
        host, n_host = mhr.mhr_tail_topk(G, H, Rq, 25, cand_type=1)
        dev, n_dev = mhr.mhr_tail_topk(G, torch.from_numpy(H).cuda(),
                                       torch.from_numpy(Rq.astype(np.int16)).cuda(), 25, cand_type=1)
        torch.cuda.synchronize()
        assert n_dev.cpu().numpy().tolist() == n_host.tolist()
        dev = mhr.tails_from_device(dev, 25)
        for q in range(9):
            assert dev[q][: n_host[q]].tobytes() == host[q][: n_host[q]].tobytes()
        empty, n_empty = mhr.mhr_tail_topk(G, H, Rq, 5, cand_type=200)
        assert n_empty.tolist() == [0] * 9
        none, n_none = mhr.mhr_tail_topk(G, H[:0], Rq[:0], 5)
        assert n_none.shape == (0,)
    finally:
        G.close()
    want, n_want = oracle.tail_topk(g, H, Rq, 25, cand_type=1)
    compare(host, n_host, want, n_want)


def test_argument_errors(mhr):
    rng = np.random.default_rng(5)
    g = random_kg(rng, 100, 300, 4, 8)
    G = mhr.load_kg(g)
    H = np.array([1, 2], dtype=np.uint32)
    Rq = np.array([0, 3], dtype=np.uint16)
    try:
        for kw, status in [(dict(K=0), mhr.MHR_EINVAL), (dict(K=4097), mhr.MHR_ERANGE),
                           (dict(K=5, cand_type=256), mhr.MHR_EINVAL), (dict(K=5, cand_type=-2), mhr.MHR_EINVAL)]:
            with pytest.raises(mhr.MhrError) as e:
                mhr.mhr_tail_topk(G, H, Rq, **kw)
            assert e.value.status == status
        with pytest.raises(mhr.MhrError) as e:
            mhr.mhr_tail_topk(G, np.array([100], dtype=np.uint32), Rq[:1], 5)
        assert e.value.status == mhr.MHR_EINVAL
        with pytest.raises(mhr.MhrError) as e:
            mhr.mhr_tail_topk(G, H[:1], np.array([4], dtype=np.uint16), 5)
        assert e.value.status == mhr.MHR_EINVAL
        # the graph stays usable after rejected calls
        out, n = mhr.mhr_tail_topk(G, H, Rq, 5)
        want, n_want = oracle.tail_topk(g, H, Rq, 5)
        compare(out, n, want, n_want)
    finally:
        G.close()


@pytest.mark.parametrize("fn", ["transe", "distmult"])
def test_medium_graph_full_size(mhr, fn):
    # the benchmark's configuration: the 1M-vertex, d = 128 graph, 64 heads
    # (the K persons of Alg. 4) against every vertex of one type, K = 50, and
    # one head against every vertex (Alg. 3)
    g = synth.workload("medium")[0]
    rng = np.random.default_rng(8)
    H, Rq = queries(rng, g, 64)
    run(mhr, g, H, Rq, 50, 0, fn)
    run(mhr, g, H[:1], Rq[:1], 50, -1, fn)
