"""Ordering MLP kernels vs the fp64 reference (oracle/mlp.py), training labels
vs the exact path enumeration, and the learned order's effect on the search
(identical results, work pruned reported)."""

import numpy as np
import pytest

import oracle
import synth
from oracle import mlp as omlp
from oracle.mitm import MITM
from tests._graphs import random_kg

pytestmark = pytest.mark.gpu


def bf16_round(x):
    return synth.bf16_bits_to_f32(synth.to_bf16_bits(np.asarray(x, dtype=np.float32)))


def make_model(mhr, rng):
    p = np.zeros(mhr.learn.N_PARAMS, dtype=np.float32)
    p[:65536] = rng.standard_normal(65536) * 0.06
    p[65536:65792] = rng.standard_normal(256) * 0.1
    p[65792:66048] = rng.standard_normal(256) * 0.1
    p[66048] = 0.25
    return mhr.OrderingMLP(params=p), p


def split(p):
    return p[:65536].reshape(256, 256), p[65536:65792], p[65792:66048], float(p[66048])


@pytest.fixture(scope="module")
def mhr():
    import paper_2406_07727_gb300 as m
    import paper_2406_07727_gb300.learn  # noqa: F401
    return m


def test_forward_and_backward_match_fp64_reference(mhr):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    model, p = make_model(mhr, rng)
    B = 300                                   # several 32-row tiles and a ragged tail
    Xf = rng.standard_normal((B, 256)).astype(np.float32)
    Xbits = synth.to_bf16_bits(Xf)
    X = torch.from_numpy(Xbits.view(np.int16)).cuda()
    tgt = rng.standard_normal(B).astype(np.float32)
    y = torch.empty(B, dtype=torch.float32, device="cuda")
    z1 = torch.empty((B, 256), dtype=torch.float32, device="cuda")
    mhr.mhr_mlp_forward(model, X, y, z1)
    W1, b1, w2, b2 = split(p)
    Xr = synth.bf16_bits_to_f32(Xbits).astype(np.float64)
    Z, H, yr = omlp.forward(bf16_round(W1), b1, w2, b2, Xr)
    assert np.allclose(z1.cpu().numpy(), Z, rtol=1e-4, atol=1e-4)
    assert np.allclose(y.cpu().numpy(), yr, rtol=1e-4, atol=1e-4)
    work = torch.empty((B, 256), dtype=torch.float32, device="cuda")
    grads = torch.empty(mhr.learn.N_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    mhr.mhr_mlp_backward(model, X, torch.from_numpy(tgt).cuda(), y, z1, work, grads, loss)
    g = grads.cpu().numpy()
    dW1, db1, dw2, db2 = omlp.backward(bf16_round(W1), b1, w2, b2, Xr, tgt)
    for got, want in ((g[:65536].reshape(256, 256), dW1), (g[65536:65792], db1), (g[65792:66048], dw2),
                      (np.array([g[66048]]), np.array([db2]))):
        assert np.linalg.norm(got - want) <= 1e-3 * max(1e-6, np.linalg.norm(want))
    assert abs(float(loss.item()) - omlp.loss(bf16_round(W1), b1, w2, b2, Xr, tgt)) <= 1e-4 * omlp.loss(
        bf16_round(W1), b1, w2, b2, Xr, tgt)


def test_adam_and_bf16_conversion(mhr):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    n = 1000
    p = rng.standard_normal(n).astype(np.float32)
    gs = [rng.standard_normal(n).astype(np.float32) for _ in range(3)]
    P = torch.from_numpy(p.copy()).cuda()
    M1 = torch.zeros(n, device="cuda")
    M2 = torch.zeros(n, device="cuda")
    m1 = np.zeros(n)
    m2 = np.zeros(n)
    pr = p.astype(np.float64)
    for k, g in enumerate(gs, start=1):
        mhr.mhr_mlp_adam(P, torch.from_numpy(g).cuda(), M1, M2, 1e-2, k)
        m1 = 0.9 * m1 + 0.1 * g
        m2 = 0.999 * m2 + 0.001 * g.astype(np.float64) ** 2
        pr -= 1e-2 * (m1 / (1 - 0.9 ** k)) / (np.sqrt(m2 / (1 - 0.999 ** k)) + 1e-8)
    assert np.allclose(P.cpu().numpy(), pr, rtol=1e-5, atol=1e-6)
    dst = torch.empty(n, dtype=torch.int16, device="cuda")
    mhr.mhr_mlp_to_bf16(P, dst)
    assert np.array_equal(dst.cpu().numpy().view(np.uint16), synth.to_bf16_bits(P.cpu().numpy()))


@pytest.mark.parametrize("dtype,d", [("f32", 64), ("bf16", 128), ("f32", 200), ("f32", 5)])
def test_feature_gather(mhr, dtype, d):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(d)
    g = random_kg(rng, 300, 2000, 3, d, dtype=dtype)
    G = mhr.load_kg(g)
    va = rng.integers(0, g.n, 77).astype(np.int32)
    vb = rng.integers(0, g.n, 77).astype(np.int32)
    X = mhr.mhr_mlp_features(G, torch.from_numpy(va).cuda(), torch.from_numpy(vb).cuda())
    got = X.cpu().numpy().view(np.uint16)
    e = g.vemb_f32()
    want = np.zeros((77, 256), dtype=np.float32)
    k = min(d, 128)
    want[:, :k] = e[va, :k]
    want[:, 128:128 + k] = e[vb, :k]
    assert np.array_equal(got, synth.to_bf16_bits(want))
    G.close()


def test_training_labels_match_path_enumeration(mhr):
    """best = best fp32 path score through the intermediate vertex: within the
    path error bound of the exact best fp64 score through it."""
    rng = np.random.default_rng(3)
    g = random_kg(rng, 120, 3000, 3, 8)
    G = mhr.load_kg(g)
    S = rng.integers(0, g.n, 6).astype(np.uint32)
    T = rng.integers(0, g.n, 6).astype(np.uint32)
    ok = S != T
    S, T = S[ok], T[ok]
    near_v, end_v, own, best = mhr.mhr_training_labels(G, S, T, 100000)
    near_v = near_v.cpu().numpy().view(np.uint32)
    end_v = end_v.cpu().numpy().view(np.uint32)
    best = best.cpu().numpy()
    # the row bound the search prunes with is an upper bound of every path through the row
    assert np.all(best <= own.cpu().numpy())
    m = MITM(g, "transe")
    exact = {}
    for s, t in zip(S.tolist(), T.tolist()):
        for sc, u, r1, v, r2, r3 in m.all_paths(s, t):
            # a hop-1 vertex u is labelled against endpoint t, a hop-3 vertex v against s
            for key in ((u, t), (v, s)):
                exact[key] = max(exact.get(key, -np.inf), sc)
    assert len(near_v) > 0
    for x, e, b in zip(near_v.tolist(), end_v.tolist(), best.tolist()):
        assert (x, e) in exact
        assert abs(b - exact[(x, e)]) <= 1e-3 * max(1.0, abs(exact[(x, e)]))
    G.close()


@pytest.mark.parametrize("K", [50, 500])
def test_learned_order_keeps_results_and_reports_work(mhr, K):
    """Train on held-out queries, then compare natural, bound and learned
    orders (with bound pruning) against the plain search: identical results;
    the work each order prunes is recorded."""
    g = synth.gen_rmat_kg(15, 30000, 600_000, 8, 3, seed=31)
    g.vemb, g.remb = synth.gen_embeddings(g.n, g.R, 64, 1 / 8, seed=31)
    S, T = synth.queries_edge_biased(g, 32, seed=31)
    St, Tt = synth.queries_edge_biased(g, 400, seed=31, stream=3)
    G = mhr.load_kg(g)
    model, rep = mhr.train_ordering_mlp(G, St, Tt, epochs=4, batch=2048, lr=2e-3)
    assert rep.rows > 1000 and rep.loss_last < rep.loss_first
    base, nb = mhr.mhr_topk_paths_batched(G, S, T, K)
    work = {}
    for name, opts in (("natural", {"prune": 1, "order": 0}), ("bound", {"prune": 1, "order": 1}),
                       ("learned", {"prune": 1, "order": 2, "mlp": model})):
        out, n, st = mhr.mhr_topk_paths_batched(G, S, T, K, opts=opts, with_stats=True)
        assert np.array_equal(n, nb)
        for q in range(len(S)):
            assert out[q][: n[q]].tobytes() == base[q][: nb[q]].tobytes()
        work[name] = (st["edges_scanned"], st["hits"], st["pruned_edges"])
    print("work (scanned, hits, pruned):", work, "train rows", rep.rows)
    # what the trained network gains over the same provable pruning without it
    # (rows in natural order): fewer middle edges scanned (whole work items
    # skipped) and fewer hits scored
    assert work["learned"][0] < work["natural"][0]
    assert work["learned"][1] < work["natural"][1]
    want, n_want = oracle.topk_paths_batch(g, S[:4], T[:4], K)
    for q in range(4):
        assert base[q][: nb[q]]["u"].tolist() == want[q][: n_want[q]]["u"].tolist()
    G.close()
