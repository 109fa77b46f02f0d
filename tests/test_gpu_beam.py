"""Generic H-hop beam search (Alg. 6 / Alg. 7) on the GPU vs the CPU oracle,
element by element, through the C ABI."""

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


def tuples(res, n):
    return [(float(p["score"]), int(p["hops"]), [int(x) for x in p["v"][: p["hops"] + 1]],
             [int(x) for x in p["r"][: p["hops"]]]) for p in res[:n]]


def run(m, g, S, T, H, K, fn):
    G = m.load_kg(g, score_fn=fn)
    try:
        out, n_out = m.mhr_beam_paths(G, S, T, H, K)
    finally:
        G.close()
    for q in range(len(S)):
        want = tuples(oracle.beam_paths(g, int(S[q]), int(T[q]), H, K, fn=fn), K)
        assert tuples(out[q], int(n_out[q])) == want, (q, H, K, fn)


@pytest.mark.parametrize("fn", ["transe", "distmult"])
@pytest.mark.parametrize("H,K", [(1, 5), (2, 1), (2, 8), (3, 4), (3, 16), (4, 3)])
def test_random_graphs(mhr, fn, H, K):
    rng = np.random.default_rng(H * 100 + K)
    g = random_kg(rng, 300, 6000, 5, 16, scale=0.3)
    S = rng.integers(0, g.n, size=12).astype(np.uint32)
    T = ((S + 1 + rng.integers(0, g.n - 1, size=12)) % g.n).astype(np.uint32)
    run(mhr, g, S, T, H, K, fn)


def test_hub_rows_span_several_chunks(mhr):
    rng = np.random.default_rng(7)
    g = random_kg(rng, 150, 50000, 4, 8, dtype="bf16", dyadic=True)
    S = rng.integers(0, g.n, size=6).astype(np.uint32)
    T = ((S + 7) % g.n).astype(np.uint32)
    run(mhr, g, S, T, 3, 10, "transe")
    run(mhr, g, S, T, 2, 64, "transe")


def test_tiny_workload(mhr):
    g, S, T, K, _ = synth.workload("tiny")
    run(mhr, g, np.asarray(S, dtype=np.uint32), np.asarray(T, dtype=np.uint32), 3, 10, "transe")


def test_argument_errors(mhr):
    g = random_kg(np.random.default_rng(1), 50, 200, 3, 4)
    G = mhr.load_kg(g)
    S = np.array([1], dtype=np.uint32)
    T = np.array([2], dtype=np.uint32)
    try:
        for H, K, st in [(0, 5, mhr.MHR_EINVAL), (9, 5, mhr.MHR_EINVAL), (3, 0, mhr.MHR_EINVAL),
                         (3, 65, mhr.MHR_ERANGE), (6, 10, mhr.MHR_ERANGE)]:
            with pytest.raises(mhr.MhrError) as e:
                mhr.mhr_beam_paths(G, S, T, H, K)
            assert e.value.status == st
        with pytest.raises(mhr.MhrError):
            mhr.mhr_beam_paths(G, S, S, 3, 5)
    finally:
        G.close()


def test_device_arrays(mhr):
    """Queries and results as device arrays (MHR_MEM_DEVICE): the caller's
    device pointers are used directly; results equal the oracle's and the
    host-array call's."""
    import torch
    rng = np.random.default_rng(12)
    g = random_kg(rng, 300, 6000, 5, 16, scale=0.3)
    S = rng.integers(0, g.n, size=10).astype(np.uint32)
    T = ((S + 1 + rng.integers(0, g.n - 1, size=10)) % g.n).astype(np.uint32)
    H, K = 3, 8
    G = mhr.load_kg(g)
    try:
        dS = torch.from_numpy(S.view(np.int32)).cuda()
        dT = torch.from_numpy(T.view(np.int32)).cuda()
        out, n_out = mhr.mhr_beam_paths(G, dS, dT, H, K)
        assert out.is_cuda and n_out.is_cuda
        host, n_host = mhr.mhr_beam_paths(G, S, T, H, K)
    finally:
        G.close()
    dev = mhr.beams_from_device(out, K)
    dn = n_out.cpu().numpy()
    assert np.array_equal(dn, n_host)
    for q in range(len(S)):
        assert dev[q][: dn[q]].tobytes() == host[q][: n_host[q]].tobytes()
        want = tuples(oracle.beam_paths(g, int(S[q]), int(T[q]), H, K), K)
        assert tuples(dev[q], int(dn[q])) == want, q


@pytest.mark.parametrize("dyadic", [False, True])
def test_long_rows_fp32_screen(mhr, dyadic):
    """Rows of about a thousand edges (several staging sorts of the fp32
    screen per held path), with exact ties when dyadic: the band around each
    path's K-th fp32 extension must keep every extension of the fp64 K best."""
    rng = np.random.default_rng(31 + dyadic)
    g = random_kg(rng, 60, 60000, 20, 16, dyadic=dyadic, scale=0.4)
    S = rng.integers(0, g.n, size=6).astype(np.uint32)
    T = ((S + 11) % g.n).astype(np.uint32)
    for H, K in ((2, 1), (3, 16), (2, 64)):
        run(mhr, g, S, T, H, K, "transe")
        run(mhr, g, S, T, H, K, "distmult")
