"""Input generators: canonical CSR form, exact sizes, determinism (CPU only)."""

import numpy as np
import pytest

import synth


def check_canonical(g):
    off, cols, rels = g.offsets, g.cols, g.rels
    assert off[0] == 0 and off[-1] == cols.size and (np.diff(off) >= 0).all()
    assert cols.dtype == np.uint32 and rels.dtype == np.uint16 and off.dtype == np.int64
    assert (cols < g.n).all() and (rels < g.R).all()
    src = g.src_of_edges()
    assert not (src == cols).any()
    key = (src.astype(np.uint64) * np.uint64(g.n) + cols) * np.uint64(g.R) + rels
    assert (np.diff(key.astype(np.int64)) > 0).all()   # sorted by (u, col, rel), unique


def test_zipf_tiny_workload_shape():
    g = synth.gen_zipf_kg(10_000, 100_000, 8, 4, seed=0)
    check_canonical(g)
    assert g.E == 100_000
    assert g.out_degree().min() >= 1
    g2 = synth.gen_zipf_kg(10_000, 100_000, 8, 4, seed=0)
    assert (g.cols == g2.cols).all() and (g.rels == g2.rels).all()


def test_rmat_small_exact_edges():
    g = synth.gen_rmat_kg(12, 3000, 40_000, 6, 3, seed=1)
    check_canonical(g)
    assert g.E == 40_000
    od = g.out_degree()
    assert od.max() > 20 * od.mean()      # skewed


def test_canonicalize_dedups_and_drops_loops():
    off, cols, rels = synth.canonicalize(4, 2, [0, 0, 0, 1, 2, 3], [1, 1, 0, 0, 1, 0], [1, 2, 2, 1, 0, 2])
    # (0,1,1)? no: triples (u,r,v) = (0,1,1) (0,1,2) (0,0,2) (1,0,1)->loop (2,1,0) (3,0,2)
    assert off.tolist() == [0, 3, 3, 4, 5]
    assert cols.tolist() == [1, 2, 2, 0, 2]
    assert rels.tolist() == [1, 0, 1, 1, 0]


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(100_000) * rng.choice([1e-3, 1.0, 1e3], 100_000)).astype(np.float32)
    ours = synth.to_bf16_bits(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert (ours == ref).all()
    back = synth.bf16_bits_to_f32(ours)
    assert (torch.from_numpy(back) == torch.from_numpy(x).to(torch.bfloat16).float()).all()


def test_queries():
    g = synth.gen_rmat_kg(12, 3000, 40_000, 6, 3, seed=1)
    S, T = synth.queries_edge_biased(g, 50, seed=0)
    assert (S != T).all() and (g.out_degree()[S] > 0).all() and (g.in_degree()[T] > 0).all()
    S, T = synth.queries_log_degree(g, 50, max_deg=300, seed=0)
    assert (S != T).all() and (g.out_degree()[S] >= 1).all()
    s, t = synth.queries_hub(g)
    assert g.out_degree()[s[0]] == g.out_degree().max()
