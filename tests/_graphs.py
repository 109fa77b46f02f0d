"""Small graph builders shared by the tests (inputs only, no path arithmetic)."""

import json
import os

import numpy as np

import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_golden(name="hand_graph_10v.json"):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def kg_from_golden(gj, dtype="f32"):
    e = np.array(gj["edges_u_r_v"], dtype=np.int64)
    offsets, cols, rels = synth.canonicalize(gj["n"], gj["R"], e[:, 0], e[:, 1], e[:, 2])
    vemb = np.array(gj["vemb"], dtype=np.float32)
    remb = np.array(gj["remb"], dtype=np.float32)
    if dtype == "bf16":
        vemb, remb = synth.to_bf16_bits(vemb), synth.to_bf16_bits(remb)
    return synth.KG(n=gj["n"], R=gj["R"], n_types=int(max(gj["vtypes"]) + 1), offsets=offsets,
                    cols=cols, rels=rels, vtypes=np.array(gj["vtypes"], dtype=np.uint8),
                    vemb=vemb, remb=remb, dtype=dtype)


def random_kg(rng, n, m, R, d, dtype="f32", scale=0.5, dyadic=False, zero=False):
    u = rng.integers(0, n, size=m)
    v = rng.integers(0, n, size=m)
    r = rng.integers(0, R, size=m)
    offsets, cols, rels = synth.canonicalize(n, R, u, r, v)
    if zero:
        vemb = np.zeros((n, d), dtype=np.float32)
        remb = np.zeros((R, d), dtype=np.float32)
    elif dyadic:
        vemb = (rng.integers(-4, 5, size=(n, d)) / 4.0).astype(np.float32)
        remb = (rng.integers(-4, 5, size=(R, d)) / 4.0).astype(np.float32)
    else:
        vemb = (rng.standard_normal((n, d)) * scale).astype(np.float32)
        remb = (rng.standard_normal((R, d)) * scale).astype(np.float32)
    if dtype == "bf16":
        vemb, remb = synth.to_bf16_bits(vemb), synth.to_bf16_bits(remb)
    return synth.KG(n=n, R=R, n_types=3, offsets=offsets, cols=cols, rels=rels,
                    vtypes=rng.integers(0, 3, size=n).astype(np.uint8), vemb=vemb, remb=remb,
                    dtype=dtype)


def path_tuples(arr):
    """Structured path array -> list of (score, u, r1, v, r2, r3)."""
    return [(float(p["score"]), int(p["u"]), int(p["r1"]), int(p["v"]), int(p["r2"]), int(p["r3"]))
            for p in arr]
