"""Seeded synthetic typed knowledge graphs, embeddings and (s, t) query sets.

This package only draws inputs.  It holds none of the path-search arithmetic:
no edge weights, no path scores, no ranking.  Both the CPU oracle and the CUDA
library consume the arrays it produces.
"""

from .kg import (  # noqa: F401
    KG,
    canonicalize,
    gen_zipf_kg,
    gen_rmat_kg,
    gen_embeddings,
    to_bf16_bits,
    bf16_bits_to_f32,
    queries_hub,
    queries_edge_biased,
    queries_log_degree,
    workload,
    WORKLOADS,
)
