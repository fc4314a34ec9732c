"""Seeded synthetic inputs for CAPS filtered search.

This package only draws random inputs (vectors, attribute vectors, queries,
query constraints, k-means seed indices).  It holds none of the method's
arithmetic and is the one module shared by the CPU oracle tests and the GPU
path's tests and benchmark.
"""
from .synth import (  # noqa: F401
    Workload,
    CONFIGS,
    make_dense_workload,
    make_sparse_workload,
    config_small,
    config_sift1m_like,
    config_sift1m_fields,
    config_sift1m_wide,
    config_learned4m,
    with_constraints,
    config_sparse2m,
    zipf_probs,
)
