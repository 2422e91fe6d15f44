"""Seeded synthetic inputs shared by the oracle-side tests and the benchmarks.

This package holds randomness and data generation only: the Philox
counter-based generator, the chunk-index and K-means++ uniform draws laid out
on it, and the Gaussian-mixture datasets that stand in for the paper's
workloads. It contains none of the clustering arithmetic (no distances, no
means, no objective); that lives in ``oracle/`` (FP64 reference) and in the
CUDA library (product path), which never import each other.
"""
from .philox import philox4x64_10, philox_words, u64_to_unit_double, u64_mulhi
from .draws import chunk_indices, kpp_uniform_first, kpp_uniforms, chunk_draws
from . import mixtures

__all__ = [
    "philox4x64_10", "philox_words", "u64_to_unit_double", "u64_mulhi",
    "chunk_indices", "kpp_uniform_first", "kpp_uniforms", "chunk_draws",
    "mixtures",
]
