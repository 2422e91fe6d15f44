"""FP64 CPU oracle for Big-means -- TEST INFRASTRUCTURE ONLY.

Importable only by tests/, __graft_entry__.smoke() and bench.py's CPU
baseline / reference arm; the product path (paper_2204_07485_gb300) never
touches it.
"""
from .bigmeans import (big_means_workers, forgy_reseed, sq_distances, nearest, objective, kmeanspp_reseed,
                       lloyd, big_means, big_means_chunk, final_assignment,
                       BigMeansState, KppPick, LloydResult, ChunkRecord, Decisions)

__all__ = ["big_means_workers", "forgy_reseed", "sq_distances", "nearest", "objective", "kmeanspp_reseed", "lloyd",
           "big_means", "big_means_chunk", "final_assignment",
           "BigMeansState", "KppPick", "LloydResult", "ChunkRecord", "Decisions"]
