"""Seeded synthetic input generators (graphs in int32 CSR form).

This package is shared by the CPU oracle tests and the CUDA path. It holds
none of the method's arithmetic: it only builds connected, simple,
undirected graphs and picks pivots, so both sides see identical inputs.
"""
from .graphs import (Graph, grid, cycle, complete, path, star, rmat, ba, er,
                     hyperbolic, from_edges, max_degree_vertex, workload, batch_specs, batch_graph)

__all__ = ["Graph", "grid", "cycle", "complete", "path", "star", "rmat", "ba",
           "er", "hyperbolic", "from_edges", "max_degree_vertex", "workload",
           "batch_specs", "batch_graph"]
