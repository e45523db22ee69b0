"""Seeded synthetic graph streams shared by the tests, the benchmark and the oracle checks.

This package only draws inputs (graphs in CSR form and edge-update batches).
It holds none of the community-detection arithmetic.
"""
from .streams import (  # noqa: F401
    Graph, csr_from_arcs, unit_f64, splitmix64, uniform_u64, planted_partition, rmat_directed,
    random_small_graph, EdgeStream, planted_stream, rewire_stream, rmat_stream, random_batch,
    powerlaw_planted, powerlaw_stream, config_graph, cached, rmat_workload, multi_graph_workload, sized_stream, INSERT, DELETE, REWEIGHT,
    rmat_undirected_c5, c5_stream, c5_size,
)
