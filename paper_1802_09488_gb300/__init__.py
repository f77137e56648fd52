"""GB300-native adaptive geospatial join, probe side.

Kipf et al., "Adaptive Geospatial Joins for Modern Hardware": points are
mapped to 64-bit quadtree/Hilbert cell ids, looked up in an Adaptive Cell
Trie over polygon coverings (true-hit and candidate references), and only
candidate references get an exact point-in-polygon test.  The native library
(include/agj.h) does all of it; this package is its thin binding plus the
seeded synthetic workloads.
"""
from .native import (APPROX, AUTO, CONTAINS, COVERS, EXACT, INTERSECTS, AgjError, Batch, Counts, Index, LoadSpecPy, Pairs, Server, cell_ids, cell_ids_host,
                     join, join_batched, join_count, join_host, join_timed, lib, measure_fp64_rate, plain_load, train_online,
                     supercover)

__all__ = ["APPROX", "AUTO", "EXACT", "COVERS", "INTERSECTS", "CONTAINS", "AgjError", "Batch", "Index", "LoadSpecPy", "Pairs", "Server", "join", "join_batched",
           "join_host", "cell_ids", "cell_ids_host", "lib", "plain_load", "supercover", "join_timed", "Counts",
           "join_count", "measure_fp64_rate", "train_online"]
