"""Pins for the oracle's aggregation query (no GPU).

§V benchmarks "count(*) group by polygon_id" over the join.  The oracle
computes it as a histogram of its own join (np.bincount of the CSR ids);
here it is checked against brute force point by point on small inputs
(every polygon tested for every point with the plain predicate), and on a
tiling, where every point lies in at least one polygon.
"""
from collections import Counter

import numpy as np


def test_count_exact_equals_brute_force(oracle):
    from paper_1802_09488_gb300 import synth
    w = synth.c1_tiny(3000)
    ps = oracle.PolySet(w.polygons)
    got = ps.count_exact(w.points)
    want = Counter()
    for lat, lng in w.points:
        want.update(ps.hits_brute(lat, lng))
    assert got.dtype == np.uint64 and len(got) == len(w.polygons)
    assert [int(got[k]) for k in range(len(w.polygons))] == [want[k] for k in range(len(w.polygons))]
    # a tiling of the box: every point is counted at least once
    assert int(got.sum()) >= len(w.points)


def test_count_approx_equals_brute_force_on_a_covering(oracle):
    """A hand-built covering: two level-12 cells, one with references to
    polygons 0 (true) and 2 (candidate), one with polygon 1 (true)."""
    c = [oracle.id_parent(oracle.cell_id(40.70, -73.95), 12), oracle.id_parent(oracle.cell_id(40.75, -73.90), 12)]
    order = np.argsort(np.array(c, dtype=np.uint64))
    cells = np.array(c, dtype=np.uint64)[order]
    lists = [[(0 << 1) | 1, 2 << 1], [(1 << 1) | 1]]
    lists = [lists[k] for k in order]
    off = np.array([0, len(lists[0]), len(lists[0]) + len(lists[1])], dtype=np.uint64)
    refs = np.array(lists[0] + lists[1], dtype=np.uint32)
    pts = np.array([[40.70, -73.95]] * 3 + [[40.75, -73.90]] * 2 + [[10.0, 10.0]])
    got = oracle.count_approx_logical(cells, off, refs, pts, 4)
    assert list(got) == [3, 2, 3, 0]
