"""The product's logical index on the workloads' own polygon sets, checked
by the oracle (no GPU).

For the city set (300 polygons, eps = 4 m) and the fine set (40 000
overlapping polygons, eps = 10 m):
  * every covering invariant holds on every cell (oracle checker, pinned in
    test_oracle_covering.py): no overlapping cells (§III-B), true hits
    wholly inside (§II), candidates meeting their polygon, and candidate
    diagonals below eps (§III-A);
  * the approximate join read off the covering has no false negatives and
    keeps every false positive within eps by geodesic distance (§III-A).
    This is checked on a sample of the workload's points, on every polygon
    vertex, and on points on and 1 µm to either side of every edge.
The fine set at eps = 1 m is checked on the GPU machine, beside its full-size
GPU parity test, because its host build needs a few minutes.
"""
import numpy as np
import pytest

from _edge_points import check_approx_property, edge_points

ZERO = {"overlapping_cells": 0, "true_ref_not_inside": 0, "cand_ref_misses": 0, "cand_diag_ge_eps": 0, "bad_ref": 0}


@pytest.fixture(scope="module")
def agj():
    import paper_1802_09488_gb300 as m
    m.lib()
    return m


def _run(agj, oracle, polys, eps, points, edge_stride, min_fp):
    ix = agj.Index(polys, agj.APPROX, eps, host_only=True)
    cells, off, refs = ix.logical()
    ps = oracle.PolySet(polys)
    assert ps.check_covering(cells, off, refs, eps_m=eps) == ZERO
    near = edge_points(oracle, polys, stride=edge_stride)
    n_exact, n_fp, worst = check_approx_property(oracle, ps, cells, off, refs, np.concatenate([points, near]), eps)
    assert n_exact > len(points) // 2 and n_fp >= min_fp and worst < eps
    return ix


def test_city_covering_and_precision(agj, oracle):
    from paper_1802_09488_gb300 import synth
    polys = synth.c2_city_polygons()
    pts = synth.points_mixture(200_000, synth.BOX_CITY, seed=3, dist_seed=3)
    ix = _run(agj, oracle, polys, 4.0, pts, edge_stride=1, min_fp=1000)
    assert ix.stats()["n_cells"] > 1_000_000


def test_fine_covering_and_precision(agj, oracle):
    from paper_1802_09488_gb300 import synth
    polys = synth.c3_fine_polygons(40_000, seed=5)
    pts = synth.points_mixture(200_000, synth.BOX_CITY, seed=6, dist_seed=5)
    ix = _run(agj, oracle, polys, 10.0, pts, edge_stride=3, min_fp=1000)
    st = ix.stats()
    assert st["n_polys"] == 40_000 and st["max_refs"] >= 3       # overlapping polygons share cells
