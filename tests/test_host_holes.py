"""Polygons with holes on the host (no GPU): the product's logical index
against the oracle's ring semantics (the outer ring minus its holes; §II's
simple polygons widened).

* covering invariants by the oracle's independent checker: true-hit cells
  wholly inside the polygon (so never in or across a hole), candidate cells
  meeting it, disjoint cells, candidate diagonals below eps;
* the approximate join (the oracle's sorted-vector probe of the product's
  covering) contains the exact join and keeps every extra pair within eps,
  on uniform points, every vertex of every ring, and points on and 1 um to
  either side of every edge of every ring;
* the certified FP32 refine test decides like the oracle wherever it decides;
* malformed ring lists are refused.
"""
import ctypes as C

import numpy as np
import pytest

from tests._edge_points import check_approx_property, edge_points


@pytest.fixture(scope="module")
def agj():
    import paper_1802_09488_gb300 as m
    m.lib()
    return m


def _rings(p):
    return p if isinstance(p, list) else [p]


@pytest.fixture(scope="module")
def holes_c1():
    from paper_1802_09488_gb300 import synth
    w = synth.c1_tiny(20_000)
    polys = synth.with_holes(w.polygons, seed=9, frac=1.0)
    rings = [r for p in polys for r in _rings(p)]
    return polys, rings, w.points, w.eps_m


def test_ring_count_and_storage(agj, holes_c1):
    polys, rings, _, _ = holes_c1
    assert all(isinstance(p, list) and len(p) >= 2 for p in polys)
    ix = agj.Index(polys, agj.EXACT, 0, host_only=True)
    assert ix.stats()["n_polys"] == len(polys)


@pytest.mark.parametrize("mode", ["approx", "exact"])
def test_covering_invariants_with_holes(agj, oracle, holes_c1, mode):
    polys, rings, pts, eps = holes_c1
    m = agj.APPROX if mode == "approx" else agj.EXACT
    ix = agj.Index(polys, m, eps, train=pts[:3000] if mode == "exact" else None, host_only=True)
    cells, off, refs = ix.logical()
    rep = oracle.PolySet(polys).check_covering(cells, off, refs, eps_m=eps if mode == "approx" else 0.0)
    if mode == "exact":
        rep.pop("cand_ref_misses")      # §III-B: copied candidate references are rejected by the refine
    assert set(rep.values()) == {0}, rep
    # some true-hit cells exist and none lies in a hole: a point in a hole
    # centre (covered by no polygon) is referenced, if at all, as a candidate
    assert any(r & 1 for r in refs)


def test_approx_property_with_holes(agj, oracle, holes_c1):
    polys, rings, pts, eps = holes_c1
    ix = agj.Index(polys, agj.APPROX, eps, host_only=True)
    cells, off, refs = ix.logical()
    ps = oracle.PolySet(polys)
    probe = np.concatenate([pts, edge_points(oracle, rings)])
    check_approx_property(oracle, ps, cells, off, refs, probe, eps)
    # hole centres join nothing in the exact join
    centres = np.array([h.mean(0) for p in polys for h in p[1:]])
    eo, ei = ps.join_exact(centres)
    assert len(ei) == 0


def test_certified_refine_matches_oracle_near_holes(agj, oracle, holes_c1):
    polys, rings, pts, eps = holes_c1
    ix = agj.Index(polys, agj.EXACT, 0, host_only=True)
    ps = oracle.PolySet(polys)
    probe = np.concatenate([pts[:4000], edge_points(oracle, rings, offsets_m=(1e-6, -1e-6, 0.5, -0.5, 5.0, -5.0))])
    decided = 0
    for k in range(len(polys)):
        r = ix.covers_certified_host(probe, np.full(len(probe), k, dtype=np.uint32))
        for q in np.nonzero(r >= 0)[0]:
            assert bool(r[q]) == ps.covers(k, *probe[q]), (k, q)
            decided += 1
    assert decided > len(probe)


def test_malformed_rings_are_refused(agj):
    from paper_1802_09488_gb300 import native
    sq = np.array([[40.70, -73.96], [40.70, -73.94], [40.72, -73.94], [40.72, -73.96]])
    hole = np.array([[40.705, -73.955], [40.715, -73.955], [40.715, -73.945]])
    L = native.lib()

    def build(n_vertices, n_rings, ends):
        ll = np.ascontiguousarray(np.concatenate([sq, hole]))
        e = np.ascontiguousarray(np.array(ends, dtype=np.uint32))
        p = native.Polygon(n_vertices, n_rings, ll.ctypes.data, e.ctypes.data if len(ends) else None)
        arr = (native.Polygon * 1)(p)
        opts = native.BuildOpts()
        opts.host_only = 1
        h = C.c_void_p()
        rc = L.agj_build(arr, 1, 10.0, native.APPROX, C.byref(opts), C.c_void_p(0), C.byref(h))
        if rc == 0:
            L.agj_free(h)
        return rc

    assert build(7, 2, [4, 7]) == 0
    assert build(7, 2, [2, 7]) == 1          # a ring of 2 vertices
    assert build(7, 2, [4, 6]) == 1          # last end != n_vertices
    assert build(7, 2, [5, 4]) == 1          # not ascending
    assert build(7, 2, []) == 1              # no ring ends
    assert build(7, 1, []) == 0              # one ring of 7 vertices (ring_ends unused)
