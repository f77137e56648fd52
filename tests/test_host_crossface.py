"""Polygons across cube faces on the host (no GPU): the product splits each
into pieces, one per face it reaches, each the whole polygon in that face's
gnomonic plane; the oracle tests it in its own plane about the vertices'
mean.  Checked here: the logical index names input polygons, has cells on
every face the tiling reaches, passes the oracle's covering checker, and
its approximate join contains the exact join with every extra pair within
eps, on uniform points, vertices and points on and 1 um off every edge;
polygons wider than the 15-degree cap are refused.
"""
import numpy as np
import pytest

from tests._edge_points import check_approx_property, edge_points_3d


@pytest.fixture(scope="module")
def agj():
    import paper_1802_09488_gb300 as m
    m.lib()
    return m


@pytest.fixture(scope="module", params=["edge", "corner"])
def tiling(request):
    from paper_1802_09488_gb300 import synth
    box = synth.BOX_EDGE if request.param == "edge" else synth.BOX_CORNER
    polys = synth.crossface_tiling(box, seed=12 if request.param == "edge" else 13)
    pts = synth.points_uniform(20_000, box, seed=14)
    return request.param, polys, pts


def test_tiling_spans_faces(oracle, tiling):
    name, polys, pts = tiling
    faces = {oracle.face_uv(*v)[0] for p in polys for v in p}
    assert len(faces) == (2 if name == "edge" else 3)
    ps = oracle.PolySet(polys)
    assert sum(ps.face(k) == 6 for k in range(len(polys))) >= 3


@pytest.mark.parametrize("mode", ["approx", "exact"])
def test_crossface_covering_invariants(agj, oracle, tiling, mode):
    name, polys, pts = tiling
    m = agj.APPROX if mode == "approx" else agj.EXACT
    ix = agj.Index(polys, m, 10.0, train=pts[:4000] if mode == "exact" else None, host_only=True)
    st = ix.stats()
    assert st["n_polys"] == len(polys) and st["fast_ids"] == 0        # cells on several faces: FP64 ids
    cells, off, refs = ix.logical()
    assert int((refs >> 1).max()) < len(polys)
    assert len({int(c) >> 61 for c in cells}) == (2 if name == "edge" else 3)
    rep = oracle.PolySet(polys).check_covering(cells, off, refs, eps_m=10.0 if mode == "approx" else 0.0)
    if mode == "exact":
        rep.pop("cand_ref_misses")
    assert set(rep.values()) == {0}, rep


def test_crossface_approx_property(agj, oracle, tiling):
    name, polys, pts = tiling
    ix = agj.Index(polys, agj.APPROX, 10.0, host_only=True)
    cells, off, refs = ix.logical()
    probe = np.concatenate([pts, edge_points_3d(polys, stride=2)])       # the eps property holds on the edges too
    check_approx_property(oracle, oracle.PolySet(polys), cells, off, refs, probe, 10.0)


def test_too_wide_polygon_is_refused(agj):
    with pytest.raises(agj.AgjError) as e:
        agj.Index([np.array([[0.0, 30.0], [20.0, 45.0], [-20.0, 60.0]])], agj.EXACT, 0, host_only=True)
    assert e.value.status == 2
