"""GPU parity of the join predicates (§II: ST_Covers; ST_Intersects and
ST_Contains "with similar techniques"), through the C ABI, against the
CPU oracle's point-polygon relation.

ST_Intersects of a point and a polygon is ST_Covers, so those joins must be
identical; ST_Contains differs exactly on points lying on a polygon's edge
or vertex, which the refine test's FP64 fallback decides.  Inputs: the
tiny tiling's vertices (on the boundary of two or three polygons each), edge
midpoints, points 1 µm to either side of every edge, invalid points and
uniform points; the city workload at 2e6 points with its boundary points.
"""
import numpy as np
import pytest

from tests._edge_points import edge_points

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def agj(torch):
    import paper_1802_09488_gb300 as m
    m.lib()
    return m


def _dev(torch, pts):
    return torch.from_numpy(np.ascontiguousarray(pts, dtype=np.float64)).cuda()


def _csr_equal(a, b):
    assert np.array_equal(np.asarray(a[0], dtype=np.int64), np.asarray(b[0], dtype=np.int64))
    assert np.array_equal(np.asarray(a[1], dtype=np.int64), np.asarray(b[1], dtype=np.int64))


def _boundary_points(oracle, polys, uniform):
    verts = np.concatenate(polys)
    mids = np.concatenate([0.5 * (p + np.roll(p, -1, axis=0)) for p in polys])
    extra = np.array([[np.nan, -73.9], [40.7, np.inf], [95.0, 0.0], [10.0, 20.0], [40.7, -73.95]])
    return np.concatenate([verts, mids, edge_points(oracle, polys, with_vertices=False), extra, uniform])


@pytest.fixture(scope="module")
def c1():
    from paper_1802_09488_gb300 import synth
    return synth.c1_tiny(20_000)


def test_contains_equals_oracle_on_boundary_points(torch, agj, oracle, c1):
    pts = _boundary_points(oracle, c1.polygons, c1.points)
    d = _dev(torch, pts)
    ix = agj.Index(c1.polygons, agj.EXACT, 0, predicate=agj.CONTAINS)
    assert ix.stats()["predicate"] == agj.CONTAINS
    got = agj.join(ix, d).to_host()
    want = oracle.PolySet(c1.polygons, contains=True).join_exact(pts)
    _csr_equal(got, want)
    # the predicate changes the result: every vertex is on the boundary
    cov = agj.join(agj.Index(c1.polygons, agj.EXACT, 0), d).to_host()
    nv = sum(len(p) for p in c1.polygons)
    assert cov[0][nv] - cov[0][0] > got[0][nv] - got[0][0]


def test_intersects_is_covers(torch, agj, oracle, c1):
    pts = _boundary_points(oracle, c1.polygons, c1.points)
    d = _dev(torch, pts)
    got_i = agj.join(agj.Index(c1.polygons, agj.EXACT, 0, predicate=agj.INTERSECTS), d).to_host()
    got_c = agj.join(agj.Index(c1.polygons, agj.EXACT, 0, predicate=agj.COVERS), d).to_host()
    _csr_equal(got_i, got_c)
    _csr_equal(got_c, oracle.PolySet(c1.polygons).join_exact(pts))


def test_approximate_join_is_the_same_for_every_predicate(torch, agj, c1):
    d = _dev(torch, c1.points)
    res = [agj.join(agj.Index(c1.polygons, agj.APPROX, c1.eps_m, predicate=p), d).to_host()
           for p in (agj.COVERS, agj.INTERSECTS, agj.CONTAINS)]
    _csr_equal(res[0], res[1])
    _csr_equal(res[0], res[2])


def test_contains_city_2m(torch, agj, oracle):
    from paper_1802_09488_gb300 import synth
    w = synth.c2_city(2_000_000, n_train=200_000)
    pts = np.concatenate([np.concatenate(w.polygons), edge_points(oracle, w.polygons, with_vertices=False, stride=7),
                          w.points])
    ix = agj.Index(w.polygons, agj.EXACT, 0, train=w.train, predicate=agj.CONTAINS)
    got = agj.join(ix, _dev(torch, pts)).to_host()
    _csr_equal(got, oracle.PolySet(w.polygons, contains=True).join_exact(pts))


def test_contains_counts_and_batched(torch, agj, oracle, c1):
    pts = _boundary_points(oracle, c1.polygons, c1.points)
    d = _dev(torch, pts)
    ix = agj.Index(c1.polygons, agj.EXACT, 0, predicate=agj.CONTAINS)
    eo, ei = oracle.PolySet(c1.polygons, contains=True).join_exact(pts)
    counts = agj.join_count(ix, d).to_host()
    assert np.array_equal(counts, np.bincount(ei.astype(np.int64), minlength=len(c1.polygons)).astype(np.uint64))
    # a batched launch mixing a covers and a contains index: each job = its plain join
    ic = agj.Index(c1.polygons, agj.EXACT, 0)
    outs = agj.join_batched([ix, ic], [d, d])
    _csr_equal(outs[0].to_host(), (eo, ei))
    _csr_equal(outs[1].to_host(), oracle.PolySet(c1.polygons).join_exact(pts))
