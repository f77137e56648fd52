"""GPU parity for polygons across cube faces (split into one piece per face
by the build; joins report input polygon ids), through the C ABI, against
the CPU oracle, which tests such polygons in its own gnomonic plane.

Tilings of 40 km boxes on the cube edge of faces 0/1 and on the corner of
faces 0/1/2; points uniform in the box, every vertex, points 1 um to either
side of every edge.  (Points exactly on an edge of a cross-face polygon are
left out: the product tests them in a cube face's gnomonic plane and the
oracle in its own, and within the rounding of those projections, about
1e-9 m, the two may decide differently; 1 um is a thousand times that.)  Exact joins (ST_Covers and ST_Contains) bit-exact against
brute force; approximate joins bit-exact against the oracle's probe of the
index's logical covering; counts; a polygon with a hole, both across the
edge; a batched launch.
"""
import numpy as np
import pytest

from tests._edge_points import edge_points_3d

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


@pytest.fixture(scope="module", params=["edge", "corner"])
def tiling(request):
    from paper_1802_09488_gb300 import synth
    box = synth.BOX_EDGE if request.param == "edge" else synth.BOX_CORNER
    polys = synth.crossface_tiling(box, seed=12 if request.param == "edge" else 13)
    pts = np.concatenate([synth.points_uniform(200_000, box, seed=14), edge_points_3d(polys, offsets_m=(1e-6, -1e-6))])
    return polys, pts


@pytest.mark.parametrize("contains", [False, True])
def test_crossface_exact(torch, agj, oracle, tiling, contains):
    polys, pts = tiling
    ix = agj.Index(polys, agj.EXACT, 0, train=pts[:20_000], predicate=agj.CONTAINS if contains else agj.COVERS)
    got = agj.join(ix, _dev(torch, pts)).to_host()
    _csr_equal(got, oracle.PolySet(polys, contains=contains).join_exact(pts))


def test_crossface_approx_and_counts(torch, agj, oracle, tiling):
    polys, pts = tiling
    d = _dev(torch, pts)
    ia = agj.Index(polys, agj.APPROX, 4.0)
    got = agj.join(ia, d).to_host()
    cells, ro, refs = ia.logical()
    _csr_equal(got, oracle.join_approx_logical(cells, ro, refs, pts))
    counts = agj.join_count(ia, d).to_host()
    assert np.array_equal(counts, np.bincount(got[1].astype(np.int64), minlength=len(polys)).astype(np.uint64))
    ie = agj.Index(polys, agj.EXACT, 0)
    eo, ei = oracle.PolySet(polys).join_exact(pts)
    counts = agj.join_count(ie, d).to_host()
    assert np.array_equal(counts, np.bincount(ei.astype(np.int64), minlength=len(polys)).astype(np.uint64))


def test_crossface_hole_and_batched(torch, agj, oracle):
    from paper_1802_09488_gb300 import synth
    outer = np.array([[-0.2, 44.8], [-0.2, 45.2], [0.2, 45.2], [0.2, 44.8]])
    hole = np.array([[-0.05, 44.95], [0.05, 44.95], [0.05, 45.05], [-0.05, 45.05]])
    tri = np.array([[0.0, 44.9], [0.1, 45.1], [-0.1, 45.1]])
    polys = [[outer, hole], tri]
    rng = np.random.default_rng(6)
    pts = np.concatenate([np.stack([rng.uniform(-0.25, 0.25, 100_000), rng.uniform(44.75, 45.25, 100_000)], -1),
                          edge_points_3d([outer, hole, tri], offsets_m=(1e-6, -1e-6))])
    d = _dev(torch, pts)
    ix = agj.Index(polys, agj.EXACT, 0)
    want = oracle.PolySet(polys).join_exact(pts)
    _csr_equal(agj.join(ix, d).to_host(), want)
    plain = synth.c1_tiny(10).polygons
    ip = agj.Index(plain, agj.EXACT, 0)
    ia = agj.Index(polys, agj.APPROX, 2.0)
    outs = agj.join_batched([ix, ip, ia], [d, d, d])
    _csr_equal(outs[0].to_host(), want)
    _csr_equal(outs[1].to_host(), oracle.PolySet(plain).join_exact(pts))
    _csr_equal(outs[2].to_host(), agj.join(ia, d).to_host())
