"""GPU parity for polygons with holes (the outer ring minus its holes),
through the C ABI, against the CPU oracle's ring semantics.

Exact joins (ST_Covers and ST_Contains) bit-exact against the oracle's
brute force; approximate joins bit-exact against the oracle's sorted-vector
probe of the index's logical covering (whose precision the host tests pin);
counts; a batched launch with an index with holes.  Inputs: uniform and
mixture points, every vertex of every ring, points on and 1 um to either
side of every ring edge, hole centres.
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


def _rings(p):
    return p if isinstance(p, list) else [p]


def _probe_points(oracle, polys, base, stride=1):
    rings = [r for p in polys for r in _rings(p)]
    centres = np.array([h.mean(0) for p in polys if isinstance(p, list) for h in p[1:]])
    return np.concatenate([base, np.concatenate(rings), edge_points(oracle, rings, with_vertices=False, stride=stride),
                           centres])


@pytest.fixture(scope="module")
def holes_c1():
    from paper_1802_09488_gb300 import synth
    w = synth.c1_tiny(50_000)
    return synth.with_holes(w.polygons, seed=9, frac=1.0), w.points, w.eps_m


@pytest.mark.parametrize("contains", [False, True])
def test_c1_holes_exact(torch, agj, oracle, holes_c1, contains):
    polys, base, eps = holes_c1
    pts = _probe_points(oracle, polys, base)
    pred = agj.CONTAINS if contains else agj.COVERS
    ix = agj.Index(polys, agj.EXACT, 0, train=base[:5000], predicate=pred)
    got = agj.join(ix, _dev(torch, pts)).to_host()
    _csr_equal(got, oracle.PolySet(polys, contains=contains).join_exact(pts))


def test_c1_holes_approx_and_counts(torch, agj, oracle, holes_c1):
    polys, base, eps = holes_c1
    pts = _probe_points(oracle, polys, base)
    d = _dev(torch, pts)
    ix = agj.Index(polys, agj.APPROX, eps)
    got = agj.join(ix, d).to_host()
    cells, ro, refs = ix.logical()
    _csr_equal(got, oracle.join_approx_logical(cells, ro, refs, pts))
    counts = agj.join_count(ix, d).to_host()
    assert np.array_equal(counts, np.bincount(got[1].astype(np.int64), minlength=len(polys)).astype(np.uint64))
    ie = agj.Index(polys, agj.EXACT, 0)
    eo, ei = oracle.PolySet(polys).join_exact(pts)
    counts = agj.join_count(ie, d).to_host()
    assert np.array_equal(counts, np.bincount(ei.astype(np.int64), minlength=len(polys)).astype(np.uint64))


def test_city_holes_2m(torch, agj, oracle):
    """300 city polygons, 91 of them with 1-3 holes: exact and approximate
    joins of 2e6 mixture points plus the rings' boundary points."""
    from paper_1802_09488_gb300 import synth
    polys = synth.c2_city_holes_polygons()
    base = synth.points_mixture(2_000_000, synth.BOX_CITY, seed=3)
    train = synth.points_mixture(200_000, synth.BOX_CITY, seed=4, dist_seed=3)
    pts = _probe_points(oracle, polys, base, stride=5)
    d = _dev(torch, pts)
    ie = agj.Index(polys, agj.EXACT, 0, train=train)
    _csr_equal(agj.join(ie, d).to_host(), oracle.PolySet(polys).join_exact(pts))
    ia = agj.Index(polys, agj.APPROX, 4.0)
    cells, ro, refs = ia.logical()
    _csr_equal(agj.join(ia, d).to_host(), oracle.join_approx_logical(cells, ro, refs, pts))


def test_batched_with_holes(torch, agj, oracle, holes_c1):
    from paper_1802_09488_gb300 import synth
    polys, base, eps = holes_c1
    pts = _probe_points(oracle, polys, base)
    d = _dev(torch, pts)
    plain = synth.c1_tiny(10).polygons
    ih = agj.Index(polys, agj.EXACT, 0)
    ip = agj.Index(plain, agj.EXACT, 0)
    ia = agj.Index(polys, agj.APPROX, eps)
    outs = agj.join_batched([ih, ip, ia], [d, d, d])
    _csr_equal(outs[0].to_host(), oracle.PolySet(polys).join_exact(pts))
    _csr_equal(outs[1].to_host(), oracle.PolySet(plain).join_exact(pts))
    _csr_equal(outs[2].to_host(), agj.join(ia, d).to_host())
