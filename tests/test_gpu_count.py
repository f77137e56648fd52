"""GPU parity of the aggregation mode (count(*) group by polygon, §V; the
SIMD aggregation of §IV), called through the C ABI, against the oracle.

The count of polygon P is the number of points whose join pairs include P,
so it is compared exactly (integers) with the histogram of the oracle's
join: the sorted-vector probe of the index's logical covering for the
approximate mode, brute-force ST_Covers for the exact mode.  It is also
compared with the histogram of the library's own CSR join on the same
points.  The cases cover the shared-memory histogram (up to 4096 polygons)
and the global one (more polygons), cells with more than two references
(lookup table), ragged sizes, accumulation over calls, and the 1e8-point
city workload in the benchmark's launch configuration.
"""
import numpy as np
import pytest

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


def _oracle_counts(oracle, ix, polys, pts, mode, agj):
    if mode == agj.APPROX:
        cells, ro, refs = ix.logical()
        return oracle.count_approx_logical(cells, ro, refs, pts, len(polys))
    return oracle.PolySet(polys).count_exact(pts)


def _check(torch, agj, oracle, polys, pts, mode, eps=10.0, train=None):
    ix = agj.Index(polys, mode, eps, train=train)
    d = _dev(torch, pts)
    c = agj.join_count(ix, d)
    got = c.to_host()
    want = _oracle_counts(oracle, ix, polys, pts, mode, agj)
    assert np.array_equal(got, want)
    st = c.status.cpu().numpy().view(np.uint64)
    assert st[0] == want.sum() and st[1] == 0
    # the same as the histogram of the library's own CSR join
    _, ids = agj.join(ix, d).to_host()
    assert np.array_equal(got, np.bincount(ids, minlength=len(polys)).astype(np.uint64))
    return ix, c


@pytest.fixture(scope="module")
def c1():
    from paper_1802_09488_gb300 import synth
    return synth.c1_tiny(100_000)


@pytest.mark.parametrize("mode", ["approx", "exact"])
def test_c1_counts(torch, agj, oracle, c1, mode):
    m = agj.APPROX if mode == "approx" else agj.EXACT
    _, c = _check(torch, agj, oracle, c1.polygons, c1.points, m, c1.eps_m,
                  train=c1.points[:1000] if m == agj.EXACT else None)
    if m == agj.EXACT:
        assert c.status.cpu().numpy()[2] > 0          # candidates were refined


@pytest.mark.parametrize("n", [0, 1, 31, 1025, 65537])
def test_ragged_sizes_and_accumulate(torch, agj, oracle, c1, n):
    for mode in (agj.APPROX, agj.EXACT):
        ix = agj.Index(c1.polygons, mode, c1.eps_m)
        pts = c1.points[:n].reshape(-1, 2)
        d = _dev(torch, pts)
        c = agj.join_count(ix, d)
        want = _oracle_counts(oracle, ix, c1.polygons, pts, mode, agj)
        assert np.array_equal(c.to_host(), want)
        agj.join_count(ix, d, c, accumulate=True)          # adds the same counts again
        assert np.array_equal(c.to_host(), 2 * want)
        agj.join_count(ix, d, c)                           # overwrites
        assert np.array_equal(c.to_host(), want)


def test_boundary_and_invalid_points(torch, agj, oracle, c1):
    verts = np.concatenate(c1.polygons)
    mids = np.concatenate([0.5 * (p + np.roll(p, -1, axis=0)) for p in c1.polygons])
    extra = np.array([[np.nan, -73.9], [40.7, np.inf], [95.0, 0.0], [10.0, 20.0], [40.7, -73.95]])
    pts = np.concatenate([verts, mids, extra, c1.points[:3000]])
    for mode in (agj.APPROX, agj.EXACT):
        _check(torch, agj, oracle, c1.polygons, pts, mode, c1.eps_m)


def test_city_counts_2m(torch, agj, oracle):
    from paper_1802_09488_gb300 import synth
    w = synth.c2_city(2_000_000, n_train=200_000)
    _check(torch, agj, oracle, w.polygons, w.points, agj.APPROX, w.eps_m)
    _check(torch, agj, oracle, w.polygons, w.points, agj.EXACT, train=w.train)


@pytest.mark.parametrize("mode,eps", [("approx", 10.0), ("exact", 0.0)])
def test_fine_polygons_global_histogram(torch, agj, oracle, mode, eps):
    """9000 overlapping polygons: more than the shared-memory histogram
    holds, so the warps add to the global counts directly."""
    from paper_1802_09488_gb300 import synth
    polys = synth.c3_fine_polygons(9000, seed=8)
    pts = synth.points_mixture(300_000, synth.BOX_CITY, seed=9, dist_seed=8)
    train = synth.points_mixture(20_000, synth.BOX_CITY, seed=10, dist_seed=8)
    m = agj.APPROX if mode == "approx" else agj.EXACT
    _check(torch, agj, oracle, polys, pts, m, eps, train=train if m == agj.EXACT else None)


def test_lookup_table_cells(torch, agj, oracle):
    """300 copies of one triangle: every cell inside holds 300 references
    (lookup-table entries); every polygon gets the same count."""
    tri = np.array([[40.700, -73.950], [40.702, -73.950], [40.700, -73.947]])
    polys = [tri] * 300
    rng = np.random.default_rng(5)
    pts = np.stack([rng.uniform(40.6995, 40.7025, 5000), rng.uniform(-73.9505, -73.9465, 5000)], -1)
    for mode in (agj.APPROX, agj.EXACT):
        _, c = _check(torch, agj, oracle, polys, pts, mode, 10.0)
        got = c.to_host()
        assert got.min() == got.max() > 100


def test_city_full_size(torch, agj, oracle):
    """1e8 city points in the benchmark's launch configuration: counts equal
    the histogram of the library's CSR join on every polygon, and the
    oracle's counts scaled from a 2e6-point prefix agree within sampling
    noise; the prefix itself is compared exactly."""
    from paper_1802_09488_gb300 import synth
    w = synth.c2_city(100_000_000, n_train=1_000_000)
    d = _dev(torch, w.points)
    for mode in (agj.APPROX, agj.EXACT):
        ix = agj.Index(w.polygons, mode, w.eps_m, train=w.train if mode == agj.EXACT else None)
        got = agj.join_count(ix, d).to_host()
        pr = agj.join(ix, d)
        nnz = pr.check()
        ids = pr.ids[:nnz]
        hist = torch.bincount(ids.long(), minlength=len(w.polygons)).cpu().numpy().astype(np.uint64)
        assert np.array_equal(got, hist)
        del pr, ids
        pre = w.points[:2_000_000]
        want = _oracle_counts(oracle, ix, w.polygons, pre, mode, agj)
        assert np.array_equal(agj.join_count(ix, d[:2_000_000]).to_host(), want)
        del ix
        torch.cuda.empty_cache()
