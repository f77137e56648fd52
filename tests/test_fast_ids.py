"""The certified fast cell-id step (FP32 model + error bound) on the host.

The probe kernels compute leaf ids from an FP32 model of the spec's (s,t)
with a bound on its error, and trust only the levels on which both ends of
the error interval agree.  The host runs the same arithmetic
(agj_fast_ids_host); these tests check it against the oracle's FP64 ids:
every certified prefix equals the oracle's, points reported outside the
model's window lie in no indexed cell, and almost all points certify the
levels the trie walk needs."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def agj():
    import paper_1802_09488_gb300 as m
    m.lib()
    return m


def _prefix_equal(a, b, levels):
    """Leading `levels` levels (3 face bits + 2 bits per level) equal."""
    a = a.astype(np.uint64)
    b = b.astype(np.uint64)
    bits = (3 + 2 * levels.astype(np.uint64))
    sh = (np.uint64(64) - bits)
    mask = np.where(bits >= 64, np.uint64(0xFFFFFFFFFFFFFFFF),
                    ~((np.uint64(1) << sh) - np.uint64(1)))
    return (a & mask) == (b & mask)


@pytest.mark.parametrize("which", ["c1", "c2"])
def test_certified_prefix_equals_oracle(agj, oracle, which):
    from paper_1802_09488_gb300 import synth
    if which == "c1":
        polys, box, eps = synth.c1_tiny(10).polygons, synth.BOX_C1, 10.0
        pts = synth.points_uniform(400_000, box, seed=41)
    else:
        polys, box, eps = synth.c2_city_polygons(), synth.BOX_CITY, 4.0
        pts = synth.points_mixture(400_000, box, seed=42, dist_seed=3)
    ix = agj.Index(polys, agj.APPROX, eps, host_only=True)
    st = ix.stats()
    assert st["fast_ids"] == 1 and 0 < st["fast_err_cells"] < 0.05
    # points of the workload, a wider ring around the box, and exact grid points
    rng = np.random.default_rng(43)
    lat_lo, lat_hi, lng_lo, lng_hi = box.latlng_bounds()
    ring = np.stack([rng.uniform(lat_lo - 0.2, lat_hi + 0.2, 200_000), rng.uniform(lng_lo - 0.2, lng_hi + 0.2, 200_000)], -1)
    grid = np.stack(np.meshgrid(np.linspace(lat_lo, lat_hi, 300), np.linspace(lng_lo, lng_hi, 300)), -1).reshape(-1, 2)
    allp = np.concatenate([pts, ring, grid])
    ids, lv = ix.fast_ids_host(allp)
    ref = oracle.cell_ids(allp)
    inside = lv != 255
    assert _prefix_equal(ids[inside], ref[inside], lv[inside]).all()
    # outside the window: no indexed cell holds the point
    cells, _, _ = ix.logical()
    for cid in ref[~inside][::50]:
        assert oracle.logical_find(cells, int(cid)) == -1
    # the walk needs at most level 24 here; nearly every point certifies it
    frac = np.mean(lv[:len(pts)] >= 24)
    assert frac > 0.995, frac


def test_fast_model_disabled_option(agj):
    from paper_1802_09488_gb300 import synth
    ix = agj.Index(synth.c1_tiny(10).polygons, agj.APPROX, 10.0, host_only=True, fast_ids=False)
    assert ix.stats()["fast_ids"] == 0
    with pytest.raises(agj.AgjError):
        ix.fast_ids_host(np.zeros((1, 2)))


def test_fast_model_off_for_wide_windows(agj):
    """Polygons spread over more than a degree: no model (FP64 ids)."""
    polys = [np.array([[40.0, -74.0], [40.01, -74.0], [40.0, -73.99]]),
             np.array([[42.5, -71.0], [42.51, -71.0], [42.5, -70.99]])]
    ix = agj.Index(polys, agj.APPROX, 10.0, host_only=True)
    assert ix.stats()["fast_ids"] == 0


def test_certified_refine_equals_oracle(agj, oracle):
    """The certified FP32 ST_Covers test, where it decides, equals the
    oracle's FP64 predicate; random points are almost all decided, points
    a few micrometres from an edge or on a vertex are left undecided."""
    from paper_1802_09488_gb300 import synth
    polys = synth.c2_city_polygons()
    ix = agj.Index(polys, agj.EXACT, 0, host_only=True)
    ps = oracle.PolySet(polys)
    rng = np.random.default_rng(45)
    pts, pid = [], []
    # random points against a random polygon and against the polygons covering them
    cand = synth.points_mixture(20000, synth.BOX_CITY, seed=46, dist_seed=3)
    for k in range(len(cand)):
        q = int(rng.integers(0, len(polys)))
        pts.append(cand[k]); pid.append(q)
        hits = ps.hits_brute(*cand[k])
        for h in hits:
            pts.append(cand[k]); pid.append(h)
    n_random_pairs = len(pts)
    # points near edges: edge midpoints offset by 1e-4 .. 1e-11 degree, and vertices
    for q in rng.choice(len(polys), 60, replace=False):
        P = polys[q]
        for t in range(0, len(P), max(1, len(P) // 8)):
            a, b = P[t], P[(t + 1) % len(P)]
            m = 0.5 * (a + b)
            d = np.array([-(b - a)[1], (b - a)[0]])
            d /= np.linalg.norm(d)
            for off in (1e-4, 1e-6, 1e-8, 1e-9, 1e-10, 1e-11, -1e-11, -1e-9, -1e-6, -1e-4):
                pts.append(m + off * d); pid.append(q)
            pts.append(a.copy()); pid.append(q)
    pts = np.array(pts); pid = np.array(pid, dtype=np.uint32)
    got = ix.covers_certified_host(pts, pid)
    want = np.array([ps.covers(int(q), *p) for p, q in zip(pts, pid)], dtype=np.int8)
    decided = got >= 0
    assert np.array_equal(got[decided], want[decided])
    n_rand = n_random_pairs
    assert np.mean(decided[:n_rand]) > 0.999
    assert (~decided).sum() > 0          # the near-edge points exercise the fallback


def test_banded_refine_equals_all_edges(agj):
    """The band tables only skip edges that cannot change the certified
    test's answer: with and without them every (point, polygon) pair gets
    the same 1 / 0 / undecided answer, near edges and vertices included."""
    from paper_1802_09488_gb300 import synth
    polys = synth.c2_city_polygons()
    with_b = agj.Index(polys, agj.EXACT, 0, host_only=True)
    without = agj.Index(polys, agj.EXACT, 0, host_only=True, pip_bands=False)
    rng = np.random.default_rng(47)
    pts, pid = [], []
    cand = synth.points_mixture(30000, synth.BOX_CITY, seed=48, dist_seed=3)
    for k in range(len(cand)):
        pts.append(cand[k]); pid.append(int(rng.integers(0, len(polys))))
    for q in rng.choice(len(polys), 80, replace=False):
        P = polys[q]
        lat0, lat1 = P[:, 0].min(), P[:, 0].max()
        lng0, lng1 = P[:, 1].min(), P[:, 1].max()
        for _ in range(200):     # inside the bbox: every band, near band edges too
            pts.append(np.array([rng.uniform(lat0, lat1), rng.uniform(lng0, lng1)])); pid.append(q)
        for t in range(len(P)):  # vertices and points just off them in latitude
            for off in (0.0, 1e-12, -1e-12, 1e-9, -1e-9, 1e-7):
                pts.append(P[t] + np.array([off, 0.0])); pid.append(q)
    pts = np.array(pts); pid = np.array(pid, dtype=np.uint32)
    a = with_b.covers_certified_host(pts, pid)
    b = without.covers_certified_host(pts, pid)
    assert np.array_equal(a, b)
    assert (a == 1).sum() > 1000 and (a == -1).sum() > 0
