"""Pins for the oracle's ST_Covers predicate and joins (no GPU).

ST_Covers (§II): a polygon covers a point when the point is inside or on an
edge or vertex.  The PIP test is the ray-crossing rule (§II "PIP": odd number
of crossings = inside).  These tests pin the oracle's predicate against
closed forms on dyadic coordinates (where FP64 is exact), exact rational
winding numbers, and an independent 3-D spherical winding computation for
polygons given in lat/lng with geodesic edges.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

SQUARE = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], dtype=np.float64)
LSHAPE = np.array([[0, 0], [2, 0], [2, 1], [1, 1], [1, 2], [0, 2]], dtype=np.float64)


def test_square_closed_form(oracle):
    for pu, pv, want in [(0.5, 0.5, True), (0.25, 0.75, True), (1.5, 0.5, False), (-0.5, 0.5, False),
                         (0.5, 1.5, False), (0.5, -1e-300, False),
                         (0.5, 0.0, True), (0.5, 1.0, True), (0.0, 0.5, True), (1.0, 0.5, True),   # edges
                         (0.0, 0.0, True), (1.0, 1.0, True), (1.0, 0.0, True), (0.0, 1.0, True),   # vertices
                         (1.0 + 2 ** -40, 0.5, False), (0.5, 1.0 + 2 ** -40, False), (2.0, 0.0, False),
                         (-1.0, 1.0, False), (2.0, 1.0, False)]:
        assert oracle.ring_covers_uv(SQUARE, pu, pv) == want, (pu, pv)
        assert oracle.ring_covers_uv(SQUARE[::-1], pu, pv) == want, (pu, pv)


def test_lshape_closed_form(oracle):
    g = np.arange(-0.25, 2.5, 0.125)
    for pu in g:
        for pv in g:
            want = (0 <= pu <= 2 and 0 <= pv <= 1) or (0 <= pu <= 1 and 0 <= pv <= 2)
            assert oracle.ring_covers_uv(LSHAPE, pu, pv) == want, (pu, pv)
            assert oracle.ring_covers_uv(np.roll(LSHAPE, 2, axis=0)[::-1], pu, pv) == want


def _exact_winding(ring, p):
    """Exact winding number of a rational ring around p (p not on the ring)."""
    w = 0
    n = len(ring)
    for k in range(n):
        a, b = ring[k], ring[(k + 1) % n]
        o = (b[0] - a[0]) * (p[1] - a[1]) - (b[1] - a[1]) * (p[0] - a[0])
        if a[1] <= p[1] < b[1] and o > 0:
            w += 1
        elif b[1] <= p[1] < a[1] and o < 0:
            w -= 1
    return w


def _exact_on_boundary(ring, p):
    n = len(ring)
    for k in range(n):
        a, b = ring[k], ring[(k + 1) % n]
        o = (b[0] - a[0]) * (p[1] - a[1]) - (b[1] - a[1]) * (p[0] - a[0])
        if o == 0 and min(a[0], b[0]) <= p[0] <= max(a[0], b[0]) and min(a[1], b[1]) <= p[1] <= max(a[1], b[1]):
            return True
    return False


def test_random_star_polygons_exact_rational(oracle):
    """Dyadic vertices (k/1024) and dyadic points: every FP64 operation of the
    ring rule is exact there, so the oracle must equal exact rational
    arithmetic, boundary cases included."""
    rng = np.random.default_rng(21)
    for trial in range(60):
        V = int(rng.integers(3, 40))
        ang = np.sort(rng.uniform(0, 2 * np.pi, V))
        rad = rng.uniform(0.2, 1.0, V)
        ring = np.stack([np.round(rad * np.cos(ang) * 1024) / 1024, np.round(rad * np.sin(ang) * 1024) / 1024], -1)
        fr = [(Fraction(float(x)), Fraction(float(y))) for x, y in ring]
        pts = np.round(rng.uniform(-1.1, 1.1, (300, 2)) * 256) / 256
        pts = np.concatenate([pts, ring, 0.5 * (ring + np.roll(ring, -1, axis=0))])
        for pu, pv in pts:
            p = (Fraction(float(pu)), Fraction(float(pv)))
            want = _exact_on_boundary(fr, p) or (_exact_winding(fr, p) % 2 == 1)
            assert oracle.ring_covers_uv(ring, float(pu), float(pv)) == want


def _xyz(lat, lng):
    la, lo = math.radians(lat), math.radians(lng)
    return np.array([math.cos(la) * math.cos(lo), math.cos(la) * math.sin(lo), math.sin(la)])


def _spherical_winding(poly_latlng, lat, lng):
    """Sum of signed angles at p subtended by the geodesic edges, in turns."""
    p = _xyz(lat, lng)
    tot = 0.0
    n = len(poly_latlng)
    for k in range(n):
        a = _xyz(*poly_latlng[k]); b = _xyz(*poly_latlng[(k + 1) % n])
        # tangent-plane directions at p towards a and b
        ta = a - np.dot(a, p) * p
        tb = b - np.dot(b, p) * p
        ang = math.atan2(np.dot(np.cross(ta, tb), p), np.dot(ta, tb))
        tot += ang
    return tot / (2 * math.pi)


def _dist_to_edges_rad(poly_latlng, lat, lng):
    p = _xyz(lat, lng)
    best = 10.0
    n = len(poly_latlng)
    for k in range(n):
        a = _xyz(*poly_latlng[k]); b = _xyz(*poly_latlng[(k + 1) % n])
        nrm = np.cross(a, b); nrm /= np.linalg.norm(nrm)
        best = min(best, abs(math.asin(np.clip(np.dot(p, nrm), -1, 1))),
                   math.acos(np.clip(np.dot(p, a), -1, 1)), math.acos(np.clip(np.dot(p, b), -1, 1)))
    return best


@pytest.mark.parametrize("centre", [(40.7, -73.95), (10.0, 20.0), (-35.0, 150.0), (60.0, -10.0), (75.0, 40.0)])
def test_spherical_winding_crosscheck(oracle, centre):
    """ST_Covers in face (u,v) with straight edges == containment by geodesic
    edges on the sphere (gnomonic projection maps great circles to lines)."""
    rng = np.random.default_rng(int(abs(centre[0] * 100 + centre[1])))
    for trial in range(6):
        V = int(rng.integers(5, 30))
        ang = np.sort(rng.uniform(0, 2 * np.pi, V))
        rad = rng.uniform(0.05, 0.4, V)
        poly = np.stack([centre[0] + rad * np.sin(ang), centre[1] + rad * np.cos(ang)], -1)
        ps = oracle.PolySet([poly])
        if ps.face(0) < 0:
            continue
        pts = np.stack([centre[0] + rng.uniform(-0.5, 0.5, 300), centre[1] + rng.uniform(-0.5, 0.5, 300)], -1)
        for lat, lng in pts:
            if _dist_to_edges_rad(poly, lat, lng) < 1e-9:
                continue
            w = _spherical_winding(poly, lat, lng)
            want = abs(round(w)) == 1
            assert abs(w - round(w)) < 1e-6
            assert ps.covers(0, float(lat), float(lng)) == want


def test_tiling_covers_every_point(oracle):
    """c1's five polygons tile the box: every point of the box is covered by
    at least one polygon, and by two or more only on shared boundaries.
    The box's north and south sides are parallels of latitude while polygon
    edges are geodesics, which bow poleward by up to L^2 tan(lat) / (8 R)
    (a few metres for the subdivided sides); points in that sliver are
    uncovered, so a 50 m band along those two sides is excluded."""
    from paper_1802_09488_gb300 import synth
    w = synth.c1_tiny(20000)
    ps = oracle.PolySet(w.polygons)
    offs, ids = ps.join_exact(w.points)
    cnt = np.diff(offs.astype(np.int64))
    lat_lo, lat_hi, _, _ = synth.BOX_C1.latlng_bounds()
    band = 50.0 / synth.M_PER_DEG
    inner = (w.points[:, 0] > lat_lo + band) & (w.points[:, 0] < lat_hi - band)
    assert cnt[inner].min() >= 1
    assert (cnt == 0).sum() <= 20
    assert (cnt > 1).sum() <= 2        # measure-zero boundary hits only
    # brute force over all polygons, no grid, on a sample
    for k in range(0, 20000, 97):
        got = list(ids[offs[k]:offs[k + 1]])
        assert got == ps.hits_brute(*w.points[k])


def test_grid_join_equals_brute_force_random(oracle):
    rng = np.random.default_rng(22)
    polys = []
    for k in range(25):
        c = (40.0 + rng.uniform(-0.3, 0.3), -74.0 + rng.uniform(-0.3, 0.3))
        V = int(rng.integers(3, 20))
        ang = np.sort(rng.uniform(0, 2 * np.pi, V))
        rad = rng.uniform(0.01, 0.2, V)
        polys.append(np.stack([c[0] + rad * np.sin(ang), c[1] + rad * np.cos(ang)], -1))
    ps = oracle.PolySet(polys, grid_n=7)
    pts = np.stack([40.0 + rng.uniform(-0.6, 0.6, 3000), -74.0 + rng.uniform(-0.6, 0.6, 3000)], -1)
    pts[:20] = np.concatenate(polys)[:20]          # some points exactly on vertices
    offs, ids = ps.join_exact(pts, threads=3)
    for k in range(len(pts)):
        assert list(ids[offs[k]:offs[k + 1]]) == ps.hits_brute(*pts[k])


def test_polygon_wider_than_the_cap_is_rejected(oracle):
    """Polygons spanning cube faces are supported within 15 degrees of their
    vertices' mean (tests/test_oracle_crossface.py); a wider one joins
    nothing."""
    ps = oracle.PolySet([np.array([[0.0, 30.0], [20.0, 45.0], [-20.0, 60.0]])])
    assert ps.face(0) == -1
    assert not ps.covers(0, 0.0, 45.0)


def test_distance_zero_inside_and_edge_distance(oracle):
    """Distance from a point to a polygon's geodesic edge, against dense
    sampling of that edge (straight in (u,v)) with mpmath great circles."""
    import mpmath
    with mpmath.workprec(100):          # leaves the precision other tests set unchanged
        _distance_against_sampling(oracle, mpmath)


def _distance_against_sampling(oracle, mpmath):
    poly = np.array([[40.60, -74.05], [40.60, -73.85], [40.80, -73.85], [40.80, -74.05]])
    ps = oracle.PolySet([poly])
    assert ps.dist_m(0, 40.7, -73.95) == 0.0
    f, ua, va = oracle.face_uv(40.80, -74.05)
    _, ub, vb = oracle.face_uv(40.80, -73.85)
    for lat, lng in [(40.8005, -73.95), (40.81, -73.90), (40.9, -74.2), (40.85, -73.80)]:
        got = ps.dist_m(0, lat, lng)
        p = [mpmath.cos(mpmath.radians(lat)) * mpmath.cos(mpmath.radians(lng)),
             mpmath.cos(mpmath.radians(lat)) * mpmath.sin(mpmath.radians(lng)), mpmath.sin(mpmath.radians(lat))]
        best = mpmath.inf
        # nearest point on any of the four edges by sampling in (u,v), refined
        # around the coarse minimum (edges are straight in (u,v) on face 4)
        corners = [oracle.face_uv(*c)[1:] for c in poly]

        def ang_at(e, t):
            (u0, v0), (u1, v1) = corners[e], corners[(e + 1) % 4]
            u = mpmath.mpf(u0) + t * (mpmath.mpf(u1) - u0)
            v = mpmath.mpf(v0) + t * (mpmath.mpf(v1) - v0)
            q = [v, mpmath.mpf(-1), -u]
            nq = mpmath.sqrt(sum(c ** 2 for c in q))
            dot = sum(p[k] * q[k] / nq for k in range(3))
            return mpmath.acos(min(dot, 1))

        assert f == 4
        for e in range(4):
            ts = [mpmath.mpf(t) for t in np.linspace(0, 1, 201)]
            lo, hi = mpmath.mpf(0), mpmath.mpf(1)
            for _ in range(6):
                vals = [ang_at(e, t) for t in ts]
                k = int(np.argmin([float(x) for x in vals]))
                best = min(best, vals[k])
                step = (hi - lo) / (len(ts) - 1)
                lo, hi = max(mpmath.mpf(0), ts[k] - step), min(mpmath.mpf(1), ts[k] + step)
                ts = [lo + (hi - lo) * i / 40 for i in range(41)]
        want = float(best) * 6371008.8
        assert abs(got - want) <= max(1e-6 * want, 1e-4), (lat, lng, got, want)


def test_logical_probe_matches_linear_scan(oracle):
    """Sorted-vector binary search (§II) over a hand-built disjoint covering
    equals a linear scan for the unique containing cell."""
    rng = np.random.default_rng(23)
    base = oracle.cell_id(40.7, -73.95)
    cells = set()
    for L in (8, 10, 12, 13, 17, 22, 30):
        for _ in range(30):
            d = int(rng.integers(-(1 << 50), 1 << 50)) * 2
            c = oracle.id_parent(base + d, L)
            cells.add(c)
    # keep a disjoint subset
    keep = []
    for c in sorted(cells, key=lambda c: oracle.id_level(c)):
        lo, hi = oracle.id_range(c)
        if all(hi < oracle.id_range(k)[0] or lo > oracle.id_range(k)[1] for k in keep):
            keep.append(c)
    keep = np.array(sorted(keep), dtype=np.uint64)
    for c in keep:
        assert oracle.logical_find(keep, int(c)) == int(np.searchsorted(keep, c))
        lo, hi = oracle.id_range(int(c))
        assert oracle.logical_find(keep, lo) == int(np.searchsorted(keep, c))
        assert oracle.logical_find(keep, hi) == int(np.searchsorted(keep, c))
    for _ in range(3000):
        q = oracle.id_parent(base + int(rng.integers(-(1 << 50), 1 << 50)) * 2, 30)
        want = -1
        for k, c in enumerate(keep):
            lo, hi = oracle.id_range(int(c))
            if lo <= q <= hi:
                want = k
        assert oracle.logical_find(keep, q) == want
