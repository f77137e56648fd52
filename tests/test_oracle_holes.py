"""Pins for the oracle's polygons with holes (no GPU).

A polygon with holes is its outer ring minus the interiors of its hole rings
(OGC simple-feature semantics; §II joins "simple polygons" by ST_Covers and
this widens the geometry).  The oracle's relation over rings: a point on an
edge of any ring is on the boundary (covered, not contained); otherwise it is
interior when it lies inside an odd number of rings.  Pinned against closed
forms on dyadic coordinates, exact rational arithmetic, the lat/lng join, the
geodesic distance and the covering checker.
"""
from fractions import Fraction

import numpy as np

from tests.test_oracle_pip import _exact_on_boundary, _exact_winding

OUTER = np.array([[0, 0], [4, 0], [4, 4], [0, 4]], dtype=np.float64)
HOLE = np.array([[1, 1], [1, 2], [2, 2], [2, 1]], dtype=np.float64)       # opposite orientation
HOLE2 = np.array([[2.5, 2.5], [3.5, 2.5], [3.5, 3.0], [2.5, 3.0]], dtype=np.float64)


def _want_square_with_holes(u, v, holes):
    if not (0 <= u <= 4 and 0 <= v <= 4):
        return 0
    if u in (0, 4) or v in (0, 4):
        return 1
    for h in holes:
        u0, u1, v0, v1 = h[:, 0].min(), h[:, 0].max(), h[:, 1].min(), h[:, 1].max()
        if u0 <= u <= u1 and v0 <= v <= v1:
            return 1 if (u in (u0, u1) or v in (v0, v1)) else 0
    return 2


def test_square_with_holes_closed_form(oracle):
    g = np.arange(-0.5, 4.625, 0.125)
    for holes in ([HOLE], [HOLE, HOLE2], [HOLE2[::-1], HOLE[::-1]]):
        rings = [OUTER] + list(holes)
        for u in g:
            for v in g:
                want = _want_square_with_holes(u, v, holes)
                assert oracle.rings_relate_uv(rings, u, v) == want, (u, v)
                assert oracle.rings_relate_uv([OUTER[::-1]] + list(holes), u, v) == want, (u, v)


def test_one_ring_equals_the_ring_rule(oracle):
    rng = np.random.default_rng(5)
    for _ in range(200):
        u, v = rng.uniform(-0.5, 4.5, 2)
        assert oracle.rings_relate_uv([OUTER], u, v) == oracle.ring_relate_uv(OUTER, u, v)


def _star(rng, V, cx, cy, r0, r1, scale):
    ang = np.sort(rng.uniform(0, 2 * np.pi, V))
    rad = rng.uniform(r0, r1, V)
    return np.stack([np.round((cx + rad * np.cos(ang)) * scale) / scale,
                     np.round((cy + rad * np.sin(ang)) * scale) / scale], -1)


def test_random_dyadic_polygons_with_holes_exact_rational(oracle):
    """Dyadic star-shaped outer rings with one or two dyadic star holes well
    inside them: the relation must equal exact rational arithmetic (boundary
    if exactly on an edge of any ring, else odd total winding parity)."""
    rng = np.random.default_rng(23)
    for _ in range(30):
        outer = _star(rng, int(rng.integers(6, 30)), 0.0, 0.0, 0.8, 1.0, 1024)
        holes = [_star(rng, int(rng.integers(3, 12)), cx, 0.0, 0.05, 0.2, 1024)
                 for cx in ((-0.35, 0.35) if rng.random() < 0.5 else (0.0,))]
        rings = [outer] + holes
        fr = [[(Fraction(float(x)), Fraction(float(y))) for x, y in r] for r in rings]
        pts = np.round(rng.uniform(-1.1, 1.1, (150, 2)) * 256) / 256
        near = np.round(rng.uniform(-0.6, 0.6, (150, 2)) * 256) / 256
        pts = np.concatenate([pts, near] + [r for r in rings] + [0.5 * (r + np.roll(r, -1, axis=0)) for r in rings])
        for pu, pv in pts:
            p = (Fraction(float(pu)), Fraction(float(pv)))
            if any(_exact_on_boundary(r, p) for r in fr):
                want = 1
            else:
                want = 2 if sum(_exact_winding(r, p) for r in fr) % 2 else 0
            assert oracle.rings_relate_uv(rings, float(pu), float(pv)) == want


def _latlng_square(lat0, lng0, half_deg):
    return np.array([[lat0 - half_deg, lng0 - half_deg], [lat0 - half_deg, lng0 + half_deg],
                     [lat0 + half_deg, lng0 + half_deg], [lat0 + half_deg, lng0 - half_deg]])


def test_join_distance_and_predicates_with_a_hole(oracle):
    """A lat/lng square with a square hole: points in the hole join nothing and
    lie at a positive distance no larger than the hole's half-width; points
    in the body join it at distance 0; hole vertices are covered but not
    contained."""
    outer = _latlng_square(40.70, -73.95, 0.02)
    hole = _latlng_square(40.70, -73.95, 0.005)[::-1]
    poly = [outer, hole]
    cov = oracle.PolySet([poly])
    con = oracle.PolySet([poly], contains=True)
    inside_hole = np.array([[40.70, -73.95], [40.702, -73.948], [40.6985, -73.9515]])
    body = np.array([[40.71, -73.95], [40.70, -73.935], [40.685, -73.965]])
    for lat, lng in inside_hole:
        assert not cov.covers(0, lat, lng) and not con.covers(0, lat, lng)
        d = cov.dist_m(0, lat, lng)
        assert 0.0 < d <= 0.006 * 111195.0
    for lat, lng in body:
        assert cov.covers(0, lat, lng) and con.covers(0, lat, lng)
        assert cov.dist_m(0, lat, lng) == 0.0
    for lat, lng in hole:
        assert cov.covers(0, lat, lng) and not con.covers(0, lat, lng)
    o, i = cov.join_exact(np.concatenate([inside_hole, body]))
    assert list(np.diff(o)) == [0, 0, 0, 1, 1, 1]
    # the holed polygon's join = the outer ring's join minus the hole ring's
    rng = np.random.default_rng(3)
    pts = np.stack([rng.uniform(40.675, 40.725, 4000), rng.uniform(-73.975, -73.925, 4000)], -1)
    a = oracle.PolySet([outer]).join_exact(pts)
    b = oracle.PolySet([hole]).join_exact(pts)
    c = cov.join_exact(pts)
    want = (np.diff(a[0]) == 1) & (np.diff(b[0]) == 0)
    assert np.array_equal(np.diff(c[0]) == 1, want)


def test_covering_checker_sees_the_hole(oracle):
    """A true reference on a cell inside the hole, or on a cell crossing the
    hole's ring, is reported; one on a cell of the body is not."""
    outer = _latlng_square(40.70, -73.95, 0.02)
    hole = _latlng_square(40.70, -73.95, 0.005)[::-1]
    ps = oracle.PolySet([[outer, hole]])
    L = 16
    def cell_at(lat, lng):
        return oracle.id_parent(oracle.cell_id(lat, lng), L)
    in_hole = cell_at(40.70, -73.95)
    body = cell_at(40.712, -73.95)
    on_ring = cell_at(40.705, -73.95)
    cells = sorted({in_hole, body, on_ring})
    def report(true_cells):
        refs = np.array([(0 << 1) | (1 if c in true_cells else 0) for c in cells], dtype=np.uint32)
        off = np.arange(len(cells) + 1, dtype=np.uint64)
        return ps.check_covering(np.array(cells, dtype=np.uint64), off, refs)
    assert report({body})["true_ref_not_inside"] == 0
    assert report({body, in_hole})["true_ref_not_inside"] == 1
    assert report({body, on_ring})["true_ref_not_inside"] == 1
