"""Pins for the oracle's point-polygon relation and the predicates built on it
(no GPU).

§II fixes ST_Covers as the join predicate (points on an edge or a vertex are
inside) and leaves other predicates, naming ST_Intersects, to "similar
techniques".  For a point and a polygon ST_Intersects is ST_Covers (the
point meets the closed polygon); ST_Contains excludes the boundary.  The
oracle classifies a point as exterior (0), boundary (1) or interior (2):
covers = relation > 0, contains = relation == 2.  Pinned here against closed
forms on dyadic coordinates (exact in FP64) and exact rational arithmetic.
"""
from fractions import Fraction

import numpy as np

from tests.test_oracle_pip import LSHAPE, SQUARE, _exact_on_boundary, _exact_winding


def test_square_relation_closed_form(oracle):
    cases = [((0.5, 0.5), 2), ((0.25, 0.75), 2), ((1e-300, 0.5), 2), ((0.5, 1.0 - 2 ** -40), 2),
             ((0.5, 0.0), 1), ((0.5, 1.0), 1), ((0.0, 0.5), 1), ((1.0, 0.5), 1),          # edges
             ((0.0, 0.0), 1), ((1.0, 1.0), 1), ((1.0, 0.0), 1), ((0.0, 1.0), 1),          # vertices
             ((1.5, 0.5), 0), ((-0.5, 0.5), 0), ((0.5, -1e-300), 0), ((1.0 + 2 ** -40, 0.5), 0),
             ((2.0, 0.0), 0), ((-1.0, 1.0), 0)]
    for (pu, pv), want in cases:
        assert oracle.ring_relate_uv(SQUARE, pu, pv) == want, (pu, pv)
        assert oracle.ring_relate_uv(SQUARE[::-1], pu, pv) == want, (pu, pv)
        assert oracle.ring_covers_uv(SQUARE, pu, pv) == (want > 0)


def test_lshape_relation_closed_form(oracle):
    g = np.arange(-0.25, 2.5, 0.125)
    for pu in g:
        for pv in g:
            closed = (0 <= pu <= 2 and 0 <= pv <= 1) or (0 <= pu <= 1 and 0 <= pv <= 2)
            interior = (0 < pu < 2 and 0 < pv < 1) or (0 < pu < 1 and 0 < pv < 2)
            want = 2 if interior else (1 if closed else 0)
            assert oracle.ring_relate_uv(LSHAPE, pu, pv) == want, (pu, pv)
            assert oracle.ring_relate_uv(np.roll(LSHAPE, 3, axis=0)[::-1], pu, pv) == want, (pu, pv)


def test_random_star_polygons_relation_exact_rational(oracle):
    """Dyadic rings and points (exact FP64): boundary iff exactly on an edge,
    interior iff off every edge with an odd crossing count."""
    rng = np.random.default_rng(22)
    for _ in range(40):
        V = int(rng.integers(3, 32))
        ang = np.sort(rng.uniform(0, 2 * np.pi, V))
        rad = rng.uniform(0.2, 1.0, V)
        ring = np.stack([np.round(rad * np.cos(ang) * 1024) / 1024, np.round(rad * np.sin(ang) * 1024) / 1024], -1)
        fr = [(Fraction(float(x)), Fraction(float(y))) for x, y in ring]
        pts = np.round(rng.uniform(-1.1, 1.1, (200, 2)) * 256) / 256
        pts = np.concatenate([pts, ring, 0.5 * (ring + np.roll(ring, -1, axis=0))])
        for pu, pv in pts:
            p = (Fraction(float(pu)), Fraction(float(pv)))
            want = 1 if _exact_on_boundary(fr, p) else (2 if _exact_winding(fr, p) % 2 else 0)
            assert oracle.ring_relate_uv(ring, float(pu), float(pv)) == want


def test_contains_join_drops_exactly_the_boundary_points(oracle):
    """On the tiny tiling: the ST_Contains join equals the ST_Covers join
    minus the pairs whose point lies on that polygon's boundary (vertices and
    edge midpoints are on it; uniform points almost surely are not)."""
    from paper_1802_09488_gb300 import synth
    polys = synth.c1_tiny(10).polygons
    pts = np.concatenate([synth.points_uniform(3000, synth.BOX_C1, seed=9), np.concatenate(polys)])
    cov = oracle.PolySet(polys)
    con = oracle.PolySet(polys, contains=True)
    oc, ic = cov.join_exact(pts)
    ot, it = con.join_exact(pts)
    n_uniform = 3000
    for r in range(len(pts)):
        a = set(ic[oc[r]:oc[r + 1]].tolist())
        b = set(it[ot[r]:ot[r + 1]].tolist())
        assert b <= a
        for k in a - b:
            f, u, v = oracle.face_uv(*pts[r])
            uv = cov_uv(oracle, polys[k])
            assert oracle.ring_relate_uv(uv, u, v) == 1
        if r < n_uniform:
            assert a == b
        else:
            assert a - b, "a polygon vertex lies on the boundary of its own polygon"


def cov_uv(oracle, poly):
    return np.array([oracle.face_uv(lat, lng)[1:] for lat, lng in poly])
