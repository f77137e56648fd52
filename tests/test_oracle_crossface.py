"""Pins for the oracle's polygons spanning cube faces (no GPU).

§II's polygons have geodesic edges; a polygon whose vertices lie on more
than one face is tested in its own gnomonic plane about the normalised mean
of its vertices (geodesics are straight lines in any gnomonic projection
that sees the whole polygon), a plane unrelated to the cube faces the
product splits such polygons along.  Pinned against closed forms around a
cube edge, an independent spherical winding number with 3-D geodesic
distances, and the covering checker on the faces' planes.
"""
import math

import numpy as np
import pytest

from tests.test_oracle_pip import _dist_to_edges_rad, _spherical_winding

TRIANGLE = np.array([[0.0, 44.0], [1.0, 46.0], [-1.0, 46.0]])     # straddles lng 45 (faces 0 and 1)


def test_triangle_across_a_cube_edge_closed_form(oracle):
    ps = oracle.PolySet([TRIANGLE])
    assert ps.face(0) == 6
    assert oracle.face_uv(0.0, 44.5)[0] == 0 and oracle.face_uv(0.0, 45.5)[0] == 1
    for lat, lng, want in [(0.0, 44.5, True), (0.0, 45.5, True), (0.0, 45.0, True), (0.2, 45.9, True),
                           (0.0, 43.5, False), (0.0, 46.5, False), (0.9, 45.0, False), (-0.9, 45.0, False)]:
        assert ps.covers(0, lat, lng) == want, (lat, lng)
    for lat, lng in TRIANGLE:                          # vertices: boundary
        assert ps.covers(0, lat, lng)
        assert not oracle.PolySet([TRIANGLE], contains=True).covers(0, lat, lng)


def _star(rng, clat, clng, r_deg, V):
    ang = np.sort(rng.uniform(0, 2 * np.pi, V))
    rad = rng.uniform(0.4, 1.0, V) * r_deg
    return np.stack([clat + rad * np.sin(ang), clng + rad * np.cos(ang) / math.cos(math.radians(clat))], -1)


@pytest.mark.parametrize("centre", [(0.0, 45.0), (35.26, 45.0), (0.0, -135.0), (-35.26, -45.0), (60.0, 0.0)])
def test_crossface_against_spherical_winding(oracle, centre):
    """Star polygons around cube edges and corners (2-3 faces): covered iff
    the spherical winding number is odd, for points clear of the edges."""
    rng = np.random.default_rng(abs(hash(centre)) % 2**32)
    for trial in range(6):
        poly = _star(rng, centre[0], centre[1], rng.uniform(0.5, 3.0), int(rng.integers(5, 24)))
        faces = {oracle.face_uv(la, lo)[0] for la, lo in poly}
        ps = oracle.PolySet([poly])
        if len(faces) == 1:
            assert ps.face(0) == faces.pop()
            continue
        assert ps.face(0) == 6
        span = 1.3 * (np.abs(poly - centre).max())
        pts = np.stack([centre[0] + rng.uniform(-span, span, 400),
                        centre[1] + rng.uniform(-span, span, 400) / math.cos(math.radians(centre[0]))], -1)
        for lat, lng in pts:
            if _dist_to_edges_rad(poly, lat, lng) < 1e-9:
                continue
            w = _spherical_winding(poly, lat, lng)
            assert abs(w - round(w)) < 1e-6
            assert ps.covers(0, lat, lng) == (round(w) % 2 != 0), (lat, lng, w)


def _xyz(lat, lng):
    la, lo = math.radians(lat), math.radians(lng)
    return np.array([math.cos(la) * math.cos(lo), math.cos(la) * math.sin(lo), math.sin(la)])


def _dist_to_arcs_rad(poly, lat, lng):
    """Angle from p to the nearest point of the polygon's geodesic edges: the
    perpendicular when its foot lies on the arc, else the nearer end."""
    p = _xyz(lat, lng)
    best = 10.0
    for k in range(len(poly)):
        a, b = _xyz(*poly[k]), _xyz(*poly[(k + 1) % len(poly)])
        n = np.cross(a, b); n /= np.linalg.norm(n)
        foot = p - np.dot(p, n) * n
        foot /= np.linalg.norm(foot)
        on_arc = np.dot(np.cross(a, foot), n) >= 0 and np.dot(np.cross(foot, b), n) >= 0
        d = abs(math.asin(np.clip(np.dot(p, n), -1, 1))) if on_arc else \
            min(math.acos(np.clip(np.dot(p, a), -1, 1)), math.acos(np.clip(np.dot(p, b), -1, 1)))
        best = min(best, d)
    return best


def test_crossface_distance(oracle):
    ps = oracle.PolySet([TRIANGLE])
    assert ps.dist_m(0, 0.0, 45.0) == 0.0
    for lat, lng in [(0.0, 43.0), (0.0, 47.0), (2.0, 45.0), (-1.5, 46.5), (0.0, 44.9 - 1e-3)]:
        want = _dist_to_arcs_rad(TRIANGLE, lat, lng) * 6371008.8
        if ps.covers(0, lat, lng):
            assert ps.dist_m(0, lat, lng) == 0.0
        else:
            assert abs(ps.dist_m(0, lat, lng) - want) <= 1e-6 * want, (lat, lng)


def test_crossface_holes_and_join(oracle):
    """A polygon across the cube edge with a hole across the same edge: the
    hole's points join nothing; the join equals brute force and the
    outer-minus-hole relation."""
    outer = np.array([[-2.0, 43.0], [-2.0, 47.0], [2.0, 47.0], [2.0, 43.0]])
    hole = np.array([[-0.5, 44.5], [0.5, 44.5], [0.5, 45.5], [-0.5, 45.5]])
    ps = oracle.PolySet([[outer, hole], TRIANGLE])
    assert ps.face(0) == 6 and ps.face(1) == 6
    rng = np.random.default_rng(4)
    pts = np.stack([rng.uniform(-2.5, 2.5, 3000), rng.uniform(42.5, 47.5, 3000)], -1)
    o, ids = ps.join_exact(pts)
    a = oracle.PolySet([outer]).join_exact(pts)
    h = oracle.PolySet([hole]).join_exact(pts)
    t = oracle.PolySet([TRIANGLE]).join_exact(pts)
    for r in range(len(pts)):
        want = []
        if a[0][r + 1] > a[0][r] and not h[0][r + 1] > h[0][r]:
            want.append(0)
        if t[0][r + 1] > t[0][r]:
            want.append(1)
        assert list(ids[o[r]:o[r + 1]]) == want
        assert list(ids[o[r]:o[r + 1]]) == ps.hits_brute(*pts[r])


def test_covering_checker_on_both_faces(oracle):
    """Cells of either face under the triangle: true references on cells well
    inside pass; on a cell crossing an edge, or outside, they are flagged."""
    ps = oracle.PolySet([TRIANGLE])
    L = 12
    def cell(lat, lng):
        return oracle.id_parent(oracle.cell_id(lat, lng), L)
    inside0, inside1 = cell(0.0, 44.6), cell(0.0, 45.4)
    crossing = cell(0.625, 45.25)      # the triangle's upper edge passes here
    outside = cell(0.0, 47.0)
    for c, bad in [(inside0, 0), (inside1, 0), (crossing, 1), (outside, 1)]:
        rep = ps.check_covering(np.array([c], dtype=np.uint64), np.array([0, 1], dtype=np.uint64),
                                np.array([1], dtype=np.uint32))
        assert rep["true_ref_not_inside"] == bad, (c, rep)
        assert rep["bad_ref"] == 0
    # a candidate reference on a far cell misses the polygon
    rep = ps.check_covering(np.array([cell(0.0, 50.0)], dtype=np.uint64), np.array([0, 1], dtype=np.uint64),
                            np.array([0], dtype=np.uint32))
    assert rep["cand_ref_misses"] == 1
