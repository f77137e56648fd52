"""Test inputs near polygon boundaries, and the approximate join's precision
check (§III-A) written with the oracle's pieces.

Polygon edges are geodesics, i.e. straight segments in the polygon's face
(u,v) plane (gnomonic projection).  Points "on" an edge are taken on that
segment and points "off" it are moved perpendicular to it in (u,v), by a
distance in metres converted with the oracle's great-circle distance.  The
(lat, lng) of a (u,v) point comes from the inverse of the face projection
(the face table of S2's published convention).  Rounding to (lat, lng)
doubles moves a point by about a nanometre, which is far below the 1 µm
offsets.
"""
import numpy as np

_FACE_XYZ = {
    0: lambda u, v: (np.ones_like(u), u, v),
    1: lambda u, v: (-u, np.ones_like(u), v),
    2: lambda u, v: (-u, -v, np.ones_like(u)),
    3: lambda u, v: (-np.ones_like(u), -v, -u),
    4: lambda u, v: (v, -np.ones_like(u), -u),
    5: lambda u, v: (v, u, -np.ones_like(u)),
}


def face_uv_to_latlng(face, u, v):
    x, y, z = _FACE_XYZ[face](np.asarray(u, dtype=np.float64), np.asarray(v, dtype=np.float64))
    lat = np.degrees(np.arctan2(z, np.hypot(x, y)))
    lng = np.degrees(np.arctan2(y, x))
    return np.stack([lat, lng], -1)


def edge_points(oracle, polys, offsets_m=(0.0, 1e-6, -1e-6), ts=(0.5, 0.25), with_vertices=True, stride=1):
    """For every `stride`-th edge of every polygon: the points at parameters
    ts along it, moved by each of offsets_m metres along its (u,v) normal;
    plus every vertex.  Returns an (N, 2) array of (lat, lng)."""
    out = []
    for P in polys:
        P = np.asarray(P, dtype=np.float64)
        uv = np.array([oracle.face_uv(la, lo)[1:] for la, lo in P])
        face = oracle.face_uv(*P[0])[0]
        if with_vertices:
            out.append(P)
        for k in range(0, len(P), stride):
            a, b = uv[k], uv[(k + 1) % len(P)]
            d = b - a
            L = float(np.hypot(d[0], d[1]))
            if L == 0.0:
                continue
            m_per_uv = oracle.uv_dist_m(face, a[0], a[1], b[0], b[1]) / L
            nrm = np.array([-d[1], d[0]]) / L
            for t in ts:
                p = a + t * d
                for off in offsets_m:
                    q = p + nrm * (off / m_per_uv)
                    out.append(face_uv_to_latlng(face, q[0:1], q[1:2]))
    return np.concatenate(out)


def check_approx_property(oracle, ps, cells, off, refs, points, eps_m):
    """§III-A on `points`: the approximate result read off the logical
    covering (sorted-vector probe) contains every exact pair (brute force),
    and each extra pair's point lies within eps of the polygon by geodesic
    distance.  Returns (exact pairs, false-positive pairs, worst distance)."""
    ao, ai = oracle.join_approx_logical(cells, off, refs, points)
    eo, ei = ps.join_exact(points)
    a_row = np.repeat(np.arange(len(points), dtype=np.uint64), np.diff(ao.astype(np.int64)))
    e_row = np.repeat(np.arange(len(points), dtype=np.uint64), np.diff(eo.astype(np.int64)))
    akey = (a_row << np.uint64(32)) | ai.astype(np.uint64)
    ekey = (e_row << np.uint64(32)) | ei.astype(np.uint64)
    missing = ~np.isin(ekey, akey)
    assert not missing.any(), f"{int(missing.sum())} exact pairs missing from the approximate join, " \
                              f"first point {int(e_row[missing][0])}"
    extra = akey[~np.isin(akey, ekey)]
    worst = 0.0
    for key in extra:
        p, q = int(key >> np.uint64(32)), int(key & np.uint64(0xFFFFFFFF))
        d = ps.dist_m(q, *points[p])
        # a point on an edge shared by two polygons is covered by one of them;
        # its distance to the other can round to 0 m
        assert 0.0 <= d <= eps_m * (1 + 1e-9), (p, q, d)
        worst = max(worst, d)
    return len(ekey), len(extra), worst


def edge_points_3d(polys, offsets_m=(0.0, 1e-6, -1e-6), ts=(0.5, 0.25), stride=1):
    """Like edge_points for polygons that may span cube faces: points on each
    geodesic edge (normalised chords between the vertices' unit vectors) and
    moved by offsets_m metres along the edge's great-circle normal, plus
    every vertex.  (lat, lng) rows."""
    R = 6371008.8
    out = []
    for P in polys:
        P = np.asarray(P, dtype=np.float64)
        la, lo = np.radians(P[:, 0]), np.radians(P[:, 1])
        xyz = np.stack([np.cos(la) * np.cos(lo), np.cos(la) * np.sin(lo), np.sin(la)], -1)
        out.append(P)
        for k in range(0, len(P), stride):
            a, b = xyz[k], xyz[(k + 1) % len(P)]
            n = np.cross(a, b)
            if np.linalg.norm(n) == 0.0:
                continue
            n /= np.linalg.norm(n)
            for t in ts:
                p = (1 - t) * a + t * b
                p /= np.linalg.norm(p)
                for off in offsets_m:
                    q = p + n * (off / R)
                    q /= np.linalg.norm(q)
                    out.append(np.array([[np.degrees(np.arcsin(q[2])), np.degrees(np.arctan2(q[1], q[0]))]]))
    return np.concatenate(out)
