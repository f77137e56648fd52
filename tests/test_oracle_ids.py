"""Pins for the oracle's cell-id map (no GPU).

Each check ties the oracle to something other than itself: mpmath at high
precision, closed forms of the cube-face layout (§II "Google S2": three face
bits, bit pairs per level, one marker bit), exhaustive enumeration of small
levels (Hilbert continuity, decode round trips) and the prefix property that
children share their parent's prefix (§II "Space-filling curves").
"""
import math

import mpmath
import numpy as np
import pytest

mpmath.mp.prec = 200


def ulp(x: float) -> float:
    return math.ulp(x) if x != 0 else math.ulp(0.0)


def _mp_sincosd(d):
    with mpmath.workprec(200):
        a = mpmath.mpf(d) * mpmath.pi / 180
        return +mpmath.sin(a), +mpmath.cos(a)


def test_sincosd_against_mpmath(oracle):
    rng = np.random.default_rng(11)
    ds = list(rng.uniform(-180, 180, 4000)) + list(rng.uniform(-1e-3, 1e-3, 200))
    ds += [0.0, 1e-300, -1e-300, 30.0, 45.0, -45.0, 44.999999999, 45.000000001, 60.0, 89.9999, 90.0, 120.0,
           135.0, 135.00000001, 179.999999, 180.0, -180.0, -90.0, 40.7, -73.95]
    worst = 0.0
    with mpmath.workprec(200):        # independent of the precision other tests leave set
        for d in ds:
            s, c = oracle.sincosd(d)
            ms, mc = _mp_sincosd(d)
            for got, want in ((s, ms), (c, mc)):
                if abs(want) < mpmath.mpf("1e-40"):      # exact zero of sin/cos (mpmath's pi is finite)
                    assert abs(got) < 1e-40
                    continue
                worst = max(worst, float(abs(mpmath.mpf(got) - want) / ulp(float(want))))
    assert worst <= 3.0, worst


def test_sincosd_exact_special_values(oracle):
    assert oracle.sincosd(0.0) == (0.0, 1.0)
    s, c = oracle.sincosd(90.0)
    assert s == 1.0 and c == 0.0
    s, c = oracle.sincosd(180.0)
    assert s == 0.0 and c == -1.0
    s, c = oracle.sincosd(-90.0)
    assert s == -1.0 and c == 0.0


def _mp_face_uv(lat, lng):
    """Independent high-precision face/(u,v): xyz in mpmath, face by largest
    |component|, (u,v) from the cube-face formulas."""
    sp, cp = _mp_sincosd(lat)
    sl, cl = _mp_sincosd(lng)
    x, y, z = cp * cl, cp * sl, sp
    comps = [x, y, z]
    axis = max(range(3), key=lambda k: abs(comps[k]))
    face = axis + (3 if comps[axis] < 0 else 0)
    uv = {
        0: (y / x, z / x), 1: (-x / y, z / y), 2: (-x / z, -y / z),
        3: (z / x, y / x), 4: (z / y, -x / y), 5: (-y / z, -x / z),
    }[face]
    return face, uv


def test_face_uv_against_mpmath(oracle):
    rng = np.random.default_rng(12)
    lat = np.degrees(np.arcsin(rng.uniform(-1, 1, 3000)))
    lng = rng.uniform(-180, 180, 3000)
    worst = 0.0
    for a, b in zip(lat, lng):
        f, u, v = oracle.face_uv(float(a), float(b))
        mf, (mu, mv) = _mp_face_uv(float(a), float(b))
        # skip points within 1e-12 of a face boundary (face choice is then a tie)
        if f != mf:
            assert abs(abs(float(mu)) - 1) < 1e-9 or abs(abs(float(mv)) - 1) < 1e-9
            continue
        worst = max(worst, abs(u - float(mu)) / 2.0 ** -52, abs(v - float(mv)) / 2.0 ** -52)
    assert worst <= 8.0, worst


@pytest.mark.parametrize("lat,lng,face", [(0, 0, 0), (0, 90, 1), (90, 0, 2), (0, 180, 3), (0, -90, 4), (-90, 0, 5)])
def test_face_centres(oracle, lat, lng, face):
    f, u, v = oracle.face_uv(lat, lng)
    assert f == face and u == 0.0 and v == 0.0
    cid = oracle.cell_id(lat, lng)
    # centre of a face: s = t = 1/2 -> i = j = 2^29
    fa, lev, i, j = oracle.id_decode(cid)
    assert (fa, lev, i, j) == (face, 30, 1 << 29, 1 << 29)
    # the level-0 ancestor is the face cell: face<<61 | 1<<60
    assert oracle.id_parent(cid, 0) == (face << 61) | (1 << 60)
    assert oracle.id_level((face << 61) | (1 << 60)) == 0


def test_id_bit_layout(oracle):
    rng = np.random.default_rng(13)
    for _ in range(200):
        lat = float(rng.uniform(-90, 90)); lng = float(rng.uniform(-180, 180))
        cid = oracle.cell_id(lat, lng)
        f, _, _ = oracle.face_uv(lat, lng)
        assert cid >> 61 == f
        assert cid & 1 == 1                     # leaf: marker bit is the lsb
        for L in range(0, 31):
            p = oracle.id_parent(cid, L)
            assert oracle.id_level(p) == L
            lsb = 1 << (2 * (30 - L))
            assert p & (2 * lsb - 1) == lsb     # marker bit then zeros
            lo, hi = oracle.id_range(p)
            assert lo <= cid <= hi


def test_st_transform_closed_forms(oracle):
    assert oracle.uv_to_st(0.0) == 0.5
    assert oracle.uv_to_st(1.0) == 1.0
    assert oracle.uv_to_st(-1.0) == 0.0
    assert oracle.st_to_uv(0.5) == 0.0
    assert oracle.st_to_uv(1.0) == 1.0
    assert oracle.st_to_uv(0.0) == -1.0
    assert oracle.st_to_uv(0.75) == (4 * 0.75 * 0.75 - 1) / 3
    for s in np.linspace(0, 1, 257):
        assert abs(oracle.uv_to_st(oracle.st_to_uv(float(s))) - s) < 4e-16


def test_level1_order_face0_and_face1(oracle):
    def children(face):
        out = []
        for i in range(2):
            for j in range(2):
                cid = oracle.id_parent(oracle.id_from_face_ij(face, i << 29, j << 29), 1)
                out.append((cid, (i, j)))
        return [ij for _, ij in sorted(out)]
    # canonical frame: digits 0..3 visit (0,0),(0,1),(1,1),(1,0); odd faces start swapped
    assert children(0) == [(0, 0), (0, 1), (1, 1), (1, 0)]
    assert children(1) == [(0, 0), (1, 0), (1, 1), (0, 1)]
    assert children(4) == [(0, 0), (0, 1), (1, 1), (1, 0)]


@pytest.mark.parametrize("face", range(6))
def test_hilbert_continuity_exhaustive(oracle, face):
    """Consecutive cells along the curve share an edge (levels 1..6)."""
    for L in range(1, 7):
        n = 1 << L
        ids = []
        for i in range(n):
            for j in range(n):
                cid = oracle.id_parent(oracle.id_from_face_ij(face, i << (30 - L), j << (30 - L)), L)
                ids.append((cid, i, j))
        ids.sort()
        assert len({c for c, _, _ in ids}) == n * n
        step = 2 * (1 << (2 * (30 - L)))
        for (c0, i0, j0), (c1, i1, j1) in zip(ids, ids[1:]):
            assert c1 - c0 == step
            assert abs(i0 - i1) + abs(j0 - j1) == 1


@pytest.mark.parametrize("face", range(6))
def test_decode_roundtrip_exhaustive(oracle, face):
    for L in range(0, 6):
        n = 1 << L
        for i in range(n):
            for j in range(n):
                cid = oracle.id_parent(oracle.id_from_face_ij(face, i << (30 - L), j << (30 - L)), L)
                assert oracle.id_decode(cid) == (face, L, i, j)


def test_children_share_parent_prefix(oracle):
    rng = np.random.default_rng(14)
    for _ in range(300):
        face = int(rng.integers(0, 6)); L = int(rng.integers(0, 29))
        i = int(rng.integers(0, 1 << 30)); j = int(rng.integers(0, 1 << 30))
        c = oracle.id_parent(oracle.id_from_face_ij(face, i, j), L)
        lo, hi = oracle.id_range(c)
        kids = []
        for di in range(2):
            for dj in range(2):
                ci = ((i >> (30 - L)) << 1 | di) << (29 - L)
                cj = ((j >> (30 - L)) << 1 | dj) << (29 - L)
                k = oracle.id_parent(oracle.id_from_face_ij(face, ci, cj), L + 1)
                assert oracle.id_parent(k, L) == c
                klo, khi = oracle.id_range(k)
                assert lo <= klo and khi <= hi
                kids.append((klo, khi))
        kids.sort()
        assert kids[0][0] == lo and kids[-1][1] == hi
        for (a0, a1), (b0, b1) in zip(kids, kids[1:]):
            assert b0 == a1 + 2          # the even value between is not a leaf id


def test_point_lies_in_its_cell_rect(oracle):
    rng = np.random.default_rng(15)
    lat = np.degrees(np.arcsin(rng.uniform(-1, 1, 2000)))
    lng = rng.uniform(-180, 180, 2000)
    for a, b in zip(lat, lng):
        f, u, v = oracle.face_uv(float(a), float(b))
        cid = oracle.cell_id(float(a), float(b))
        for L in (0, 5, 13, 22, 30):
            fr, r = oracle.cell_uv_rect(oracle.id_parent(cid, L))
            assert fr == f
            tol = 4e-16
            assert r[0] - tol <= u <= r[1] + tol and r[2] - tol <= v <= r[3] + tol


def test_face_cell_diagonal_closed_form(oracle):
    # opposite corners of a cube face: unit vectors (1,1,1)/sqrt3 and (1,-1,-1)/sqrt3
    expect = 6371008.8 * math.acos(-1.0 / 3.0)
    for face in range(6):
        d = oracle.cell_diag_m((face << 61) | (1 << 60))
        assert abs(d - expect) < 1e-6 * expect


def test_invalid_points(oracle):
    for lat, lng in [(float("nan"), 0.0), (0.0, float("nan")), (90.0000001, 0.0), (0.0, 180.0000001),
                     (float("inf"), 0.0), (-91.0, 5.0)]:
        assert oracle.cell_id(lat, lng) == 0
        assert oracle.face_uv(lat, lng)[0] == -1
    assert oracle.cell_id(90.0, 180.0) != 0
