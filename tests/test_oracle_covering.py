"""Pins for the oracle's covering checker (no GPU).

The checker tests the invariants of a logical index: indexed cells do not
overlap (§III-B "no overlap between the indexed cells"); a true-hit cell lies
wholly inside its polygon (§II: interior coverings are completely contained);
a candidate cell meets its polygon (§II coverings); in approximate mode every
candidate cell's diagonal is below the precision (§III-A); and every
reference names a polygon on the cell's face.

A checker that never counts passes every real covering, so each counter is
pinned here by hand-made bad coverings that must raise exactly that counter
by a known amount, beside good coverings that must raise none.  The
fixture is a square polygon in one face's (u,v) plane over a 4 x 4 block
of level-16 cells.  The square extends a tenth of a cell past the inner 2
x 2 block on every side, so:
  * the four inner cells lie strictly inside the square (valid true hits);
  * the twelve ring cells cross its edges (valid candidates, invalid true hits);
  * cells one column further out miss it by 0.9 cell (invalid candidates).
The square's (u,v) corners are mapped to (lat, lng) by the gnomonic inverse
of the face projection (the face table of S2's published convention), and
the oracle maps them back.  The round trip moves a corner by about 1e-16 in
(u,v), far below the 0.1-cell (3e-6) margins.
"""
import math

import numpy as np
import pytest

LEVEL = 16


def _face_uv_to_latlng(face, u, v):
    # unit-cube point of face (u, v), the inverse of the face/(u,v) projection
    x, y, z = {0: (1.0, u, v), 1: (-u, 1.0, v), 2: (-u, -v, 1.0),
               3: (-1.0, -v, -u), 4: (v, -1.0, -u), 5: (v, u, -1.0)}[face]
    lat = math.degrees(math.atan2(z, math.hypot(x, y)))
    lng = math.degrees(math.atan2(y, x))
    return lat, lng


def _cell(oracle, face, i, j, level=LEVEL):
    """Cell (i, j) at `level` of a face, via the oracle's (pinned) leaf id."""
    sh = 30 - level
    leaf = oracle.id_from_face_ij(face, (i << sh) | (1 << (sh - 1)), (j << sh) | (1 << (sh - 1)))
    return oracle.id_parent(leaf, level)


@pytest.fixture(scope="module")
def block(oracle):
    """(face, i0, j0, polygon set, square's uv corners): the 4 x 4 block of
    level-16 cells (i0 .. i0+3, j0 .. j0+3) around the city centre."""
    face, lvl, i, j = oracle.id_decode(oracle.id_parent(oracle.cell_id(40.70, -73.95), LEVEL))
    assert lvl == LEVEL
    i0, j0 = i - 1, j - 1
    r_lo = oracle.cell_uv_rect(_cell(oracle, face, i0 + 1, j0 + 1))[1]
    r_hi = oracle.cell_uv_rect(_cell(oracle, face, i0 + 2, j0 + 2))[1]
    wu = r_lo[1] - r_lo[0]
    wv = r_lo[3] - r_lo[2]
    u0, u1 = r_lo[0] - 0.1 * wu, r_hi[1] + 0.1 * wu
    v0, v1 = r_lo[2] - 0.1 * wv, r_hi[3] + 0.1 * wv
    corners = [(u0, v0), (u1, v0), (u1, v1), (u0, v1)]
    ring = np.array([_face_uv_to_latlng(face, u, v) for u, v in corners])
    for (u, v), (la, lo) in zip(corners, ring):          # the round trip stays on the face, within 1e-14
        f, uu, vv = oracle.face_uv(la, lo)
        assert f == face and abs(uu - u) < 1e-14 and abs(vv - v) < 1e-14
    ps = oracle.PolySet([ring])
    return face, i0, j0, ps


def _check(ps, entries, eps_m=0.0):
    """entries: list of (cell, [ref, ...]); the covering is sorted by cell."""
    entries = sorted(entries, key=lambda e: e[0])
    cells = np.array([c for c, _ in entries], dtype=np.uint64)
    off = np.zeros(len(entries) + 1, dtype=np.uint64)
    refs = []
    for k, (_, rr) in enumerate(entries):
        refs.extend(rr)
        off[k + 1] = len(refs)
    return ps.check_covering(cells, off, np.array(refs, dtype=np.uint32), eps_m=eps_m)


TRUE, CAND = 1, 0      # ref = polygon_id << 1 | interior


def _good(oracle, face, i0, j0):
    inner = [(_cell(oracle, face, i0 + a, j0 + b), [TRUE]) for a in (1, 2) for b in (1, 2)]
    ring = [(_cell(oracle, face, i0 + a, j0 + b), [CAND]) for a in range(4) for b in range(4)
            if a in (0, 3) or b in (0, 3)]
    return inner, ring


ZERO = {"overlapping_cells": 0, "true_ref_not_inside": 0, "cand_ref_misses": 0, "cand_diag_ge_eps": 0, "bad_ref": 0}


def _only(key, n):
    d = dict(ZERO)
    d[key] = n
    return d


def test_good_covering_raises_nothing(oracle, block):
    face, i0, j0, ps = block
    inner, ring = _good(oracle, face, i0, j0)
    assert _check(ps, inner + ring, eps_m=10_000.0) == ZERO
    # a candidate cell holding the whole polygon meets it (a vertex inside)
    parent = oracle.id_parent(_cell(oracle, face, i0, j0), LEVEL - 2)
    assert _check(ps, [(parent, [CAND])]) == ZERO
    # candidates wholly inside the polygon also meet it
    assert _check(ps, [(c, [CAND]) for c, _ in inner]) == ZERO


def test_overlapping_cells_are_counted(oracle, block):
    face, i0, j0, ps = block
    inner, ring = _good(oracle, face, i0, j0)
    c = inner[0][0]
    # the same cell twice: one overlapping neighbour pair
    assert _check(ps, [(c, [TRUE]), (c, [TRUE])]) == _only("overlapping_cells", 1)
    # an ancestor beside its descendant: one pair
    anc = oracle.id_parent(c, LEVEL - 3)
    assert _check(ps, [(anc, [CAND]), (c, [TRUE])]) == _only("overlapping_cells", 1)
    # a child of a ring cell, on the side the polygon reaches into, added to
    # the good covering: one pair
    child_leaf = oracle.id_from_face_ij(face, ((i0 + 1) << 14) | 8000, (j0 << 14) | 16380)
    child = oracle.id_parent(child_leaf, LEVEL + 2)
    rep = _check(ps, inner + ring + [(child, [CAND])])
    assert rep == _only("overlapping_cells", 1)
    # the next cell along the curve touches but does not overlap
    nxt = c + 2 * (c & (~c + 1))
    assert _check(ps, [(c, [TRUE]), (nxt, [CAND])])["overlapping_cells"] == 0


def test_true_ref_on_a_crossing_cell_is_counted(oracle, block):
    face, i0, j0, ps = block
    inner, ring = _good(oracle, face, i0, j0)
    # every ring cell, one side after another, turned into a true hit
    for k in range(len(ring)):
        bad = list(ring)
        bad[k] = (bad[k][0], [TRUE])
        assert _check(ps, inner + bad) == _only("true_ref_not_inside", 1), k
    assert _check(ps, inner + [(c, [TRUE]) for c, _ in ring]) == _only("true_ref_not_inside", len(ring))
    # a true hit on a cell wholly outside (its centre is out, no edge meets it)
    far = _cell(oracle, face, i0 - 40, j0 + 1)
    assert _check(ps, inner + ring + [(far, [TRUE])]) == _only("true_ref_not_inside", 1)
    # a true hit on a cell holding the whole polygon (edges meet it)
    parent = oracle.id_parent(_cell(oracle, face, i0, j0), LEVEL - 2)
    assert _check(ps, [(parent, [TRUE])]) == _only("true_ref_not_inside", 1)


def test_candidate_ref_on_a_far_cell_is_counted(oracle, block):
    face, i0, j0, ps = block
    inner, ring = _good(oracle, face, i0, j0)
    # one column (row) beyond the ring on each side: 0.9 cell from the polygon
    near_miss = [_cell(oracle, face, i0 - 1, j0 + 1), _cell(oracle, face, i0 + 4, j0 + 2),
                 _cell(oracle, face, i0 + 1, j0 - 1), _cell(oracle, face, i0 + 2, j0 + 4)]
    for c in near_miss:
        assert _check(ps, inner + ring + [(c, [CAND])]) == _only("cand_ref_misses", 1)
    far = _cell(oracle, face, i0 + 300, j0 - 200)
    assert _check(ps, inner + ring + [(far, [CAND])] + [(c, [CAND]) for c in near_miss]) == \
        _only("cand_ref_misses", 5)


def test_candidate_cell_diagonal_against_eps(oracle, block):
    face, i0, j0, ps = block
    inner, ring = _good(oracle, face, i0, j0)
    diag = max(oracle.cell_diag_m(c) for c, _ in ring)
    dmin = min(oracle.cell_diag_m(c) for c, _ in ring)
    assert 100.0 < dmin <= diag < 400.0            # level 16: ~150 m cells
    assert _check(ps, inner + ring, eps_m=diag * 1.001) == ZERO
    assert _check(ps, inner + ring, eps_m=dmin * 0.999) == _only("cand_diag_ge_eps", len(ring))
    # eps = 0 switches the check off (exact mode); true-hit cells never count
    assert _check(ps, inner + ring, eps_m=0.0) == ZERO
    assert _check(ps, inner, eps_m=1.0) == ZERO
    # a cell with a true and a candidate reference counts once
    two = [(c, [TRUE, CAND]) for c, _ in inner[:1]]
    assert _check(ps, two, eps_m=1.0) == _only("cand_diag_ge_eps", 1)


def test_bad_references_are_counted(oracle, block):
    face, i0, j0, ps = block
    inner, ring = _good(oracle, face, i0, j0)
    c = inner[0][0]
    # polygon 1 does not exist (one polygon in the set)
    assert _check(ps, inner + ring + [(_cell(oracle, face, i0 + 9, j0), [(1 << 1) | 1])]) == _only("bad_ref", 1)
    assert _check(ps, [(c, [TRUE, (7 << 1)])]) == _only("bad_ref", 1)
    # a cell on another face referencing the polygon
    other = _cell(oracle, (face + 1) % 6, 100, 100)
    assert _check(ps, inner + ring + [(other, [CAND])]) == _only("bad_ref", 1)
