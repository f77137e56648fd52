"""Points next to cell edges, located in the FP64 spec's own arithmetic.

For a level L, a line of constant longitude (or latitude) across a window
is bisected with the oracle's cell ids until two adjacent doubles fall in
different level-L cells: the larger one is the first point of the next
cell.  Around each such edge the points returned are at +-1 .. +-4 ulps,
and at +-m times a distance given in level-30 cells (converted with the
local rate of change of the spec's level-30 index along the line).  These
are the places where a certified prefix (FP32 model +- its error bound)
could disagree with the spec if the bound were too small.
"""
import numpy as np


def _parent_ids(oracle, pts, level):
    ids = oracle.cell_ids(pts)
    lsb = np.uint64(1) << np.uint64(2 * (30 - level))
    return (ids & ~(np.uint64(2) * lsb - np.uint64(1))) | lsb


def edge_points(oracle, window, levels, lines_per_level, err_cells, rng, axis=0,
                ulps=(1, 2, 3, 4), multiples=(0.5, 0.9, 1.1, 2.0, 4.0, 8.0)):
    """window = (lat_lo, lat_hi, lng_lo, lng_hi).  axis 0 bisects latitude
    along meridians, axis 1 longitude along parallels.  Returns (points,
    level of the edge each point lies next to, its distance from the edge
    in units of err_cells: 0 for the points a few ulps away)."""
    lat_lo, lat_hi, lng_lo, lng_hi = window
    out, lv_out, m_out = [], [], []
    for L in levels:
        fixed = rng.uniform(lng_lo, lng_hi, lines_per_level) if axis == 0 else \
            rng.uniform(lat_lo, lat_hi, lines_per_level)
        lo_c = np.full(lines_per_level, lat_lo if axis == 0 else lng_lo)
        hi_c = np.full(lines_per_level, lat_hi if axis == 0 else lng_hi)
        # a random sub-span per line, about eight level-L cells long (a face
        # spans ~90 degrees) where the window allows
        span = np.minimum(hi_c - lo_c, 8.0 * 90.0 / 2.0 ** L)
        start = lo_c + rng.uniform(0, 1, lines_per_level) * (hi_c - lo_c - span)
        a, b = start, start + span

        def pts_at(c):
            return np.stack([c, fixed], -1) if axis == 0 else np.stack([fixed, c], -1)

        pa, pb = _parent_ids(oracle, pts_at(a), L), _parent_ids(oracle, pts_at(b), L)
        keep = pa != pb
        if not keep.any():
            continue
        a, b, fixed, pa = a[keep], b[keep], fixed[keep], pa[keep]
        # invariant: parent(a) == pa != parent(b); stop at adjacent doubles
        for _ in range(200):
            mid = a + 0.5 * (b - a)
            done = (mid <= a) | (mid >= b)
            if done.all():
                break
            same = _parent_ids(oracle, pts_at(mid), L) == pa
            a = np.where(~done & same, mid, a)
            b = np.where(~done & ~same, mid, b)
        edge = b                                   # first double of the next cell
        pts, dist = [], []
        for k in ulps:
            up, dn = edge.copy(), edge.copy()
            for _ in range(k):
                up = np.nextafter(up, np.inf)
                dn = np.nextafter(dn, -np.inf)
            pts += [up, dn]
            dist += [0.0, 0.0]
        # rate of the level-30 index along the line, from a 1000-cell step
        step = 1000.0 * 90.0 / 2.0 ** 30
        i0 = _leaf_ij(oracle, pts_at(edge - step))
        i1 = _leaf_ij(oracle, pts_at(edge + step))
        rate = np.maximum(np.abs(i1 - i0).max(axis=1), 1.0) / (2 * step)      # cells per degree
        for m in multiples:
            d = m * err_cells / rate
            pts += [edge + d, edge - d]
            dist += [m, m]
        for c, m in zip(pts, dist):
            out.append(pts_at(c))
            lv_out.append(np.full(len(c), L))
            m_out.append(np.full(len(c), m))
    return np.concatenate(out), np.concatenate(lv_out), np.concatenate(m_out)


def _leaf_ij(oracle, pts):
    ids = oracle.cell_ids(pts)
    ij = np.zeros((len(ids), 2))
    for k, cid in enumerate(ids):
        _, _, i, j = oracle.id_decode(int(cid))
        ij[k] = (i, j)
    return ij


def prefix_equal(a, b, levels):
    """Leading `levels` levels (3 face bits + 2 bits per level) equal."""
    a = a.astype(np.uint64)
    b = b.astype(np.uint64)
    bits = (3 + 2 * levels.astype(np.uint64))
    sh = (np.uint64(64) - bits)
    mask = np.where(bits >= 64, np.uint64(0xFFFFFFFFFFFFFFFF), ~((np.uint64(1) << sh) - np.uint64(1)))
    return (a & mask) == (b & mask)
