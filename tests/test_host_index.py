"""Host-side tests of the library (no GPU): C-ABI exports, the super-covering
merge (§III-B), the lookup-table encoding (§III-C, Fig. 6b), and indexes
built on the host checked against the oracle's invariants and probes."""
import json
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def agj():
    import paper_1802_09488_gb300 as m
    m.lib()
    return m


def test_library_exports_every_declared_symbol(agj):
    import ctypes
    src = open(os.path.join(ROOT, "include", "agj.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = sorted(set(re.findall(r"\b(agj_[a-z_0-9]+)\s*\(", src)))
    assert len(names) >= 15
    L = ctypes.CDLL(agj.native._build.LIB)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_strerror_names_every_status(agj):
    L = agj.lib()
    for s in range(10):
        assert L.agj_strerror(s).decode() != "unknown status"


def test_lut_golden_example(agj):
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "lut_example.json")))
    lists = [[(t << 1) | 1 for t in e["true"]] + [c << 1 for c in e["candidate"]] for e in g["lists"]]
    words, offs = agj.native.lut_encode(lists)
    assert list(words) == g["expected_words"]
    assert list(offs) == g["expected_word_offsets"]
    # decoding returns the same sets
    for e, o in zip(g["lists"], offs):
        nt = words[o]
        assert sorted(words[o + 1:o + 1 + nt]) == sorted(e["true"])
        nc = words[o + 1 + nt]
        assert sorted(words[o + 2 + nt:o + 2 + nt + nc]) == sorted(e["candidate"])
    # a repeated list is stored once
    w2, o2 = agj.native.lut_encode(lists + [lists[0]])
    assert list(w2) == g["expected_words"] and list(o2) == [0, 5, 0]


def _cell(oracle, lat, lng, level):
    return oracle.id_parent(oracle.cell_id(lat, lng), level)


def test_conflict_resolution_difference_cells(agj, oracle):
    """§III-B: c1 ancestor of c2 two levels down -> d has six cells, the cell
    count grows by five, c1's references are copied to d and c2, and d plus
    c2 exactly tile c1."""
    c1 = _cell(oracle, 40.7, -73.95, 10)
    c2 = _cell(oracle, 40.7, -73.95, 12)
    for order in ([c1, c2], [c2, c1]):
        refs = [0 << 1, (1 << 1) | 1] if order[0] == c1 else [(1 << 1) | 1, 0 << 1]
        cells, off, rr = agj.supercover(order, refs)
        assert len(cells) == 7                      # 2 input cells -> 7: "+5"
        k2 = list(cells).index(c2)
        assert sorted(rr[off[k2]:off[k2 + 1]]) == [0 << 1, (1 << 1) | 1]
        for k in range(7):
            if k != k2:
                assert list(rr[off[k]:off[k + 1]]) == [0 << 1]
        lo1, hi1 = oracle.id_range(c1)
        ranges = sorted(oracle.id_range(int(c)) for c in cells)
        assert ranges[0][0] == lo1 and ranges[-1][1] == hi1
        for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
            assert b0 == a1 + 2
    for dl in range(1, 6):
        cells, _, _ = agj.supercover([c1, _cell(oracle, 40.7, -73.95, 10 + dl)], [0, 3])
        assert len(cells) == 1 + 3 * dl             # |d| = 3 (level difference)


def test_supercover_duplicates_and_true_wins(agj, oracle):
    c = _cell(oracle, 40.7, -73.95, 14)
    cells, off, rr = agj.supercover([c, c, c], [2 << 1, (2 << 1) | 1, 5 << 1])
    assert list(cells) == [c]
    assert list(rr) == [(2 << 1) | 1, 5 << 1]
    # a coarse cell inserted after finer disjoint ones: difference + merged refs
    a = _cell(oracle, 40.7, -73.95, 16)
    b = _cell(oracle, 40.71, -73.95, 16)
    top = oracle.id_parent(a, 12)
    assert oracle.id_parent(b, 12) == top
    cells, off, rr = agj.supercover([a, b, top], [1, 3, 4])
    lo, hi = oracle.id_range(top)
    ranges = sorted(oracle.id_range(int(x)) for x in cells)
    assert ranges[0][0] == lo and ranges[-1][1] == hi
    for k, x in enumerate(cells):
        want = sorted(([1] if x == a else []) + ([3] if x == b else []) + [4])
        assert sorted(rr[off[k]:off[k + 1]]) == want


def _walk_trie(nodes, lut, ft, cid):
    """Reference walk of the flattened trie in Python (Listing 'Probe Adaptive
    Cell Trie'); returns the list of refs (id << 1 | interior) or []."""
    M = (1 << 64) - 1
    f = cid >> 61
    root, pbits, prefix = int(ft[3 * f]), int(ft[3 * f + 1]), int(ft[3 * f + 2])
    if root == 0xFFFFFFFF:
        return []
    key = (cid << 3) & M
    if pbits:
        if key >> (64 - pbits) != prefix:
            return []
        key = (key << pbits) & M
    node = root
    for _ in range(8):
        e = int(nodes[node * 256 + (key >> 56)])
        key = (key << 8) & M
        tag = e & 3
        if tag == 0:
            if e == 0:
                return []
            node = e >> 11
            continue
        if tag == 1:
            p = (e >> 2) & 0x7FFFFFFF
            return [] if p == 0x7FFFFFFF else [p]
        if tag == 2:
            return [(e >> 2) & 0x7FFFFFFF, (e >> 33) & 0x7FFFFFFF]
        off = (e >> 2) & 0x7FFFFFFF
        nt = int(lut[off]); T = [int(x) << 1 | 1 for x in lut[off + 1:off + 1 + nt]]
        nc = int(lut[off + 1 + nt]); Cc = [int(x) << 1 for x in lut[off + 2 + nt:off + 2 + nt + nc]]
        return T + Cc
    raise AssertionError("walk deeper than 8 levels")


@pytest.fixture(scope="module")
def c1(agj):
    from paper_1802_09488_gb300 import synth
    return synth.c1_tiny(30000)


@pytest.mark.parametrize("mode", ["approx", "exact"])
def test_c1_index_invariants_and_trie(agj, oracle, c1, mode):
    m = agj.APPROX if mode == "approx" else agj.EXACT
    train = c1.points[:3000] if mode == "exact" else None
    ix = agj.Index(c1.polygons, m, c1.eps_m, train=train, host_only=True)
    st = ix.stats()
    cells, off, refs = ix.logical()
    assert st["n_cells"] == len(cells) and np.all(np.diff(cells.astype(np.uint64)) > 0)
    ps = oracle.PolySet(c1.polygons)
    rep = ps.check_covering(cells, off, refs, eps_m=c1.eps_m if mode == "approx" else 0.0)
    if mode == "exact":
        # The super-covering merge copies an ancestor's candidate references
        # to every difference cell without re-testing them (§III-B), so an
        # exact-mode candidate may miss its polygon; the PIP rejects it.
        rep.pop("cand_ref_misses")
    assert set(rep.values()) == {0}, rep
    assert st["max_depth"] <= 8
    # no false negatives: every exact pair is referenced by the point's cell
    ao, ai = oracle.join_approx_logical(cells, off, refs, c1.points)
    eo, ei = ps.join_exact(c1.points)
    for p in range(len(c1.points)):
        assert set(ei[eo[p]:eo[p + 1]].tolist()) <= set(ai[ao[p]:ao[p + 1]].tolist())
    nodes, lut, ft = ix.trie()
    ids = oracle.cell_ids(c1.points)
    for k in range(0, len(ids), 7):
        cid = int(ids[k])
        j = oracle.logical_find(cells, cid)
        want = sorted(int(x) for x in refs[off[j]:off[j + 1]]) if j >= 0 else []
        assert sorted(_walk_trie(nodes, lut, ft, cid)) == want


def test_c1_approx_property_oracle(agj, oracle, c1):
    """Approx output is a superset of the exact join; every extra pair lies
    within eps of its polygon by geodesic distance (§III-A precision)."""
    ix = agj.Index(c1.polygons, agj.APPROX, c1.eps_m, host_only=True)
    cells, off, refs = ix.logical()
    ao, ai = oracle.join_approx_logical(cells, off, refs, c1.points)
    ps = oracle.PolySet(c1.polygons)
    eo, ei = ps.join_exact(c1.points)
    n_fp = 0
    worst = 0.0
    for p in range(len(c1.points)):
        A = set(ai[ao[p]:ao[p + 1]].tolist())
        E = set(ei[eo[p]:eo[p + 1]].tolist())
        assert E <= A
        for q in A - E:
            d = ps.dist_m(q, *c1.points[p])
            worst = max(worst, d)
            n_fp += 1
            assert d <= c1.eps_m * (1 + 1e-9)
    assert n_fp > 0 and worst < c1.eps_m


def test_exact_training_refines_expensive_cells(agj, oracle):
    from paper_1802_09488_gb300 import synth
    polys = synth.voronoi_tiling(30, synth.BOX_CITY, seed=9, vmin=20, vmax=80)
    pts = synth.points_mixture(20000, synth.BOX_CITY, seed=9)
    train = synth.points_mixture(20000, synth.BOX_CITY, seed=10, dist_seed=9)
    base = agj.Index(polys, agj.EXACT, 0, host_only=True)
    trained = agj.Index(polys, agj.EXACT, 0, train=train, host_only=True)
    ps = oracle.PolySet(polys)

    def solely_true(ix):
        cells, off, refs = ix.logical()
        rep = ps.check_covering(cells, off, refs)
        rep.pop("cand_ref_misses")
        assert sum(rep.values()) == 0, rep
        ids = oracle.cell_ids(pts)
        good = 0
        for cid in ids:
            j = oracle.logical_find(cells, int(cid))
            if j >= 0 and all(r & 1 for r in refs[off[j]:off[j + 1]]):
                good += 1
        return good / len(ids)

    a, b = solely_true(base), solely_true(trained)
    assert trained.stats()["n_nodes"] > base.stats()["n_nodes"]
    assert b > a + 0.05, (a, b)


def test_build_rejects_bad_polygons(agj):
    with pytest.raises(agj.AgjError) as e:
        agj.Index([np.array([[40.0, -74.0], [40.1, -74.0]])], agj.APPROX, 10.0, host_only=True)
    assert e.value.status == 1
    # a polygon across cube faces is supported within 15 degrees of its
    # vertices' mean (tests/test_host_crossface.py); a wider one is refused
    with pytest.raises(agj.AgjError) as e:
        agj.Index([np.array([[0.0, 30.0], [20.0, 45.0], [-20.0, 60.0]])], agj.APPROX, 10.0, host_only=True)
    assert e.value.status == 2
    with pytest.raises(agj.AgjError) as e:
        agj.Index([np.array([[40.0, -74.0], [40.1, -74.0], [np.nan, -74.1]])], agj.APPROX, 10.0, host_only=True)
    assert e.value.status == 1
    with pytest.raises(agj.AgjError):
        agj.Index([np.array([[40.0, -74.0], [40.1, -74.0], [40.0, -74.1]])], agj.APPROX, 0.0, host_only=True)


def test_host_ids_match_oracle(agj, oracle):
    rng = np.random.default_rng(5)
    lat = np.degrees(np.arcsin(rng.uniform(-1, 1, 20000)))
    lng = rng.uniform(-180, 180, 20000)
    pts = np.stack([lat, lng], -1)
    pts[:5] = [[np.nan, 0], [91, 0], [0, 181], [90, 180], [-90, -180]]
    assert np.array_equal(agj.cell_ids_host(pts), oracle.cell_ids(pts))


def test_auto_mode_picks_approx_or_exact_by_budget(agj, oracle):
    """§III-A: the approximate index when it fits the memory budget, else the
    exact index trained within it; AUTO needs a budget."""
    from paper_1802_09488_gb300 import synth
    w = synth.c1_tiny(20_000)
    ref = agj.Index(w.polygons, agj.APPROX, w.eps_m, host_only=True)
    bytes_approx = ref.stats()["n_nodes"] * 2048 + ref.stats()["n_lut_words"] * 4
    roomy = agj.Index(w.polygons, agj.AUTO, w.eps_m, budget_bytes=bytes_approx, host_only=True)
    assert roomy.mode == agj.APPROX and roomy.stats()["n_cells"] == ref.stats()["n_cells"]
    tight = agj.Index(w.polygons, agj.AUTO, w.eps_m, budget_bytes=bytes_approx - 1, train=w.points[:5000],
                      host_only=True)
    st = tight.stats()
    assert tight.mode == agj.EXACT and st["n_nodes"] * 2048 <= bytes_approx
    cells, off, refs = tight.logical()
    rep = oracle.PolySet(w.polygons).check_covering(cells, off, refs)
    rep.pop("cand_ref_misses")
    assert set(rep.values()) == {0}
    with pytest.raises(agj.AgjError) as e:
        agj.Index(w.polygons, agj.AUTO, w.eps_m, host_only=True)
    assert e.value.status == 1


@pytest.mark.parametrize("mode", ["approx", "exact"])
def test_join_work_space_covers_every_smaller_join(agj, c1, mode):
    """agj_join_requirements(n) must cover every join of m <= n points, also
    across the size where a join switches from 2 to 4 points per lane (2^21):
    buffers sized once for the largest batch are reused for smaller ones."""
    m = agj.APPROX if mode == "approx" else agj.EXACT
    ix = agj.Index(c1.polygons, m, c1.eps_m, host_only=True)
    wide = 1 << 21
    sizes = sorted({0, 1, 127, 128, 129, 4097, 65537, 1_000_003, wide - 129, wide - 128, wide - 2, wide - 1,
                    wide, wide + 1, wide + 127, wide + 300, 3 * wide + 5, 10**8})
    reqs = [ix.requirements(n) for n in sizes]
    best_ids = best_scratch = 0
    for n, (ids_cap, scratch) in zip(sizes, reqs):
        assert ids_cap == n * max(ix.stats()["max_refs"], 1)
        best_ids, best_scratch = max(best_ids, ids_cap), max(best_scratch, scratch)
        assert ids_cap == best_ids and scratch == best_scratch, n     # non-decreasing in n
