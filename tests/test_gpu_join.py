"""GPU parity: the CUDA path, called through the C ABI, against the CPU oracle.

* cell ids: bit-exact (integer output of FP64 arithmetic done the same way);
* approx join: bit-exact CSR against the oracle's sorted-vector probe of the
  index's logical covering (§II, §III-B), which itself is checked against the
  exact join and the eps bound on the CPU (test_host_index.py);
* exact join: bit-exact CSR against brute-force ST_Covers over all polygons
  (§III-A: filter and refine yields the plain join).
Sizes span many tiles of 1024 points and a ragged tail; the full-size city
workload (1e8 points) is checked on sampled rows plus size-independent
properties.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def agj(torch):
    import paper_1802_09488_gb300 as m
    m.lib()
    return m


def _dev(torch, pts):
    return torch.from_numpy(np.ascontiguousarray(pts, dtype=np.float64)).cuda()


def _csr_equal(a_off, a_ids, b_off, b_ids, rows=None):
    a_off = np.asarray(a_off, dtype=np.int64)
    b_off = np.asarray(b_off, dtype=np.int64)
    if rows is None:
        assert np.array_equal(a_off, b_off)
        assert np.array_equal(np.asarray(a_ids, dtype=np.int64), np.asarray(b_ids, dtype=np.int64))
        return
    for r in rows:
        assert list(a_ids[a_off[r]:a_off[r + 1]]) == list(b_ids[b_off[r]:b_off[r + 1]]), r


def test_cell_ids_bit_exact(torch, agj, oracle):
    rng = np.random.default_rng(31)
    n = 1_000_003
    lat = np.degrees(np.arcsin(rng.uniform(-1, 1, n)))
    lng = rng.uniform(-180, 180, n)
    pts = np.stack([lat, lng], -1)
    pts[:8] = [[np.nan, 0], [91, 0], [0, 181], [90, 180], [-90, -180], [0, 0], [45, 45], [35.26438968, 45]]
    got = agj.cell_ids(_dev(torch, pts)).cpu().numpy().view(np.uint64)
    assert np.array_equal(got, oracle.cell_ids(pts))
    from paper_1802_09488_gb300 import synth
    w = synth.points_mixture(500_000, synth.BOX_CITY, 3)
    assert np.array_equal(agj.cell_ids(_dev(torch, w)).cpu().numpy().view(np.uint64), oracle.cell_ids(w))


@pytest.fixture(scope="module")
def c1():
    from paper_1802_09488_gb300 import synth
    return synth.c1_tiny(100_000)


def test_c1_approx_bit_exact(torch, agj, oracle, c1):
    ix = agj.Index(c1.polygons, agj.APPROX, c1.eps_m)
    pr = agj.join(ix, _dev(torch, c1.points))
    off, ids = pr.to_host()
    cells, ro, refs = ix.logical()
    eo, ei = oracle.join_approx_logical(cells, ro, refs, c1.points)
    _csr_equal(off, ids, eo, ei)
    st = pr.status.cpu().numpy()
    assert st[0] == len(ids) and st[1] == 0


def test_c1_exact_bit_exact(torch, agj, oracle, c1):
    ix = agj.Index(c1.polygons, agj.EXACT, 0, train=c1.points[:1000])
    pr = agj.join(ix, _dev(torch, c1.points))
    off, ids = pr.to_host()
    eo, ei = oracle.PolySet(c1.polygons).join_exact(c1.points)
    _csr_equal(off, ids, eo, ei)
    assert pr.status.cpu().numpy()[2] > 0          # candidates were refined


def test_c1_exact_untrained_and_boundary_points(torch, agj, oracle, c1):
    """Points exactly on polygon vertices and edge midpoints (ST_Covers counts
    them inside, §II), plus invalid and far-away points."""
    ix = agj.Index(c1.polygons, agj.EXACT, 0)
    verts = np.concatenate(c1.polygons)
    mids = np.concatenate([0.5 * (p + np.roll(p, -1, axis=0)) for p in c1.polygons])
    extra = np.array([[np.nan, -73.9], [40.7, np.inf], [95.0, 0.0], [10.0, 20.0], [-40.7, 106.05], [40.7, -73.95]])
    pts = np.concatenate([verts, mids, extra, c1.points[:5000]])
    pr = agj.join(ix, _dev(torch, pts))
    off, ids = pr.to_host()
    eo, ei = oracle.PolySet(c1.polygons).join_exact(pts)
    _csr_equal(off, ids, eo, ei)


@pytest.mark.parametrize("n", [0, 1, 2, 1023, 1024, 1025, 4097, 65537])
def test_ragged_sizes(torch, agj, oracle, c1, n):
    for mode in (agj.APPROX, agj.EXACT):
        ix = agj.Index(c1.polygons, mode, c1.eps_m)
        pts = c1.points[:n]
        pr = agj.join(ix, _dev(torch, pts.reshape(-1, 2)))
        off, ids = pr.to_host()
        assert len(off) == n + 1 and off[0] == 0 and off[-1] == len(ids)
        if mode == agj.APPROX:
            cells, ro, refs = ix.logical()
            eo, ei = oracle.join_approx_logical(cells, ro, refs, pts.reshape(-1, 2))
        else:
            eo, ei = oracle.PolySet(c1.polygons).join_exact(pts.reshape(-1, 2))
        _csr_equal(off, ids, eo, ei)


def test_pairs_reuse_and_capacity_errors(torch, agj, c1):
    ix = agj.Index(c1.polygons, agj.APPROX, c1.eps_m)
    pr = agj.Pairs(ix, 10_000)
    a = agj.join(ix, _dev(torch, c1.points[:10_000]), pr)
    o1, i1 = a.to_host()
    b = agj.join(ix, _dev(torch, c1.points[:10_000]), pr)   # same buffers, reset per call
    o2, i2 = b.to_host()
    assert np.array_equal(o1, o2) and np.array_equal(i1, i2)
    pr.c.scratch_bytes = 16                                  # too small: refused before any launch
    with pytest.raises(agj.AgjError) as e:
        agj.join(ix, _dev(torch, c1.points[:10_000]), pr)
    assert e.value.status == 8


def test_tile_width_switch_and_scratch_reuse(torch, agj, oracle):
    """A plain join of 2**21 points or more runs 4 points per lane, a smaller
    one 2; work space sized for the wider join serves both, and both match
    the oracle row for row on either side of the switch."""
    from paper_1802_09488_gb300 import synth
    wide = (1 << 21) + 300
    w = synth.c1_tiny(wide)
    pts = _dev(torch, w.points)
    for mode in (agj.APPROX, agj.EXACT):
        ix = agj.Index(w.polygons, mode, w.eps_m)
        pr = agj.Pairs(ix, wide)
        if mode == agj.APPROX:
            cells, ro, refs = ix.logical()
            eo, ei = oracle.join_approx_logical(cells, ro, refs, w.points)
        else:
            eo, ei = oracle.PolySet(w.polygons).join_exact(w.points)
        for n in (wide, (1 << 21) - 1, 70_000):
            off, ids = agj.join(ix, pts[:n], pr).to_host()
            assert len(off) == n + 1
            _csr_equal(off, ids, eo[:n + 1], ei[:int(eo[n])])


@pytest.fixture(scope="module")
def city_small():
    from paper_1802_09488_gb300 import synth
    return synth.c2_city(2_000_000, n_train=200_000)


def test_city_approx_and_exact_2m(torch, agj, oracle, city_small):
    w = city_small
    pts = _dev(torch, w.points)
    ia = agj.Index(w.polygons, agj.APPROX, w.eps_m)
    off, ids = agj.join(ia, pts).to_host()
    cells, ro, refs = ia.logical()
    eo, ei = oracle.join_approx_logical(cells, ro, refs, w.points)
    _csr_equal(off, ids, eo, ei)
    ie = agj.Index(w.polygons, agj.EXACT, 0, train=w.train)
    off, ids = agj.join(ie, pts).to_host()
    xo, xi = oracle.PolySet(w.polygons).join_exact(w.points)
    _csr_equal(off, ids, xo, xi)


def test_city_full_size_sampled(torch, agj, oracle):
    """The 1e8-point city workload in the launch configuration the benchmark
    times: sampled rows against the oracle, and CSR properties on all rows."""
    from paper_1802_09488_gb300 import synth
    w = synth.c2_city(100_000_000, n_train=1_000_000)
    pts = _dev(torch, w.points)
    rng = np.random.default_rng(77)
    rows = np.sort(rng.choice(len(w.points), 20000, replace=False))
    ps = oracle.PolySet(w.polygons)
    for mode in (agj.APPROX, agj.EXACT):
        ix = agj.Index(w.polygons, mode, w.eps_m, train=w.train if mode == agj.EXACT else None)
        pr = agj.join(ix, pts)
        nnz = pr.check()
        off = pr.offsets.cpu().numpy().view(np.uint32).astype(np.int64)
        assert off[0] == 0 and off[-1] == nnz and np.all(np.diff(off) >= 0)
        sub = w.points[rows]
        if mode == agj.APPROX:
            cells, ro, refs = ix.logical()
            eo, ei = oracle.join_approx_logical(cells, ro, refs, sub)
        else:
            eo, ei = ps.join_exact(sub)
        ids = pr.ids[:nnz].cpu().numpy().view(np.uint32)
        for k, r in enumerate(rows):
            assert ids[off[r]:off[r + 1]].tolist() == ei[eo[k]:eo[k + 1]].tolist(), (mode, r)
        del pr, ix
        torch.cuda.empty_cache()


def test_fast_ids_match_fp64_path(torch, agj, oracle):
    """The certified FP32 id path and the FP64 id path give identical CSR on
    the city mixture, and only a few points fall back to FP64."""
    from paper_1802_09488_gb300 import synth
    polys = synth.c2_city_polygons()
    pts = synth.points_mixture(3_000_000, synth.BOX_CITY, seed=44, dist_seed=3)
    d = _dev(torch, pts)
    for mode in (agj.APPROX, agj.EXACT):
        fast = agj.Index(polys, mode, 4.0, train=pts[:30000] if mode == agj.EXACT else None)
        slow = agj.Index(polys, mode, 4.0, train=pts[:30000] if mode == agj.EXACT else None, fast_ids=False)
        assert fast.stats()["fast_ids"] == 1 and slow.stats()["fast_ids"] == 0
        pf = agj.join(fast, d)
        of, idf = pf.to_host()
        assert pf.fallbacks() < 0.002 * len(pts)
        ps_ = agj.join(slow, d)
        os_, ids_ = ps_.to_host()
        assert ps_.fallbacks() == 0
        _csr_equal(of, idf, os_, ids_)


@pytest.fixture(scope="module")
def c3_small():
    """The fine-polygon workload's structure at a tenth of its polygon count:
    a Voronoi tessellation over a skewed seed field, each polygon scaled
    about its centroid so that points hit 0-3 polygons."""
    from paper_1802_09488_gb300 import synth
    polys = synth.c3_fine_polygons(4000, seed=5)
    pts = synth.points_mixture(300_000, synth.BOX_CITY, seed=6, dist_seed=5)
    train = synth.points_mixture(30_000, synth.BOX_CITY, seed=7, dist_seed=5)
    return polys, pts, train


@pytest.mark.parametrize("mode,eps", [("approx", 1.0), ("approx", 10.0), ("exact", 0.0)])
def test_c3_fine_overlapping_polygons(torch, agj, oracle, c3_small, mode, eps):
    polys, pts, train = c3_small
    if mode == "exact":
        ix = agj.Index(polys, agj.EXACT, 0, train=train)
        eo, ei = oracle.PolySet(polys).join_exact(pts)
    else:
        ix = agj.Index(polys, agj.APPROX, eps)
        cells, ro, refs = ix.logical()
        eo, ei = oracle.join_approx_logical(cells, ro, refs, pts)
    off, ids = agj.join(ix, _dev(torch, pts)).to_host()
    _csr_equal(off, ids, eo, ei)
    hits = np.diff(np.asarray(off, np.int64))
    assert hits.max() >= 2 and (hits == 0).any()       # overlaps and gaps are exercised


def test_c3_exact_many_polygons(torch, agj, oracle):
    """More polygons than the shared-memory counters of the candidate
    grouping hold (> 8192): counting and scattering use global atomics."""
    from paper_1802_09488_gb300 import synth
    polys = synth.c3_fine_polygons(9000, seed=8)
    pts = synth.points_mixture(200_000, synth.BOX_CITY, seed=9, dist_seed=8)
    train = synth.points_mixture(20_000, synth.BOX_CITY, seed=10, dist_seed=8)
    ix = agj.Index(polys, agj.EXACT, 0, train=train)
    pr = agj.join(ix, _dev(torch, pts))
    off, ids = pr.to_host()
    eo, ei = oracle.PolySet(polys).join_exact(pts)
    _csr_equal(off, ids, eo, ei)
    assert pr.status.cpu().numpy()[2] > 10_000          # candidates were refined


def test_join_host_pinned_pageable_and_unaligned(torch, agj, c1):
    """The end-to-end host call gives the device join's CSR whether the
    points are pinned, pageable, or unaligned (staged) host memory."""
    ix = agj.Index(c1.polygons, agj.EXACT, 0, train=c1.points[:1000])
    pts = np.ascontiguousarray(c1.points[:50_000])
    ref_off, ref_ids = agj.join(ix, _dev(torch, pts)).to_host()
    pairs = agj.Pairs(ix, len(pts))
    staging = torch.empty((len(pts), 2), dtype=torch.float64, device="cuda")
    raw = np.empty(2 * len(pts) + 1)
    odd = raw[1:].reshape(-1, 2)
    odd[:] = pts
    for src in (torch.from_numpy(pts).pin_memory(), pts, odd):
        off = np.empty(len(pts) + 1, dtype=np.uint32)
        ids = np.empty(len(ref_ids) + 8, dtype=np.uint32)
        nnz = agj.join_host(ix, src, pairs, staging, off, ids)
        assert nnz == len(ref_ids)
        assert np.array_equal(off, ref_off) and np.array_equal(ids[:nnz], ref_ids)
    # page-locked output arrays
    for src in (torch.from_numpy(pts).pin_memory(), pts):
        off = torch.empty(len(pts) + 1, dtype=torch.int32).pin_memory()
        ids = torch.empty(len(ref_ids), dtype=torch.int32).pin_memory()
        nnz = agj.join_host(ix, src, pairs, staging, off, ids)
        assert nnz == len(ref_ids)
        assert np.array_equal(off.numpy().view(np.uint32), ref_off)
        assert np.array_equal(ids.numpy().view(np.uint32), ref_ids)
    # an ids buffer one short: nothing is written past it, and the call
    # reports the missing capacity
    guard = torch.full((len(ref_ids) + 64,), -7, dtype=torch.int32).pin_memory()
    short = guard[:len(ref_ids) - 1]
    off = torch.empty(len(pts) + 1, dtype=torch.int32).pin_memory()
    with pytest.raises(agj.AgjError):
        agj.join_host(ix, pts, pairs, staging, off, short)
    assert (guard[len(ref_ids) - 1:].numpy() == -7).all()


def test_scan_wait_is_bounded_and_reported(torch, agj, c1):
    """A look-back whose predecessor never publishes runs out its bounded
    wait, reports AGJ_ETIMEOUT, and leaves the device usable."""
    import ctypes
    rc = agj.lib().agj_selftest_scan_timeout(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 6                      # AGJ_ETIMEOUT
    ix = agj.Index(c1.polygons, agj.APPROX, c1.eps_m)
    off, ids = agj.join(ix, _dev(torch, c1.points[:10_000])).to_host()
    assert off[-1] == len(ids) > 0


def test_probe_table_wait_is_bounded_and_reported(torch, agj, c1):
    """A probe block whose shared-table barrier never completes runs out its
    bounded wait, reports AGJ_ETIMEOUT, and leaves the device usable."""
    import ctypes
    rc = agj.lib().agj_selftest_ready_timeout(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 6                      # AGJ_ETIMEOUT
    ix = agj.Index(c1.polygons, agj.APPROX, c1.eps_m)
    off, ids = agj.join(ix, _dev(torch, c1.points[:10_000])).to_host()
    assert off[-1] == len(ids) > 0


def test_join_host_large(torch, agj):
    """A 2e7-point host join equals the device join bit for bit, approximate
    and exact, with page-locked or pageable buffers; an ids buffer one short
    reports the missing capacity and is not overrun."""
    from paper_1802_09488_gb300 import synth
    polys = synth.c2_city_polygons()
    n = 20_000_000
    pts = synth.points_mixture(n, synth.BOX_CITY, seed=31, dist_seed=3)
    train = synth.points_mixture(100_000, synth.BOX_CITY, seed=32, dist_seed=3)
    h_pts = torch.from_numpy(pts).pin_memory()
    staging = torch.empty((n, 2), dtype=torch.float64, device="cuda")
    for ix in (agj.Index(polys, agj.APPROX, 4.0), agj.Index(polys, agj.EXACT, 0, train=train)):
        ref_off, ref_ids = agj.join(ix, h_pts.cuda()).to_host()
        pairs = agj.Pairs(ix, n)
        for src, pinned_out in ((h_pts, True), (pts, False)):
            if pinned_out:
                off = torch.empty(n + 1, dtype=torch.int32).pin_memory()
                ids = torch.empty(len(ref_ids), dtype=torch.int32).pin_memory()
            else:
                off = np.empty(n + 1, dtype=np.uint32)
                ids = np.empty(len(ref_ids), dtype=np.uint32)
            nnz = agj.join_host(ix, src, pairs, staging, off, ids)
            got_off = off.numpy().view(np.uint32) if pinned_out else off
            got_ids = ids.numpy().view(np.uint32) if pinned_out else ids
            assert nnz == len(ref_ids)
            assert np.array_equal(got_off, ref_off) and np.array_equal(got_ids, ref_ids)
        guard = torch.full((len(ref_ids) + 64,), -7, dtype=torch.int32).pin_memory()
        off = torch.empty(n + 1, dtype=torch.int32).pin_memory()
        with pytest.raises(agj.AgjError):
            agj.join_host(ix, h_pts, pairs, staging, off, guard[:len(ref_ids) - 1])
        assert (guard[len(ref_ids) - 1:].numpy() == -7).all()
