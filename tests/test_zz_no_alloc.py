"""The allocation-free approximate join, checked against agj_join.

Some callers cannot allocate device memory at join time: code that runs
under a device-memory budget split up front, plugins hosted by a framework
that owns every device allocation, and latency-bound loops where a
cudaMalloc could synchronise the device and stall other streams.
agj_join_approx_noalloc serves them from a static device array of the
library.  This test calls it through the C ABI twice in a row and checks
each result against the CSR of the allocating entry point, agj_join (integer
output, so the comparison is exact), and checks that a size beyond the
array's maximum is refused before anything is launched.  Further cases:
a join just under the maximum (every tile state of the array in use), an
index whose cells hold 256 references (lookup-table cells), and the
refusals for an exact-mode index, a misaligned point pointer, too small an
id buffer and a result beyond 32-bit offsets.  Every refused call returns
before any kernel is launched.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

AGJ_EINVAL = 1
AGJ_ECAPACITY = 8
MAX_POINTS = 1 << 24


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1802_09488_gb300 as agj

    L = agj.lib()
    fn = L.agj_join_approx_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p]
    return torch, agj, fn


def _call(torch, fn, ix, pts, n, cap, ptr_shift=0):
    """One call through the C ABI into fresh outputs; returns (rc, offsets,
    ids, status) with the outputs read back after a synchronize."""
    d_off = torch.full((n + 1,), -1, dtype=torch.int32, device="cuda")
    d_ids = torch.full((max(cap, 1),), -1, dtype=torch.int32, device="cuda")
    d_status = torch.full((4,), -1, dtype=torch.int64, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = fn(ix.handle, C.c_void_p(pts.data_ptr() + ptr_shift), n, C.c_void_p(d_off.data_ptr()),
            C.c_void_p(d_ids.data_ptr()), cap, C.c_void_p(d_status.data_ptr()), stream)
    torch.cuda.synchronize()
    return rc, d_off.cpu().numpy().view(np.uint32), d_ids.cpu().numpy().view(np.uint32), \
        d_status.cpu().numpy().view(np.uint64)


def test_noalloc_join_matches_join_on_two_calls():
    torch, agj, fn = _setup()
    from paper_1802_09488_gb300 import synth

    w = synth.c1_tiny(100_003)
    n = len(w.points)
    ix = agj.Index(w.polygons, agj.APPROX, w.eps_m)
    pts = torch.from_numpy(w.points).cuda()
    want_off, want_ids = agj.join(ix, pts).to_host()

    cap = n * max(ix.stats()["max_refs"], 1)
    d_off = torch.empty(n + 1, dtype=torch.int32, device="cuda")
    d_ids = torch.empty(cap, dtype=torch.int32, device="cuda")
    d_status = torch.empty(4, dtype=torch.int64, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        d_off.fill_(-1)
        d_ids.fill_(-1)
        d_status.fill_(-1)
        rc = fn(ix.handle, C.c_void_p(pts.data_ptr()), n, C.c_void_p(d_off.data_ptr()),
                C.c_void_p(d_ids.data_ptr()), cap, C.c_void_p(d_status.data_ptr()), stream)
        assert rc == 0, (call, rc)
        torch.cuda.synchronize()
        st = d_status.cpu().numpy().view(np.uint64)
        assert st[1] == 0, (call, st)
        nnz = int(st[0])
        assert nnz == len(want_ids)
        assert np.array_equal(d_off.cpu().numpy().view(np.uint32), want_off), call
        assert np.array_equal(d_ids[:nnz].cpu().numpy().view(np.uint32), want_ids), call

    rc = fn(ix.handle, C.c_void_p(pts.data_ptr()), MAX_POINTS + 1, C.c_void_p(d_off.data_ptr()),
            C.c_void_p(d_ids.data_ptr()), cap, C.c_void_p(d_status.data_ptr()), stream)
    assert rc == AGJ_ECAPACITY


def test_noalloc_just_under_the_maximum():
    """2^24 - 1 points: all but the last point of the array's 2^24, so every
    tile state and the last tile's offsets[n] write are in use."""
    torch, agj, fn = _setup()
    from paper_1802_09488_gb300 import synth
    w = synth.c1_tiny(MAX_POINTS - 1)
    n = len(w.points)
    ix = agj.Index(w.polygons, agj.APPROX, w.eps_m)
    pts = torch.from_numpy(w.points).cuda()
    want_off, want_ids = agj.join(ix, pts).to_host()
    cap = n * max(ix.stats()["max_refs"], 1)
    rc, off, ids, st = _call(torch, fn, ix, pts, n, cap)
    assert rc == 0 and st[1] == 0 and int(st[0]) == len(want_ids)
    assert np.array_equal(off, want_off)
    assert np.array_equal(ids[:len(want_ids)], want_ids)


def _stacked(agj, k):
    """k copies of one small triangle: each cell inside holds k references."""
    tri = np.array([[40.700, -73.950], [40.702, -73.950], [40.700, -73.947]])
    return agj.Index([tri] * k, agj.APPROX, 10.0)


def test_noalloc_lookup_table_cells_and_refusals():
    torch, agj, fn = _setup()
    from paper_1802_09488_gb300 import synth
    ix = _stacked(agj, 256)
    assert ix.stats()["max_refs"] == 256
    rng = np.random.default_rng(5)
    pts_np = np.stack([rng.uniform(40.6995, 40.7025, 4099), rng.uniform(-73.9505, -73.9465, 4099)], -1)
    pts = torch.from_numpy(pts_np).cuda()
    want_off, want_ids = agj.join(ix, pts).to_host()
    assert len(want_ids) > 256 * 100
    n = len(pts_np)
    cap = n * 256
    rc, off, ids, st = _call(torch, fn, ix, pts, n, cap)
    assert rc == 0 and st[1] == 0
    assert np.array_equal(off, want_off) and np.array_equal(ids[:len(want_ids)], want_ids)
    # refused before any launch: too small an id buffer, a misaligned pointer
    assert _call(torch, fn, ix, pts, n, cap - 1)[0] == AGJ_ECAPACITY
    assert _call(torch, fn, ix, pts, n - 1, cap, ptr_shift=8)[0] == AGJ_EINVAL
    # 2^24 points x 256 references = 2^32 ids: beyond 32-bit offsets, refused
    # even with a capacity that claims room (the check comes before the
    # capacity check and before any launch; no point or id is read)
    big = torch.zeros((MAX_POINTS, 2), dtype=torch.float64, device="cuda")
    d_ids = torch.empty(1, dtype=torch.int32, device="cuda")
    d_off = torch.empty(MAX_POINTS + 1, dtype=torch.int32, device="cuda")
    d_st = torch.empty(4, dtype=torch.int64, device="cuda")
    rc = fn(ix.handle, C.c_void_p(big.data_ptr()), MAX_POINTS, C.c_void_p(d_off.data_ptr()),
            C.c_void_p(d_ids.data_ptr()), 1 << 32, C.c_void_p(d_st.data_ptr()),
            C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == AGJ_ECAPACITY
    # an exact-mode index is refused
    w = synth.c1_tiny(1000)
    ie = agj.Index(w.polygons, agj.EXACT, 0)
    pe = torch.from_numpy(w.points).cuda()
    assert _call(torch, fn, ie, pe, len(w.points), len(w.points) * 8)[0] == AGJ_EINVAL
