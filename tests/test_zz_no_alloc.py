"""The allocation-free approximate join, checked against agj_join.

Some callers cannot allocate device memory at join time: code that runs
under a device-memory budget split up front, plugins hosted by a framework
that owns every device allocation, and latency-bound loops where a
cudaMalloc could synchronise the device and stall other streams.
agj_join_approx_noalloc serves them from a static device array of the
library.  This test calls it through the C ABI twice in a row and checks
each result against the CSR of the allocating entry point, agj_join (integer
output, so the comparison is exact), and checks that a size beyond the
array's maximum is refused before anything is launched.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

AGJ_ECAPACITY = 8
MAX_POINTS = 1 << 24


def test_noalloc_join_matches_join_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1802_09488_gb300 as agj
    from paper_1802_09488_gb300 import synth

    L = agj.lib()
    fn = L.agj_join_approx_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p]

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
