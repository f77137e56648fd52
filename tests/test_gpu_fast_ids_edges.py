"""GPU joins of points next to cell edges: the certified FP32 cell ids give
the same CSR as the FP64 spec ids (§II cell ids; the probe's certified
prefix, with the FP64 id recomputed where a level is not certified).

The points are those of test_fast_ids_edges.py: for every level 1-30 with
edges in the window, edges located exactly in the spec's FP64 arithmetic,
and points +-1..4 ulps and 0.5-8 error bounds away from them.  Both modes,
on the windows of the tiny, city and fine-polygon workloads; the
approximate join is also compared with the oracle's probe of the logical
covering and the exact join with brute force.
"""
import numpy as np
import pytest

from test_fast_ids_edges import _workload, near_edge_points

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


@pytest.mark.parametrize("name", ["c1", "c2", "c3"])
def test_join_next_to_cell_edges_fast_equals_fp64(torch, agj, oracle, name):
    polys, box, eps = _workload(name)
    probe = agj.Index(polys, agj.APPROX, eps, host_only=True)
    pts, _, _ = near_edge_points(oracle, box, probe.stats()["fast_err_cells"], seed={"c1": 1, "c2": 2, "c3": 3}[name])
    d = torch.from_numpy(np.ascontiguousarray(pts)).cuda()
    for mode in (agj.APPROX, agj.EXACT):
        train = pts[::7] if mode == agj.EXACT else None
        fast = agj.Index(polys, mode, eps, train=train)
        slow = agj.Index(polys, mode, eps, train=train, fast_ids=False)
        assert fast.stats()["fast_ids"] == 1 and slow.stats()["fast_ids"] == 0
        pf = agj.join(fast, d)
        of, idf = pf.to_host()
        os_, ids_ = agj.join(slow, d).to_host()
        assert np.array_equal(of, os_) and np.array_equal(idf, ids_)
        assert pf.fallbacks() > 0                 # the ulp-close points needed the FP64 id
        if mode == agj.APPROX:
            cells, ro, refs = fast.logical()
            eo, ei = oracle.join_approx_logical(cells, ro, refs, pts)
        else:
            eo, ei = oracle.PolySet(polys).join_exact(pts)
        assert np.array_equal(of.astype(np.int64), eo.astype(np.int64)) and np.array_equal(idf, ei)
