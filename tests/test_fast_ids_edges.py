"""The certified fast cell ids next to cell edges (no GPU).

The probe's FP32 model of the spec's (i, j) is trusted only on the leading
levels where both ends of its error interval fall in the same cell.  That
is sound as long as the model's error never exceeds the bound the host
derived.  The bound is tested here where it matters: for every level 1-30
with edges inside each workload's window, edges are located exactly in the
spec's FP64 arithmetic (adjacent doubles in different cells), and points at
+-1..4 ulps and at 0.5-8 times the bound from them must get certified
prefixes equal to the oracle ids' prefixes.  The GPU side (the join with
the fast ids equal to the join with FP64 ids on the same points) is in
test_gpu_fast_ids_edges.py.
"""
import numpy as np
import pytest

from _cell_edges import edge_points, prefix_equal


@pytest.fixture(scope="module")
def agj():
    import paper_1802_09488_gb300 as m
    m.lib()
    return m


def _workload(name):
    from paper_1802_09488_gb300 import synth
    if name == "c1":
        return synth.c1_tiny(10).polygons, synth.BOX_C1, 10.0
    if name == "c2":
        return synth.c2_city_polygons(), synth.BOX_CITY, 4.0
    return synth.c3_fine_polygons(4000, seed=5), synth.BOX_CITY, 10.0


def near_edge_points(oracle, box, err, seed):
    """(points, edge level, distance from the edge in units of err; 0 for
    the points a few ulps away) along meridians and parallels."""
    rng = np.random.default_rng(seed)
    win = box.latlng_bounds()
    a = edge_points(oracle, win, range(1, 31), 40, err, rng, axis=0)
    b = edge_points(oracle, win, range(1, 31), 40, err, rng, axis=1)
    return tuple(np.concatenate([x, y]) for x, y in zip(a, b))


@pytest.mark.parametrize("name", ["c1", "c2", "c3"])
def test_certified_prefix_next_to_cell_edges(agj, oracle, name):
    polys, box, eps = _workload(name)
    ix = agj.Index(polys, agj.APPROX, eps, host_only=True)
    st = ix.stats()
    assert st["fast_ids"] == 1
    err = st["fast_err_cells"]
    pts, edge_level, dist = near_edge_points(oracle, box, err, seed={"c1": 1, "c2": 2, "c3": 3}[name])
    assert len(np.unique(edge_level)) >= 15 and len(pts) > 10_000
    ids, lv = ix.fast_ids_host(pts)
    ref = oracle.cell_ids(pts)
    inside = lv != 255
    assert inside.mean() > 0.9
    # every certified prefix is the spec's
    assert prefix_equal(ids[inside], ref[inside], lv[inside]).all()
    # a point a few ulps from a level-L edge has the edge inside its error
    # interval, so it is certified to fewer than L levels
    ulp = inside & (dist == 0)
    assert ulp.sum() > 1000 and (lv[ulp] < edge_level[ulp]).all()
    # the bound is not vacuous: points 2-8 bounds away certify past the edge
    far = inside & (dist >= 2.0)
    assert np.mean(lv[far] >= edge_level[far]) > 0.95
