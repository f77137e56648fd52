"""Training from a device point stream (agj_train_online, §III-D).

The device pass returns only the points that land in cells with candidate
references; the host trainer splits those cells.  Since points elsewhere
cannot change training, the index trained this way must equal the one
agj_build trains on the host from the same points and budget: same logical
covering, cell for cell and reference for reference.  The exact join's
output does not change (it is the brute-force ST_Covers result before and
after), while fewer candidates reach the refine step.
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


def test_online_training_equals_host_training(torch, agj, oracle):
    from paper_1802_09488_gb300 import synth
    polys = synth.c2_city_polygons()
    train = synth.points_mixture(1_000_000, synth.BOX_CITY, seed=4, dist_seed=3)
    pts = synth.points_mixture(2_000_000, synth.BOX_CITY, seed=5, dist_seed=3)
    d_pts = torch.from_numpy(pts).cuda()
    online = agj.Index(polys, agj.EXACT, 0)
    before = agj.join(online, d_pts)
    off0, ids0 = before.to_host()
    cand0 = int(before.status.cpu().numpy()[2])
    nodes0 = online.stats()["n_nodes"]
    budget = 64 << 20
    agj.train_online(online, torch.from_numpy(train).cuda(), budget_bytes=budget)
    host = agj.Index(polys, agj.EXACT, 0, train=train, budget_bytes=budget, host_only=True)
    for a, b in zip(online.logical(), host.logical()):
        assert np.array_equal(a, b)
    st = online.stats()
    assert st["n_nodes"] > nodes0 and st["n_nodes"] == host.stats()["n_nodes"]
    after = agj.join(online, d_pts)
    off1, ids1 = after.to_host()
    assert np.array_equal(off0, off1) and np.array_equal(ids0, ids1)
    eo, ei = oracle.PolySet(polys).join_exact(pts)
    assert np.array_equal(off1.astype(np.int64), eo.astype(np.int64)) and np.array_equal(ids1, ei)
    cand1 = int(after.status.cpu().numpy()[2])
    assert cand1 < 0.7 * cand0, (cand0, cand1)
    # a second stream keeps refining within a larger budget; output still exact
    agj.train_online(online, torch.from_numpy(pts[:500_000]).cuda(), budget_bytes=2 * budget)
    assert online.stats()["n_nodes"] >= st["n_nodes"]
    off2, ids2 = agj.join(online, d_pts).to_host()
    assert np.array_equal(off2, off1) and np.array_equal(ids2, ids1)


def test_online_training_refuses_approximate_indexes(torch, agj):
    from paper_1802_09488_gb300 import synth
    w = synth.c1_tiny(1000)
    ix = agj.Index(w.polygons, agj.APPROX, w.eps_m)
    with pytest.raises(agj.AgjError) as e:
        agj.train_online(ix, torch.from_numpy(w.points).cuda())
    assert e.value.status == 1
