"""GPU tests of the served form: requests served by continuous batching
(many requests per launch, several launches in flight) give exactly the
plain join's CSR for their points - alone and in the mix - and the CPU
oracle's; the Poisson load generator and the plain per-request baseline
run and account for every request."""
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


@pytest.fixture(scope="module")
def sets(agj):
    """Two polygon sets, each with an approximate (eps 4 m) and an exact
    index, and a point pool per set."""
    from paper_1802_09488_gb300 import synth
    out = []
    for k, (n_polys, box) in enumerate([(5, synth.BOX_C1), (60, synth.BOX_CITY)]):
        polys = synth.voronoi_tiling(n_polys, box, seed=50 + k, vmin=8 if n_polys <= 16 else 20,
                                     vmax=64 if n_polys <= 16 else 200)
        pool = synth.points_mixture(200_000, box, seed=60 + k)
        ax = agj.Index(polys, agj.APPROX, 4.0)
        ex = agj.Index(polys, agj.EXACT, 0, train=pool[:2000])
        out.append((polys, pool, ax, ex))
    return out


def _indexes(sets):
    return [s[2] for s in sets] + [s[3] for s in sets]   # ids: approx 0..S-1, exact S..2S-1


def _requests(sets, count, seed, max_points=4000):
    rng = np.random.default_rng(seed)
    S = len(sets)
    reqs = []
    for i in range(count):
        s = int(rng.integers(0, S))
        exact = bool(rng.random() < 0.3)
        n = int(min(max_points, np.floor(rng.pareto(1.2)) + 1))
        if i % 50 == 7:
            n = 0 if i % 100 == 7 else 1
        start = int(rng.integers(0, sets[s][1].shape[0] - max(n, 1)))
        reqs.append((s + (S if exact else 0), sets[s][1][start:start + n]))
    return reqs


def _plain(torch, agj, ix, pts):
    if len(pts) == 0:
        return np.zeros(1, np.uint32), np.zeros(0, np.uint32)
    pr = agj.join(ix, torch.from_numpy(np.ascontiguousarray(pts)).cuda())
    off, ids = pr.to_host()
    return off.copy(), ids.copy()


@pytest.mark.parametrize("stage_points", [False, True])
def test_server_mix_equals_alone_and_plain(torch, agj, oracle, sets, stage_points):
    """Points read by the kernels from the client's host buffers (where the
    device reads pageable memory) or staged through pinned buffers."""
    idx = _indexes(sets)
    reqs = _requests(sets, 600, seed=1)
    srv = agj.Server(idx, n_slots=3, max_step_requests=256, max_step_points=1 << 16, stage_points=stage_points)
    assert srv.stats()["host_reads"] in (0, 1)
    if stage_points:
        assert srv.stats()["host_reads"] == 0
    tickets = [srv.submit(i, p) for i, p in reqs]          # a burst: many requests per launch
    mixed = [srv.poll(t) for t in tickets]
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["steps"] < len(reqs) and st["step_requests_max"] > 1
    steps = np.array([m[2]["step"] for m in mixed])
    assert len(np.unique(steps)) < len(reqs)
    for k in range(0, len(reqs), 7):                       # alone: one request per launch
        i, p = reqs[k]
        off, ids, res = srv.poll(srv.submit(i, p))
        assert np.array_equal(off, mixed[k][0]) and np.array_equal(ids, mixed[k][1]), k
    for k, (i, p) in enumerate(reqs):
        off, ids = _plain(torch, agj, idx[i], p)
        assert np.array_equal(mixed[k][0], off), k
        assert np.array_equal(mixed[k][1], ids), k
        assert mixed[k][2]["nnz"] == len(ids)
        r = mixed[k][2]
        assert r["t_submit_ns"] <= r["t_start_ns"] <= r["t_done_ns"]
    # a few requests against the oracle directly
    S = len(sets)
    for k in range(0, len(reqs), 97):
        i, p = reqs[k]
        polys = sets[i % S][0]
        if len(p) == 0:
            continue
        if i >= S:
            eo, ei = oracle.PolySet(polys).join_exact(p)
        else:
            cells, ro, refs = idx[i].logical()
            eo, ei = oracle.join_approx_logical(cells, ro, refs, p)
        assert np.array_equal(np.asarray(mixed[k][0], np.int64), np.asarray(eo, np.int64))
        assert np.array_equal(np.asarray(mixed[k][1], np.int64), np.asarray(ei, np.int64))
    srv.close()


def test_server_limits(torch, agj, sets):
    idx = _indexes(sets)
    srv = agj.Server(idx, n_slots=1, max_step_requests=4, max_step_points=1000)
    with pytest.raises(agj.AgjError):
        srv.submit(0, sets[0][1][:1001])                   # larger than a launch
    # more requests than a launch takes: served over several launches
    ts = [srv.submit(1, sets[1][1][k * 300:(k + 1) * 300]) for k in range(10)]
    outs = [srv.poll(t) for t in ts]
    assert len({o[2]["step"] for o in outs}) >= 3
    for k, o in enumerate(outs):
        off, ids = _plain(torch, agj, idx[1], sets[1][1][k * 300:(k + 1) * 300])
        assert np.array_equal(o[0], off) and np.array_equal(o[1], ids)
    srv.close()


def test_server_and_plain_load(torch, agj, sets):
    idx = _indexes(sets)
    S = len(sets)
    spec = agj.LoadSpecPy(rate=20_000, n_requests=3000, pools=[s[1] for s in sets], approx_index=list(range(S)),
                          exact_index=list(range(S, 2 * S)), zipf_alpha=1.2, max_points=8192, exact_fraction=0.1,
                          seed=5, warmup_requests=300)
    srv = agj.Server(idx, n_slots=4, max_step_points=1 << 17)
    r = srv.load(spec)
    # unaligned client buffers are staged, aligned ones read in place
    raw = np.empty(2 * 5000 + 1, dtype=np.float64)
    odd = raw[1:].reshape(-1, 2)
    odd[:] = sets[1][1][:5000]
    off, ids, _ = srv.poll(srv.submit(1, odd))
    ref = _plain(torch, agj, idx[1], sets[1][1][:5000])
    assert np.array_equal(off, ref[0]) and np.array_equal(ids, ref[1])
    assert r["requests"] == 2700 and r["rejected"] == 0
    assert 0 < r["p50_us"] <= r["p99_us"] <= r["max_us"]
    assert r["points_per_s"] > 0
    srv.close()
    spec_small = agj.LoadSpecPy(rate=20_000, n_requests=500, pools=[s[1] for s in sets], approx_index=list(range(S)),
                                exact_index=list(range(S, 2 * S)), zipf_alpha=1.2, max_points=8192,
                                exact_fraction=0.1, seed=5, warmup_requests=50)
    p = agj.plain_load(idx, spec_small)
    assert p["requests"] == 450 and p["p50_us"] > 0


def test_server_admission_by_device_memory(torch, agj, sets):
    """An arena of 1.3 times the largest request's launch bytes: no two
    requests fit it together, so every launch holds one request and the
    peak use stays within the budget, while the four slots keep trying to
    launch the next request before the previous one has returned its
    memory (the scheduler waits); every result equals its plain join.  A
    request that could never fit the arena is refused at submit."""
    idx = _indexes(sets)
    rng = np.random.default_rng(3)
    reqs = []
    for k in range(60):              # 15 000 - 20 000 points: any two exceed 1.3 x the largest
        s_ = int(rng.integers(0, len(sets)))
        n = int(rng.integers(15_000, 20_001))
        start = int(rng.integers(0, sets[s_][1].shape[0] - n))
        reqs.append((s_ + (len(sets) if k % 3 == 2 else 0), sets[s_][1][start:start + n]))
    # the launch bytes of the largest request: one slot, one request per launch
    probe = agj.Server(idx, n_slots=1, max_step_requests=1, max_step_points=1 << 15, stage_points=True)
    for t in [probe.submit(i, p) for i, p in reqs]:
        probe.poll(t)
    one = probe.stats()["peak_bytes_in_use"]
    probe.close()
    assert one > 0
    budget = int(1.3 * one)
    srv = agj.Server(idx, n_slots=4, max_step_requests=256, max_step_points=1 << 16, hbm_budget_bytes=budget,
                     stage_points=True)
    assert srv.stats()["device_bytes"] <= budget
    tickets = [(srv.submit(i, p), i, p) for i, p in reqs]
    outs = [(srv.poll(t), i, p) for t, i, p in tickets]
    st = srv.stats()
    assert st["steps"] == len(reqs) and st["step_requests_max"] == 1
    assert 0 < st["peak_bytes_in_use"] <= budget and st["memory_waits"] > 0
    for (off, ids, res), i, p in outs:
        ref = _plain(torch, agj, idx[i], p)
        assert np.array_equal(off, ref[0]) and np.array_equal(ids, ref[1])
    srv.close()
    # an arena below one request of max_step_points: large requests refused, small ones served
    tiny = agj.Server(idx, n_slots=2, max_step_requests=64, max_step_points=1 << 16, hbm_budget_bytes=4 << 20,
                      stage_points=True)
    with pytest.raises(agj.AgjError) as e:
        tiny.submit(3, sets[1][1][:60_000])
    assert e.value.status == 3
    off, ids, _ = tiny.poll(tiny.submit(3, sets[1][1][:500]))
    ref = _plain(torch, agj, idx[3], sets[1][1][:500])
    assert np.array_equal(off, ref[0]) and np.array_equal(ids, ref[1])
    tiny.close()
    # a budget above the free device memory is refused at creation
    free, _ = torch.cuda.mem_get_info()
    with pytest.raises(agj.AgjError) as e:
        agj.Server(idx, hbm_budget_bytes=free + (1 << 30))
    assert e.value.status == 3


def test_server_admits_indexes_by_free_memory(torch, agj, sets):
    """agj_server_add_index uploads a host-built index when it fits the free
    device memory less the reserve (requests to it then equal the plain
    join), and refuses it with AGJ_EBUDGET when the reserve leaves no room,
    while requests in flight keep running."""
    from paper_1802_09488_gb300 import synth
    idx = _indexes(sets)
    polys = synth.voronoi_tiling(40, synth.BOX_CITY, seed=71, vmin=20, vmax=120)
    pts = synth.points_mixture(50_000, synth.BOX_CITY, seed=72)
    srv = agj.Server(idx, n_slots=2, max_step_points=1 << 16)
    busy = [srv.submit(1, sets[1][1][k * 5000:(k + 1) * 5000]) for k in range(20)]   # in flight meanwhile
    host_a = agj.Index(polys, agj.APPROX, 4.0, host_only=True)
    host_e = agj.Index(polys, agj.EXACT, 0, train=pts[:5000], host_only=True)
    ka, ke = srv.add_index(host_a), srv.add_index(host_e)
    st = srv.stats()
    assert (ka, ke) == (len(idx), len(idx) + 1) and st["n_indexes"] == len(idx) + 2 and st["index_bytes"] > 0
    for k in (ka, ke):
        off, ids, _ = srv.poll(srv.submit(k, pts))
        ref = _plain(torch, agj, srv.indexes[k], pts)       # now resident: joinable directly too
        assert np.array_equal(off, ref[0]) and np.array_equal(ids, ref[1])
    for t in busy:
        srv.poll(t)
    srv.close()
    # a reserve as large as the free memory: no index fits
    free, _ = torch.cuda.mem_get_info()
    srv = agj.Server(idx, n_slots=1, max_step_requests=4, max_step_points=1 << 12,
                     hbm_reserve_bytes=free - (16 << 20))     # a small arena, then ~14 MB beyond the reserve
    assert agj.Index(polys, agj.APPROX, 4.0, host_only=True).stats()["n_nodes"] * 2048 > 16 << 20
    with pytest.raises(agj.AgjError) as e:
        srv.add_index(agj.Index(polys, agj.APPROX, 4.0, host_only=True))
    assert e.value.status == 3 and srv.stats()["n_indexes"] == len(idx)
    srv.close()
