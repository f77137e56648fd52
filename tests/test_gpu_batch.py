"""GPU parity of the batched form: every job of one batched launch sequence
(agj_batch_run / agj_join_batched) equals the plain join of the same (index,
points) bit for bit, status words included, and the CPU oracle (brute-force
ST_Covers for exact jobs, the sorted-vector probe of the logical covering for
approximate ones).  Jobs mix modes, index sizes and batch sizes, with empty,
one-point and ragged batches; every tiling option of the plan is covered, with
and without the CUDA graph, and plans are re-run on new point buffers."""
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
    return torch.from_numpy(np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 2)).cuda()


@pytest.fixture(scope="module")
def jobs():
    from paper_1802_09488_gb300 import synth
    js = synth.batched_jobs(m=10, seed=3, polys=(5, 300), points=(1_000, 60_000), exact_every=2)
    # edge cases: empty, one point, one warp tile +- 1, invalid points
    sizes = [0, 1, 63, 64, 65, 129]
    for j, n in enumerate(sizes):
        js[j].points = js[j].points[:n]
    bad = np.array([[np.nan, 0.0], [95.0, 1.0], [10.0, 20.0]])
    js[6].points = np.concatenate([bad, js[6].points])
    return js


@pytest.fixture(scope="module")
def indexes(agj, jobs):
    out = []
    for jb in jobs:
        if jb.exact:
            out.append(agj.Index(jb.polygons, agj.EXACT, 0, train=jb.train))
        else:
            out.append(agj.Index(jb.polygons, agj.APPROX, jb.eps_m))
    return out


@pytest.fixture(scope="module")
def expected(torch, agj, oracle, jobs, indexes):
    """Per job: (offsets, ids, status) of the plain join, checked against the oracle."""
    exp = []
    for jb, ix in zip(jobs, indexes):
        pr = agj.join(ix, _dev(torch, jb.points))
        off, ids = pr.to_host()
        st = pr.status.cpu().numpy().copy()
        if jb.exact:
            eo, ei = oracle.PolySet(jb.polygons).join_exact(jb.points.reshape(-1, 2))
        else:
            cells, ro, refs = ix.logical()
            eo, ei = oracle.join_approx_logical(cells, ro, refs, jb.points.reshape(-1, 2))
        assert np.array_equal(np.asarray(off, np.int64), np.asarray(eo, np.int64))
        assert np.array_equal(np.asarray(ids, np.int64), np.asarray(ei, np.int64))
        exp.append((off.copy(), ids.copy(), st))
    return exp


def _check(pairs, expected):
    for j, (pr, (off, ids, st)) in enumerate(zip(pairs, expected)):
        got_off, got_ids = pr.to_host()
        assert np.array_equal(got_off, off), j
        assert np.array_equal(got_ids, ids), j
        assert np.array_equal(pr.status.cpu().numpy(), st), j


@pytest.mark.parametrize("ppt,ctas,graph", [(1, 1, True), (2, 0, True), (2, 3, True), (4, 2, True), (1, 0, False), (4, 1, False)])
def test_batch_equals_plain_and_oracle(torch, agj, jobs, indexes, expected, ppt, ctas, graph):
    b = agj.Batch(indexes, [len(jb.points) for jb in jobs], points_per_lane=ppt, ctas_per_sm=ctas, graph=graph)
    pts = [_dev(torch, jb.points) for jb in jobs]
    pairs = b.pairs()
    for _ in range(2):                       # replay: work space and status are reset each run
        b.run(pts, pairs)
        torch.cuda.synchronize()
        _check(pairs, expected)
    # new point buffers and outputs: the descriptors are uploaded again
    pts2 = [p.clone() for p in pts]
    pairs2 = b.pairs()
    b.run(pts2, pairs2)
    torch.cuda.synchronize()
    _check(pairs2, expected)
    b.close()


def test_join_batched_one_shot(torch, agj, jobs, indexes, expected):
    pairs = agj.join_batched(indexes, [_dev(torch, jb.points) for jb in jobs])
    _check(pairs, expected)


def test_batch_single_job_and_reordered(torch, agj, jobs, indexes, expected):
    """A plan of one job, and the jobs in reverse order (other tile and
    polygon offsets), give the same per-job output."""
    k = 9
    b = agj.Batch([indexes[k]], [len(jobs[k].points)])
    pr = b.run([_dev(torch, jobs[k].points)], b.pairs())
    torch.cuda.synchronize()
    _check(pr, [expected[k]])
    rev = list(range(len(jobs)))[::-1]
    b = agj.Batch([indexes[j] for j in rev], [len(jobs[j].points) for j in rev])
    pr = b.run([_dev(torch, jobs[j].points) for j in rev], b.pairs())
    torch.cuda.synchronize()
    _check(pr, [expected[j] for j in rev])


def test_batch_rejects_small_outputs(torch, agj, jobs, indexes):
    b = agj.Batch(indexes[6:8], [len(jobs[6].points), len(jobs[7].points)])
    pairs = b.pairs()
    pairs[1].c.ids_capacity = 0
    with pytest.raises(agj.AgjError):
        b.run([_dev(torch, jobs[6].points), _dev(torch, jobs[7].points)], pairs)


@pytest.mark.parametrize("which", ["approx", "exact"])
def test_batch_single_mode_plans(torch, agj, jobs, indexes, expected, which):
    """Plans whose jobs are all approximate (no refine step, no candidate
    work space) or all exact."""
    sel = [j for j, jb in enumerate(jobs) if jb.exact == (which == "exact")]
    for ppt, ctas in ((2, 0), (4, 3)):
        b = agj.Batch([indexes[j] for j in sel], [len(jobs[j].points) for j in sel], points_per_lane=ppt,
                      ctas_per_sm=ctas)
        pr = b.run([_dev(torch, jobs[j].points) for j in sel], b.pairs())
        torch.cuda.synchronize()
        _check(pr, [expected[j] for j in sel])
        b.close()


@pytest.fixture(scope="module")
def big_jobs(agj):
    """Two city-scale jobs (one approximate, one exact, 3.2e6 points each):
    enough tiles that a mixed plan launches each mode's probe and emit on
    its own."""
    from paper_1802_09488_gb300 import synth
    polys = synth.c2_city_polygons()
    pts = synth.points_mixture(6_400_000, synth.BOX_CITY, seed=21, dist_seed=3)
    train = synth.points_mixture(100_000, synth.BOX_CITY, seed=22, dist_seed=3)
    ia = agj.Index(polys, agj.APPROX, 4.0)
    ie = agj.Index(polys, agj.EXACT, 0, train=train)
    return polys, [(ia, pts[:3_200_000]), (ie, pts[3_200_000:])]


@pytest.mark.parametrize("ppt,ctas,graph", [(2, 0, True), (1, 3, True), (2, 0, False)])
def test_batch_mode_split_launches(torch, agj, oracle, jobs, indexes, expected, big_jobs, ppt, ctas, graph):
    """A mixed plan over 1e5+ tiles (each mode's probe, scan and emit on its
    own tiles; with the graph the two chains are parallel branches; one warp
    per tile and persistent): every job equals its plain join, and sampled
    rows of the big jobs equal the oracle."""
    polys, big = big_jobs
    ix = [b[0] for b in big] + indexes
    pts = [b[1] for b in big] + [jb.points for jb in jobs]
    b = agj.Batch(ix, [len(p) for p in pts], points_per_lane=ppt, ctas_per_sm=ctas, graph=graph)
    dev = [_dev(torch, p) for p in pts]
    pr = b.pairs()
    for _ in range(2):                       # replay: both chains' scan states and tickets are reset
        b.run(dev, pr)
    torch.cuda.synchronize()
    _check(pr[2:], expected)
    rng = np.random.default_rng(5)
    ps = oracle.PolySet(polys)
    for k, (index, p) in enumerate(big):
        plain = agj.join(index, _dev(torch, p))
        off, ids = plain.to_host()
        got_off, got_ids = pr[k].to_host()
        assert np.array_equal(got_off, off) and np.array_equal(got_ids, ids), k
        assert np.array_equal(pr[k].status.cpu().numpy(), plain.status.cpu().numpy()), k
        rows = np.sort(rng.choice(len(p), 2000, replace=False))
        if k == 1:
            eo, ei = ps.join_exact(p[rows])
        else:
            cells, ro, refs = index.logical()
            eo, ei = oracle.join_approx_logical(cells, ro, refs, p[rows])
        for r, row in enumerate(rows):
            assert list(ids[off[row]:off[row + 1]]) == list(ei[eo[r]:eo[r + 1]]), (k, row)
    b.close()
