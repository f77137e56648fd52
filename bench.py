#!/usr/bin/env python3
"""Benchmark of the probe side of the adaptive geospatial join on one GB300.

Workload (city-scale plain join): 300 Voronoi polygons (20-400 vertices)
tiling a 45 km x 50 km box and 1e8 FP64 points from a 32-cluster Gaussian
mixture plus 20 % uniform noise (seeded, synthetic stand-ins for the paper's
NYC neighbourhoods and taxi points).  One step joins the same device-resident
points twice: once against the approximate index (eps = 4 m) and once
against the exact index (trained on a 1 % sample), so `value` counts 2 n
point-joins per step.  Points (1.6 GB) exceed L2, so no flush is needed
between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank holds its own index replica and joins its own 1e8
points (weak scaling); the join has no collective.  `--impl reference` times
the CPU oracle (the reference for this method) on bounded samples of the same
workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "points joined/sec at 1 GB300 (approx eps and exact) vs plain join; p50/p99 latency"
# approx: k_zero, k_probe<approx>, k_scan_counts, k_emit<approx>
# exact:  k_zero, k_probe<exact>, k_count, k_poly_scan, k_scatter, k_pip, k_scan_counts, k_emit<exact>
LAUNCHES_PER_STEP = {"approx": 4, "exact": 8}
# DRAM bytes (read + write) per point of the probe kernels on the city workload,
# from one `ncu --set full` capture of a 16e6-point join of the current kernels
# (dram__bytes_read.sum + dram__bytes_write.sum divided by the points); a full
# launch's traffic scales with its points (the trie gathers per point do not
# depend on n).  Re-captured whenever a probe kernel changes (empty: the
# kernels changed since the last capture, traffic reported as null).  The
# last capture (25.6 and 26.2 B per point) predates the probes' current
# wait loop for their shared tables, so the figures are not reported.
PROBE_DRAM_BYTES_PER_POINT = {}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n-points", type=int, default=100_000_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the batched and served forms")
    ap.add_argument("--extras", default="count,cellid,c1,onepass",
                    help="comma list of extra measurements: count (aggregation mode), cellid (the FP64 cell-id "
                         "kernel), c1 (1000 tiny joins in one graph), onepass (the one-pass approximate join "
                         "against the three-kernel one); empty for none")
    ap.add_argument("--workload", choices=["c2", "c3", "c1"], default="c2",
                    help="c2: city (default); c3: 40 000 fine overlapping polygons; c1: 5 polygons, uniform points")
    ap.add_argument("--eps", type=float, default=None, help="approximate precision in metres (default per workload)")
    ap.add_argument("--only", choices=["batched", "served", "sort-study"], default=None,
                    help="run only that form (or the sort-prepass study) and print its JSON object")
    ap.add_argument("--form-reps", type=int, default=10, help="timed repetitions of the batched form")
    ap.add_argument("--batched-tiling", default=None, help="points_per_lane,ctas_per_sm: skip the autotuner")
    ap.add_argument("--c4-polys", default=None,
                    help="lo,hi polygons per set of the batched form (default 5,300; the workload's own range is "
                         "5,40000)")
    ap.add_argument("--c4-jobs", type=int, default=None, help="jobs of the batched form (default 64)")
    return ap.parse_args()


# Batched form: 64 (polygon set, point batch) jobs, polygon counts and batch
# sizes log-uniform (per-job seeds), every second job exact.  The polygon
# range is cut from 5-40 000 to 5-300 so that generating and indexing the
# 64 sets stays within the bench's time budget.
C4 = {"m": 64, "seed": 11, "polys": (5, 300), "points": (1_000, 10_000_000)}
# Served form: 16 resident sets (approximate eps = 4 m and exact index each),
# Poisson arrivals at 2e5 requests/s, sizes 1-65 536 Zipf(1.2), 10 % exact.
# Set sizes cut from 300-40 000 to 300-1 500 polygons for the same reason.
C5 = {"sets": 16, "polys": (300, 1500), "rate": 2e5, "requests": 300_000, "warmup": 50_000, "zipf": 1.2,
      "max_points": 65536, "exact_fraction": 0.1, "plain_requests": 5_000, "saturate_rate": 4e6}


def batched_form(agj, torch, reps: int = 10, tiling=None, polys=None, m=None) -> dict:
    """64 plain joins in sequence vs one batched plan (graph replay) over the
    same jobs, with the autotuned tiling; outputs compared job by job."""
    import numpy as np
    from paper_1802_09488_gb300 import autotune, synth
    t0 = time.perf_counter()
    polys = polys or C4["polys"]
    m = m or C4["m"]
    jobs = synth.batched_jobs(m=m, seed=C4["seed"], polys=polys, points=C4["points"])
    idx = [agj.Index(j.polygons, agj.EXACT, 0, train=j.train) if j.exact else agj.Index(j.polygons, agj.APPROX, j.eps_m)
           for j in jobs]
    prep_s = time.perf_counter() - t0
    pts = [torch.from_numpy(j.points).cuda() for j in jobs]
    ns = [len(j.points) for j in jobs]
    N = sum(ns)
    s = torch.cuda.current_stream()
    plain_pairs = [agj.Pairs(ix, n) for ix, n in zip(idx, ns)]

    def time_it(fn):
        for _ in range(1 if reps == 1 else 3):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            fn()
            b.record(s)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return sorted(ts)[len(ts) // 2]

    def plain():
        for ix, p, pr in zip(idx, pts, plain_pairs):
            agj.join(ix, p, pr)

    plain_ms = time_it(plain)
    ref = [pr.to_host() for pr in plain_pairs]
    if tiling is None:
        tuned = autotune.tune(idx, pts, use_cache=False)
    else:
        tuned = {"points_per_lane": tiling[0], "ctas_per_sm": tiling[1], "sweep": None}
    plan = agj.Batch(idx, ns, points_per_lane=tuned["points_per_lane"], ctas_per_sm=tuned["ctas_per_sm"])
    bp = plan.pairs()
    batch_ms = time_it(lambda: plan.run(pts, bp))
    same = all(np.array_equal(a[0], b.to_host()[0]) and np.array_equal(a[1], b.to_host()[1]) for a, b in zip(ref, bp))
    out = {"workload": (f"c4{'' if polys == (5, 40_000) else '-reduced'}: {m} jobs, polygons log-uniform "
                        f"{polys[0]}-{polys[1]}, "
                        f"points log-uniform {C4['points'][0]:.0e}-{C4['points'][1]:.0e}, every 2nd job exact"),
           "points": N, "plain_ms": plain_ms, "batched_ms": batch_ms,
           "plain_points_per_s": N / (plain_ms / 1e3), "batched_points_per_s": N / (batch_ms / 1e3),
           "speedup_vs_plain": plain_ms / batch_ms, "identical_output": bool(same),
           "tiling": {"points_per_lane": tuned["points_per_lane"], "ctas_per_sm": tuned["ctas_per_sm"],
                      "sweep": tuned["sweep"]},
           "graph": True, "prep_s": prep_s}
    plan.close()
    return out


def served_form(agj) -> dict:
    """Poisson requests through the server (continuous batching) vs the same
    arrivals served one plain join per request."""
    import numpy as np
    from paper_1802_09488_gb300 import synth
    t0 = time.perf_counter()
    rng = np.random.default_rng(21)
    lo, hi = C5["polys"]
    sizes = np.exp(rng.uniform(np.log(lo), np.log(hi), C5["sets"])).round().astype(int)
    pools, idx_a, idx_e = [], [], []
    for k, npl in enumerate(sizes):
        polys = synth.voronoi_tiling(int(npl), synth.BOX_CITY, seed=300 + k, vmin=20, vmax=400) if npl <= 1000 \
            else synth.c3_fine_polygons(int(npl), seed=300 + k)
        pools.append(synth.points_mixture(1 << 20, synth.BOX_CITY, seed=400 + k, dist_seed=300 + k))
        idx_a.append(agj.Index(polys, agj.APPROX, 4.0))
        idx_e.append(agj.Index(polys, agj.EXACT, 0, train=pools[-1][:10_000]))
    idx = idx_a + idx_e
    S = C5["sets"]
    prep_s = time.perf_counter() - t0

    def spec(rate, n, warm):
        return agj.LoadSpecPy(rate=rate, n_requests=n, pools=pools, approx_index=list(range(S)),
                              exact_index=list(range(S, 2 * S)), zipf_alpha=C5["zipf"], max_points=C5["max_points"],
                              exact_fraction=C5["exact_fraction"], seed=7, warmup_requests=warm)

    srv = agj.Server(idx, n_slots=4, max_step_points=1 << 20)
    r = srv.load(spec(C5["rate"], C5["requests"], C5["warmup"]))
    st = srv.stats()
    srv.close()
    srv = agj.Server(idx, n_slots=4, max_step_points=1 << 22)     # larger launches for the saturated run
    sat = srv.load(spec(C5["saturate_rate"], int(C5["saturate_rate"] // 2), int(C5["saturate_rate"] // 8)))
    srv.close()
    p = agj.plain_load(idx, spec(C5["rate"], C5["plain_requests"], C5["plain_requests"] // 10))
    keys = ("achieved_rate", "points_per_s", "p50_us", "p99_us", "mean_us", "max_us", "requests", "rejected")
    return {"workload": (f"c5-reduced: {S} resident sets of {lo}-{hi} polygons (approx eps 4 m + exact index each), "
                         f"Poisson {C5['rate']:.0e} req/s, Zipf({C5['zipf']}) sizes 1-{C5['max_points']}, "
                         f"{C5['exact_fraction']:.0%} exact"),
            "served": {k: r[k] for k in keys} | {"steps": st["steps"], "max_requests_per_step": st["step_requests_max"],
                                                 "slots": st["n_slots"], "slot_device_bytes": st["device_bytes"],
                                                 "points_read_from_host_memory": bool(st["host_reads"])},
            "served_saturated": {k: sat[k] for k in keys} | {"offered_rate": sat["offered_rate"]},
            "plain_per_request": {k: p[k] for k in keys},
            "speedup_points_per_s_vs_plain": r["points_per_s"] / max(p["points_per_s"], 1e-9),
            "capacity_vs_plain": sat["points_per_s"] / max(p["points_per_s"], 1e-9),
            "index_device_bytes": sum(ix.stats()["device_bytes"] for ix in idx), "prep_s": prep_s}


def _event(torch, stream):
    """A timing event whose CUDA handle exists (torch creates it on the first
    record), so that the library can record it."""
    e = torch.cuda.Event(enable_timing=True)
    e.record(stream)
    return e


def count_mode(agj, torch, ia, ie, d_pts, n, peaks, steps) -> dict:
    """Aggregation mode (count(*) group by polygon, §V) on the same resident
    points and indexes: per-mode points/s and the count probe's roofline
    (16 B point + 8 B per trie entry read; no per-point output)."""
    import numpy as np
    s = torch.cuda.current_stream()
    out = {}
    for name, ix in (("approx", ia), ("exact", ie)):
        c = agj.join_count(ix, d_pts)
        c.to_host()
        evs = [[_event(torch, s) for _ in range(4)] for _ in range(max(steps, 3))]
        for ev in evs:
            agj.join_count(ix, d_pts, c, events=ev)
        torch.cuda.synchronize()
        counts = c.to_host()
        st = c.status.cpu().numpy().view(np.uint64)
        total = [ev[0].elapsed_time(ev[3]) for ev in evs]
        probe = [ev[0].elapsed_time(ev[1]) for ev in evs]
        g = float(st[3]) / n
        bpp = 16 + 8 * g
        tp = statistics.mean(probe)
        out[name] = {"points_per_s": n / (statistics.mean(total) / 1e3), "ms": statistics.mean(total),
                     "probe_ms": tp, "pairs_counted": int(st[0]), "polygons_nonzero": int((counts > 0).sum()),
                     "trie_entries_read_per_point": g,
                     "roofline_probe": {"kernel": f"k_agg_probe_{name}", "bound": "hbm",
                                        "achieved": bpp * n / (tp / 1e3) / 1e9, "peak": peaks["hbm_gbs"],
                                        "unit": "GB/s", "frac": bpp * n / (tp / 1e3) / 1e9 / peaks["hbm_gbs"],
                                        "algorithmic_bytes_per_point": bpp, "peak_source": peaks["source"]}}
    return out


# FP64 operations per point of the cell-id kernel at source level
# (agj_geom.cuh): two sin/cos of degrees (reduction 4, Horner 14 + 16,
# assembly 5, squares 1: 40 each), the xyz products (2), two divisions for
# (u, v), two quadratic st transforms (4-5 each: 9 on this site's face,
# one coordinate negative), two scalings before the floors (2).  Each
# division and square root counts once here, although the GPU expands
# them into several FP64 instructions.
CELL_ID_FP64_OPS = 95


def one_pass(agj, torch, ia, d_pts, reps: int = 10) -> dict:
    """The one-pass approximate join (probe, per-tile look-back scan and emit
    in one kernel; the allocation-free entry point, at most 2^24 points)
    against the three-kernel join (probe, scan, emit) on the same first
    2^24 - 1 resident points, both into device outputs."""
    import ctypes as C
    import numpy as np
    n = min(int(d_pts.shape[0]), (1 << 24) - 1)
    pts = d_pts[:n]
    L = agj.lib()
    fn = L.agj_join_approx_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p]
    cap = n * max(ia.stats()["max_refs"], 1)
    off = torch.empty(n + 1, dtype=torch.int32, device="cuda")
    ids = torch.empty(cap, dtype=torch.int32, device="cuda")
    st = torch.empty(4, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream()

    def run_one():
        rc = fn(ia.handle, C.c_void_p(pts.data_ptr()), n, C.c_void_p(off.data_ptr()), C.c_void_p(ids.data_ptr()), cap,
                C.c_void_p(st.data_ptr()), C.c_void_p(s.cuda_stream))
        assert rc == 0

    pr = agj.Pairs(ia, n)

    def timed(fn_):
        fn_()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = _event(torch, s), _event(torch, s)
            a.record(s)
            fn_()
            b.record(s)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    t1 = timed(run_one)
    t3 = timed(lambda: agj.join(ia, pts, pr))
    o3, i3 = pr.to_host()
    same = bool(np.array_equal(off.cpu().numpy().view(np.uint32), o3) and
                np.array_equal(ids[:len(i3)].cpu().numpy().view(np.uint32), i3))
    return {"points": n, "one_pass_ms": t1, "three_kernel_ms": t3, "identical_output": same,
            "note": "one-pass: k_join_approx (4 points per lane, a look-back per warp tile); three-kernel: "
                    "k_probe, k_scan_counts, k_emit"}


def cell_id_kernel(agj, torch, d_pts, n) -> dict:
    """k_cell_ids (the FP64 spec path, bit-exact ids) on the resident points,
    reported against the device's FP64 rate measured by the library's own
    FMA microbenchmark."""
    ids = torch.empty(n, dtype=torch.int64, device="cuda")
    agj.cell_ids(d_pts, out=ids)
    ts = []
    for _ in range(5):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        agj.cell_ids(d_pts, out=ids)
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b))
    del ids
    fp64 = agj.measure_fp64_rate()
    ms = statistics.median(ts)
    achieved = CELL_ID_FP64_OPS * n / (ms / 1e3)
    return {"kernel": "k_cell_ids", "ms": ms, "points_per_s": n / (ms / 1e3), "bound": "fp64",
            "fp64_ops_per_point": CELL_ID_FP64_OPS, "achieved_tflops": achieved / 1e12,
            "peak_tflops": fp64 / 1e12, "frac": achieved / fp64,
            "peak_source": "measured by agj_measure_fp64_rate (own FMA-chain kernel, 2 flops per FMA)",
            "note": "divisions and square roots counted as one operation each"}


def c1_amortized(agj, torch, peaks, joins: int = 1000) -> dict:
    """Config 1 (5 polygons, 1e5 points) is launch-bound as single joins; this
    captures `joins` back-to-back approximate joins in one CUDA graph and
    reports the amortized time per join against the method's bytes."""
    import numpy as np
    from paper_1802_09488_gb300 import synth
    w = synth.c1_tiny(100_000)
    ix = agj.Index(w.polygons, agj.APPROX, w.eps_m)
    d = torch.from_numpy(w.points).cuda()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        pr = agj.join(ix, d)
        pr.check()
        st = pr.status.cpu().numpy().view(np.uint64)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            for _ in range(joins):
                agj.join(ix, d, pr)
        g.replay()
        s.synchronize()
        ts = []
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            g.replay()
            b.record(s)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        nnz = pr.check(stream=s)
    ms = min(ts) / joins
    n = len(w.points)
    bpp = 16 + 8 * float(st[3]) / n + 4 + 4 * nnz / n
    ach = bpp * n / (ms / 1e3) / 1e9
    return {"workload": "c1-tiny-5polys-uniform-points-1e05, approx eps 10 m", "joins_in_graph": joins,
            "ms_per_join": ms, "points_per_s": n / (ms / 1e3),
            "roofline_join": {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                              "frac": ach / peaks["hbm_gbs"], "algorithmic_bytes_per_point": bpp,
                              "note": "inputs (1.6 MB) stay in L2 across the graph's joins: a warm-cache figure"}}


def sort_study(agj, torch, workload_name: str, n: int, reps: int = 5) -> dict:
    """What a sort-points-by-cell prepass could gain: the probe on points
    already sorted by cell id (the prepass's best case, its own cost left
    out) against the same points in stream order, and the prepass's cost
    itself (FP64 cell ids, a radix sort of (id, position) by the library,
    the gather of the points and the scatter of the results back to stream
    order, 12 B per point), on the workload's resident points."""
    polys, pts_np, train = workload(workload_name, n, 0)
    eps = WORKLOADS[workload_name]["eps"]
    out = {"workload": f"{WORKLOADS[workload_name]['name']}-{n:.0e}".replace("+", "")}
    d = torch.from_numpy(pts_np).cuda()
    ev = [_event(torch, torch.cuda.current_stream()) for _ in range(4)]

    def probe_ms(ix, pts, pr):
        ts = []
        for _ in range(reps + 1):
            agj.join_timed(ix, pts, pr, ev)
            torch.cuda.synchronize()
            ts.append(ev[0].elapsed_time(ev[1]))
        return statistics.median(ts[1:])

    def timed(fn):
        ts = []
        for _ in range(reps + 1):
            a, b = _event(torch, torch.cuda.current_stream()), _event(torch, torch.cuda.current_stream())
            a.record()
            fn()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts[1:])

    ids = agj.cell_ids(d)
    order = torch.sort(ids, stable=True).indices
    d_sorted = d[order].contiguous()
    results = torch.empty(n, dtype=torch.int64, device="cuda")
    src = torch.empty(n, dtype=torch.int64, device="cuda")

    def prepass():
        k = agj.cell_ids(d, out=ids)
        o = torch.sort(k, stable=True).indices
        torch.index_select(d, 0, o, out=d_sorted)
        results.index_copy_(0, o, src)            # the results' way back to stream order

    out["prepass_ms"] = timed(prepass)
    for mode_name, mode in (("approx", agj.APPROX), ("exact", agj.EXACT)):
        ix = agj.Index(polys, mode, eps, train=train if mode == agj.EXACT else None)
        pr = agj.Pairs(ix, n)
        t_stream = probe_ms(ix, d, pr)
        t_sorted = probe_ms(ix, d_sorted, pr)
        out[mode_name] = {"probe_stream_order_ms": t_stream, "probe_sorted_ms": t_sorted,
                          "gain_ms": t_stream - t_sorted,
                          "net_ms_with_prepass": t_sorted + out["prepass_ms"] - t_stream}
        del pr, ix
        torch.cuda.empty_cache()
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "source": "fallback"}


WORKLOADS = {
    "c2": {"name": "c2-city-300polys-mixture-points", "eps": 4.0},
    "c3": {"name": "c3-fine-40000polys-overlapping-mixture-points", "eps": 10.0},
    "c1": {"name": "c1-tiny-5polys-uniform-points", "eps": 10.0},
}


def workload(name: str, n: int, rank: int):
    from paper_1802_09488_gb300 import synth
    if name == "c3":
        polys = synth.c3_fine_polygons(40_000, seed=5)
        pts = synth.points_mixture(n, synth.BOX_CITY, seed=6 + 1000 * rank, dist_seed=5)
        train = synth.points_mixture(max(n // 100, 1000), synth.BOX_CITY, seed=7, dist_seed=5)
    elif name == "c1":
        polys = synth.voronoi_tiling(5, synth.BOX_C1, seed=1, vmin=8, vmax=64)
        pts = synth.points_uniform(n, synth.BOX_C1, seed=0 + 1000 * rank)
        train = synth.points_uniform(max(n // 100, 1000), synth.BOX_C1, seed=2)
    else:
        polys = synth.c2_city_polygons()
        pts = synth.points_mixture(n, synth.BOX_CITY, seed=3 + 1000 * rank, dist_seed=3)
        train = synth.points_mixture(max(n // 100, 1000), synth.BOX_CITY, seed=4, dist_seed=3)
    return polys, pts, train


def max_over_ranks(x: float, dist, device) -> float:
    """The largest of every rank's x (x itself with one process): the job's
    time is its slowest rank's."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def step_config(args, n: int, n_polys: int, eps: float, n_train: int, world: int) -> dict:
    """The workload both arms report: per-GPU point count, polygons, precision
    and training sample of the exact index."""
    return {"workload": f"{WORKLOADS[args.workload]['name']}-{n:.0e}".replace("+", ""), "n_points_per_gpu": n,
            "polygons": n_polys, "eps_m": eps, "exact_train_points": n_train,
            "step": "approx join + exact join of the same points",
            "l2": f"inputs (16 B x {n:.0e} = {16 * n / 1e9:.2f} GB) " + ("larger than L2, no flush" if 16 * n > 2e8
                                                                         else "smaller than L2: warm-cache figure"),
            "parallelism": f"replicas x{world}"}


def cpu_oracle_rate(polys, cells, ro, refs, pts, budget_s: float = 12.0):
    """Oracle points/s on the host cores for approx (sorted-vector probe of the
    logical covering) and exact (grid-prefiltered brute force), each on a
    bounded prefix sample of the same points sized to ~budget_s/2 seconds."""
    import oracle
    ps = oracle.PolySet(polys)
    cores = os.cpu_count() or 1
    out = {}
    for mode in ("approx", "exact"):
        m = 20000
        while True:
            t0 = time.perf_counter()
            if mode == "approx":
                oracle.join_approx_logical(cells, ro, refs, pts[:m])
            else:
                ps.join_exact(pts[:m])
            dt = time.perf_counter() - t0
            if dt > budget_s / 8 or m >= len(pts):
                break
            m = min(len(pts), int(m * max(2.0, (budget_s / 2) / max(dt, 1e-3))))
        out[mode] = {"points": m, "seconds": dt, "rate": m / dt}
    # one step = an approx join and an exact join of the same points
    t_step_per_point = 1.0 / out["approx"]["rate"] + 1.0 / out["exact"]["rate"]
    return {"value": 2.0 / t_step_per_point, "unit": "points/s", "cores": cores, "kind": "oracle",
            "sample": (f"approx: sorted-vector probe on the first {out['approx']['points']} points; exact: "
                       f"grid-prefiltered brute force on the first {out['exact']['points']} points; "
                       f"{cores} threads; rate = 2 / (1/approx + 1/exact)"),
            "per_mode_points_per_s": {k: v["rate"] for k, v in out.items()}}


def run_reference(args, rank: int):
    if rank != 0:
        return
    import paper_1802_09488_gb300 as agj
    n = min(args.n_points, 20_000_000)
    polys, pts, train = workload(args.workload, n, 0)
    eps = args.eps if args.eps is not None else WORKLOADS[args.workload]["eps"]
    ix = agj.Index(polys, agj.APPROX, eps, host_only=True)
    cells, ro, refs = ix.logical()
    import oracle
    ps = oracle.PolySet(polys)
    cores = os.cpu_count() or 1
    # size each step's sample to ~6 s of CPU work
    m = 200_000
    t0 = time.perf_counter()
    oracle.join_approx_logical(cells, ro, refs, pts[:m])
    ps.join_exact(pts[:m])
    dt = time.perf_counter() - t0
    m = int(min(n, max(50_000, m * 6.0 / max(dt, 1e-3))))
    times = []
    for it in range(args.warmup + args.steps):
        sl = pts[(it * 7919) % max(1, n - m):][:m]
        t0 = time.perf_counter()
        oracle.join_approx_logical(cells, ro, refs, sl)
        ps.join_exact(sl)
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = 2.0 * m * len(times) / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": step_config(args, args.n_points, len(polys), eps, max(args.n_points // 100, 1000), args.gpus),
            "cpu_baseline": {"value": value, "unit": "points/s", "cores": cores, "kind": "oracle",
                             "sample": f"{m} of the workload's points per step, drawn from the first {n} of its "
                                       f"stream (approx sorted-vector probe + exact brute force by the CPU oracle, "
                                       f"oracle/oracle.c), {cores} threads"},
            "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.only:
        import torch
        import paper_1802_09488_gb300 as agj
        torch.cuda.set_device(local)
        if args.only == "batched":
            tiling = tuple(int(x) for x in args.batched_tiling.split(",")) if args.batched_tiling else None
            c4p = tuple(int(x) for x in args.c4_polys.split(",")) if args.c4_polys else None
            print(json.dumps(batched_form(agj, torch, reps=args.form_reps, tiling=tiling, polys=c4p, m=args.c4_jobs)),
                  flush=True)
        elif args.only == "sort-study":
            print(json.dumps(sort_study(agj, torch, args.workload, args.n_points)), flush=True)
        else:
            print(json.dumps(served_form(agj)), flush=True)
        return
    import numpy as np
    import torch
    import paper_1802_09488_gb300 as agj

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    n = args.n_points
    polys, pts_np, train = workload(args.workload, n, rank)
    eps = args.eps if args.eps is not None else WORKLOADS[args.workload]["eps"]
    t0 = time.perf_counter()
    ia = agj.Index(polys, agj.APPROX, eps)
    ie = agj.Index(polys, agj.EXACT, 0.0, train=train)
    build_s = time.perf_counter() - t0
    d_pts = torch.from_numpy(pts_np).cuda()
    pa, pe = agj.Pairs(ia, n), agj.Pairs(ie, n)
    stream = torch.cuda.current_stream()

    for _ in range(max(args.warmup, 0)):
        agj.join(ia, d_pts, pa)
        agj.join(ie, d_pts, pe)
    nnz_a, nnz_e = pa.check(), pe.check()
    st_a = pa.status.cpu().numpy().view(np.uint64)
    st_e = pe.status.cpu().numpy().view(np.uint64)
    gathers_a = float(st_a[3]) / n          # trie entries read per point, approximate index
    gathers_e = float(st_e[3]) / n          # ... exact (trained) index
    cands_per_pt = float(st_e[2]) / n
    fallback_a, fallback_e = pa.fallbacks(), pe.fallbacks()
    refine_fb = pe.refine_fallbacks()

    barrier()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.4)

    def mk():
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)          # creates the handle
        return e

    step_ev = [(mk(), mk()) for _ in range(args.steps)]
    stage_ev = [([mk() for _ in range(4)], [mk() for _ in range(4)]) for _ in range(args.steps)]
    barrier()
    # A GPU hold ahead of the first timed event lets the host enqueue every
    # step before the device reaches them, so small joins are timed without
    # host launch gaps between their kernels (the host's per-call cost is in
    # `e2e`).  If the device still drains the queue first, the line says so.
    hold_ms = 1.0 + 0.5 * args.steps
    torch.cuda._sleep(int(hold_ms * 2.0e6))
    hold_end = mk()
    for k in range(args.steps):
        step_ev[k][0].record(stream)
        agj.join_timed(ia, d_pts, pa, stage_ev[k][0])
        agj.join_timed(ie, d_pts, pe, stage_ev[k][1])
        step_ev[k][1].record(stream)
    host_ahead = not hold_end.query()
    barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in step_ev]
    approx_ms = [ev[0][0].elapsed_time(ev[0][3]) for ev in stage_ev]
    exact_ms = [ev[1][0].elapsed_time(ev[1][3]) for ev in stage_ev]
    stages = {
        "approx": {"k_probe_approx": [ev[0][0].elapsed_time(ev[0][1]) for ev in stage_ev],
                   "k_scan_counts": [ev[0][1].elapsed_time(ev[0][2]) for ev in stage_ev],
                   "k_emit_approx": [ev[0][2].elapsed_time(ev[0][3]) for ev in stage_ev]},
        "exact": {"k_probe_exact": [ev[1][0].elapsed_time(ev[1][1]) for ev in stage_ev],
                  "refine (k_count + k_poly_scan + k_scatter + k_pip)": [ev[1][1].elapsed_time(ev[1][2]) for ev in stage_ev],
                  "csr (k_scan_counts + k_emit_exact)": [ev[1][2].elapsed_time(ev[1][3]) for ev in stage_ev]},
    }
    total_ms = step_ev[0][0].elapsed_time(step_ev[-1][1])
    total_ms = max_over_ranks(total_ms, dist, "cuda")
    # correctness of the timed runs
    assert pa.check() == nnz_a and pe.check() == nnz_e

    value = world * 2.0 * n * args.steps / (total_ms / 1000.0)
    peaks = measured_peaks()
    k_pts = nnz_a / n
    mean = statistics.mean

    def roof(kernel, bytes_per_pt, ms, note):
        achieved = bytes_per_pt * n / (ms / 1000.0) / 1e9
        tb = PROBE_DRAM_BYTES_PER_POINT.get(kernel) if args.workload == "c2" else None
        return {"kernel": kernel, "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": tb * n if tb else None,
                "traffic_unit": "DRAM bytes per launch (ncu capture of 16e6 points scaled by points)" if tb else None,
                "peak_source": peaks["source"], "algorithmic_bytes_per_point": bytes_per_pt, "ms_per_launch": ms,
                "note": note}

    t_pa = mean(stages["approx"]["k_probe_approx"])
    t_pe = mean(stages["exact"]["k_probe_exact"])
    r_pa = roof("k_probe_approx", 16 + 8 * gathers_a, t_pa,
                f"the method's bytes per point: 16 B point + 8 B per trie entry read (G = {gathers_a:.3f}, this "
                f"join's own counter); the stored entry is the pipeline's intermediate and not counted")
    r_pe = roof("k_probe_exact", 16 + 8 * gathers_e + 8 * cands_per_pt, t_pe,
                f"16 B point + 8 B per trie entry read (G = {gathers_e:.3f}, the exact index's own counter) + 8 B "
                f"per candidate queued, per point")
    roofline = r_pa if t_pa >= t_pe else r_pe
    join_roof = roof("approx join (probe + scan + emit)", 16 + 8 * gathers_a + 4 + 4 * k_pts, mean(approx_ms),
                     "the method's bytes: 16 B point + 8 B per trie entry + 4 B offset + 4 B per pair")

    def pct(v, q):
        s = sorted(v)
        return s[min(len(s) - 1, int(round(q / 100.0 * (len(s) - 1))))]

    result = {
        "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(step_config(args, n, len(polys), eps, len(train), world),
                       enqueue=(f"all {args.steps} steps enqueued behind a {hold_ms:.0f} ms GPU hold before the first "
                                f"timed event" if host_ahead else
                                "host enqueue fell behind the device: timings include host launch gaps")),
        "modes": {
            "approx": {"points_per_s": n / (statistics.mean(approx_ms) / 1000.0), "p50_ms": pct(approx_ms, 50),
                       "p99_ms": pct(approx_ms, 99), "nnz": nnz_a, "trie_entries_read_per_point": gathers_a,
                       "fp64_id_fallbacks": fallback_a},
            "exact": {"points_per_s": n / (statistics.mean(exact_ms) / 1000.0), "p50_ms": pct(exact_ms, 50),
                      "p99_ms": pct(exact_ms, 99), "nnz": nnz_e, "candidates_per_point": cands_per_pt,
                      "trie_entries_read_per_point": gathers_e,
                      "fp64_id_fallbacks": fallback_e, "fp64_refine_fallbacks": refine_fb},
        },
        "index": {"approx": ia.stats(), "exact": ie.stats(), "build_s": build_s},
        "stage_ms": {m: {k: mean(v) for k, v in d.items()} for m, d in stages.items()},
        "roofline": roofline,
        "roofline_other_probe": r_pe if roofline is r_pa else r_pa,
        "roofline_approx_join": join_roof,
        "clocks": clk,
        "gpu_launches": args.steps * (LAUNCHES_PER_STEP["approx"] + LAUNCHES_PER_STEP["exact"]),
    }

    extras = set(x for x in args.extras.split(",") if x)
    if "count" in extras:
        result["count"] = count_mode(agj, torch, ia, ie, d_pts, n, peaks, args.steps)
    if "onepass" in extras:
        result["one_pass_vs_three_kernels"] = one_pass(agj, torch, ia, d_pts)
    if "cellid" in extras:
        result["cell_id_kernel"] = cell_id_kernel(agj, torch, d_pts, n)
        torch.cuda.empty_cache()
    if "c1" in extras and rank == 0 and args.workload == "c2":
        result["c1_amortized_in_graph"] = c1_amortized(agj, torch, peaks)

    if not args.no_e2e:
        # end to end through the public host API: pinned host points in,
        # host CSR out, both modes per step
        h_pts = torch.from_numpy(pts_np).pin_memory()
        h_off = torch.empty(n + 1, dtype=torch.int32).pin_memory()
        h_ids_a = torch.empty(max(nnz_a, 1), dtype=torch.int32).pin_memory()
        h_ids_e = torch.empty(max(nnz_e, 1), dtype=torch.int32).pin_memory()
        staging = torch.empty((n, 2), dtype=torch.float64, device="cuda")
        ksteps = max(2, min(args.steps, 5))
        agj.join_host(ia, h_pts, pa, staging, h_off, h_ids_a)
        barrier()
        t0 = time.perf_counter()
        for _ in range(ksteps):
            agj.join_host(ia, h_pts, pa, staging, h_off, h_ids_a)
            agj.join_host(ie, h_pts, pe, staging, h_off, h_ids_e)
        barrier()
        dt = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
        e2e_val = world * 2.0 * n * ksteps / dt
        result["e2e"] = {"value": e2e_val, "unit": "points/s", "h2d_bytes_per_step": 2 * 16 * n,
                         "d2h_bytes_per_step": 2 * 4 * (n + 1) + 4 * (nnz_a + nnz_e) + 2 * 32, "steps": ksteps}
        del staging, h_pts

    if rank == 0 and not args.no_cpu_baseline:
        cells, ro, refs = ia.logical()
        result["cpu_baseline"] = cpu_oracle_rate(polys, cells, ro, refs, pts_np)

    if rank == 0 and not args.no_forms and args.workload == "c2":
        del pa, pe, d_pts
        torch.cuda.empty_cache()
        result["batched"] = batched_form(agj, torch, reps=args.form_reps)
        torch.cuda.empty_cache()
        result["served"] = served_form(agj)

    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result), flush=True)


if __name__ == "__main__":
    main()
