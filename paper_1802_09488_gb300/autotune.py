"""Tiling autotuner of the batched form.

A batched plan (agj_batch_create) is tiled by two options: the points each
lane of a warp tile probes (1, 2 or 4: more points per lane put more trie
gathers in flight per warp, at the cost of registers) and the probe grid
(one warp per tile, or a persistent grid of 1-8 CTAs per SM).  Which is
fastest depends on the trie sizes (how far the gathers go: L1, L2 or HBM),
on the batch sizes (how much tail a grid leaves) and on the exact share
(refine work).  `tune` times each candidate on the caller's own jobs with
CUDA events and caches the winner in a JSON file, keyed by coarse classes of
those three quantities, so later plans of the same class skip the sweep.

The cache file is `$AGJ_AUTOTUNE_CACHE`, else `_build/autotune.json` beside
the native library.
"""
from __future__ import annotations

import json
import math
import os
import threading

CANDIDATES = [(1, 0), (2, 0), (4, 0), (2, 3), (4, 3), (2, 5), (4, 5)]
_lock = threading.Lock()


def cache_path() -> str:
    p = os.environ.get("AGJ_AUTOTUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def key(indexes, ns) -> str:
    """Class of a job set: log2 of the total points, log4 of the total trie
    nodes, the exact share of the points in tenths, log2 of the job count."""
    pts = sum(int(n) for n in ns)
    nodes = sum(ix.stats()["n_nodes"] for ix in {id(ix): ix for ix in indexes}.values())
    exact = sum(int(n) for ix, n in zip(indexes, ns) if ix.stats()["mode"] == 1)
    share = round(10 * exact / pts) if pts else 0
    return f"p{int(math.log2(max(pts, 1)))}-n{int(math.log(max(nodes, 1), 4))}-e{share}-m{int(math.log2(max(len(ns), 1)))}"


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(d: dict):
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def time_plan(plan, points, pairs, reps: int = 5, stream=None) -> float:
    """Median milliseconds of one run of a plan (CUDA events on its stream)."""
    import torch
    s = stream or torch.cuda.current_stream()
    for _ in range(2):
        plan.run(points, pairs, stream=s)
    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s)
        plan.run(points, pairs, stream=s)
        b.record(s)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    ts.sort()
    return ts[len(ts) // 2]


def tune(indexes, points, candidates=None, reps: int = 5, use_cache: bool = True) -> dict:
    """Best (points_per_lane, ctas_per_sm) for these jobs: from the cache,
    else by timing every candidate plan on them.  Returns
    {"points_per_lane", "ctas_per_sm", "ms", "key", "cached", "sweep"}."""
    from .native import Batch
    ns = [int(p.shape[0]) for p in points]
    k = key(indexes, ns)
    with _lock:
        cache = _load() if use_cache else {}
    if k in cache:
        c = cache[k]
        return {"points_per_lane": c["points_per_lane"], "ctas_per_sm": c["ctas_per_sm"], "ms": c.get("ms"),
                "key": k, "cached": True, "sweep": None}
    sweep = []
    best = None
    for ppt, ctas in (candidates or CANDIDATES):
        plan = Batch(indexes, ns, points_per_lane=ppt, ctas_per_sm=ctas)
        pairs = plan.pairs()
        ms = time_plan(plan, points, pairs, reps)
        sweep.append({"points_per_lane": ppt, "ctas_per_sm": ctas, "ms": ms})
        if best is None or ms < best[2]:
            best = (ppt, ctas, ms)
        plan.close()
        del pairs
    if use_cache:
        with _lock:
            cache = _load()
            cache[k] = {"points_per_lane": best[0], "ctas_per_sm": best[1], "ms": best[2]}
            _store(cache)
    return {"points_per_lane": best[0], "ctas_per_sm": best[1], "ms": best[2], "key": k, "cached": False,
            "sweep": sweep}
