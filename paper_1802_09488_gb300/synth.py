"""Seeded synthetic workloads shaped like the paper's evaluation (§V).

The paper joins 1.23 B NYC taxi points with NYC boroughs (5 polygons),
neighbourhoods (289) and census blocks (39 184).  Those datasets are not
available here, so these generators stand in for them:

* polygon sets are Voronoi tessellations of a lat/lng box, whose shared edges
  are subdivided and jittered once and reused by both neighbours (so the
  polygons tile the box, are concave and stay simple);
* points are uniform over the box, or an 80 % / 20 % mixture of isotropic
  Gaussian clusters and uniform noise (taxi pick-ups cluster).

This module holds none of the join's arithmetic (no cell ids, no PIP); it
only draws coordinates, and both the CUDA path and the CPU oracle consume
its output.  All boxes are centred on a mid-latitude site (40.70 N,
73.95 W); metres map to degrees with 111 195 m per degree of latitude and
that times cos(latitude) per degree of longitude.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

LAT0 = 40.70
LNG0 = -73.95
M_PER_DEG = 111195.0


@dataclass
class Box:
    we_km: float            # east-west extent
    sn_km: float            # south-north extent
    lat0: float = LAT0
    lng0: float = LNG0

    @property
    def half_w(self) -> float:
        return self.we_km * 500.0

    @property
    def half_h(self) -> float:
        return self.sn_km * 500.0

    def to_latlng(self, xy: np.ndarray) -> np.ndarray:
        """local metres (x east, y north) -> (lat, lng) degrees."""
        xy = np.asarray(xy, dtype=np.float64)
        lat = self.lat0 + xy[..., 1] / M_PER_DEG
        lng = self.lng0 + xy[..., 0] / (M_PER_DEG * math.cos(math.radians(self.lat0)))
        return np.stack([lat, lng], axis=-1)

    def latlng_bounds(self) -> tuple[float, float, float, float]:
        c = self.to_latlng(np.array([[-self.half_w, -self.half_h], [self.half_w, self.half_h]]))
        return float(c[0, 0]), float(c[1, 0]), float(c[0, 1]), float(c[1, 1])


BOX_C1 = Box(40.0, 40.0)
BOX_CITY = Box(45.0, 50.0)


# ---------------------------------------------------------------------------
# points
# ---------------------------------------------------------------------------

def points_uniform(n: int, box: Box, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    x = rng.uniform(-box.half_w, box.half_w, n)
    y = rng.uniform(-box.half_h, box.half_h, n)
    return np.ascontiguousarray(box.to_latlng(np.stack([x, y], axis=-1)))


def mixture_params(box: Box, dist_seed: int, n_comp: int = 32,
                   sigma_km: tuple[float, float] = (0.5, 3.0)):
    """Centres uniform in the box, sigma ~ U[0.5, 3] km, equal weights."""
    rng = np.random.default_rng([dist_seed, 0])
    cx = rng.uniform(-box.half_w, box.half_w, n_comp)
    cy = rng.uniform(-box.half_h, box.half_h, n_comp)
    sig = rng.uniform(sigma_km[0] * 1e3, sigma_km[1] * 1e3, n_comp)
    return cx, cy, sig


def mixture_xy(n: int, box: Box, params, rng: np.random.Generator, frac_uniform: float = 0.2) -> np.ndarray:
    """80 % from the Gaussian clusters in `params` + 20 % uniform over the
    box; out-of-box samples are redrawn."""
    cx, cy, sig = params
    n_comp = len(cx)
    out = np.empty((n, 2), dtype=np.float64)
    todo = np.arange(n)
    while len(todo):
        m = len(todo)
        uni = rng.random(m) < frac_uniform
        comp = rng.integers(0, n_comp, m)
        g = rng.standard_normal((m, 2))
        x = np.where(uni, rng.uniform(-box.half_w, box.half_w, m), cx[comp] + sig[comp] * g[:, 0])
        y = np.where(uni, rng.uniform(-box.half_h, box.half_h, m), cy[comp] + sig[comp] * g[:, 1])
        ok = (np.abs(x) <= box.half_w) & (np.abs(y) <= box.half_h)
        out[todo[ok], 0] = x[ok]
        out[todo[ok], 1] = y[ok]
        todo = todo[~ok]
    return out


def points_mixture(n: int, box: Box, seed: int, dist_seed: int | None = None) -> np.ndarray:
    """n points of the mixture whose clusters are fixed by dist_seed (default:
    seed), drawn with seed."""
    params = mixture_params(box, seed if dist_seed is None else dist_seed)
    rng = np.random.default_rng([seed, 1])
    return np.ascontiguousarray(box.to_latlng(mixture_xy(n, box, params, rng)))


# ---------------------------------------------------------------------------
# polygons: Voronoi tiling with shared jittered edges
# ---------------------------------------------------------------------------

def _segments_cross(p: np.ndarray) -> bool:
    """True if the closed ring p (V,2) has two non-adjacent edges that meet."""
    n = len(p)
    a = p
    b = np.roll(p, -1, axis=0)
    i, j = np.triu_indices(n, k=2)
    keep = ~((i == 0) & (j == n - 1))
    i, j = i[keep], j[keep]
    if len(i) == 0:
        return False

    def orient(p0, p1, p2):
        return (p1[:, 0] - p0[:, 0]) * (p2[:, 1] - p0[:, 1]) - (p1[:, 1] - p0[:, 1]) * (p2[:, 0] - p0[:, 0])

    d1 = orient(a[i], b[i], a[j])
    d2 = orient(a[i], b[i], b[j])
    d3 = orient(a[j], b[j], a[i])
    d4 = orient(a[j], b[j], b[i])
    proper = (d1 * d2 < 0) & (d3 * d4 < 0)

    def on_seg(p0, p1, q):
        return ((np.minimum(p0[:, 0], p1[:, 0]) <= q[:, 0]) & (q[:, 0] <= np.maximum(p0[:, 0], p1[:, 0])) &
                (np.minimum(p0[:, 1], p1[:, 1]) <= q[:, 1]) & (q[:, 1] <= np.maximum(p0[:, 1], p1[:, 1])))

    touch = (((d1 == 0) & on_seg(a[i], b[i], a[j])) | ((d2 == 0) & on_seg(a[i], b[i], b[j])) |
             ((d3 == 0) & on_seg(a[j], b[j], a[i])) | ((d4 == 0) & on_seg(a[j], b[j], b[i])))
    return bool(proper.any() or touch.any())


def voronoi_tiling(n_polys: int, box: Box, seed: int, vmin: int, vmax: int,
                   seeds_xy: np.ndarray | None = None, jitter: float = 0.2) -> list[np.ndarray]:
    """n_polys simple polygons tiling the box, vmin..vmax vertices each,
    returned as (V,2) arrays of (lat, lng) degrees."""
    from scipy.spatial import Voronoi

    rng = np.random.default_rng(seed)
    W, H = box.half_w, box.half_h
    if seeds_xy is None:
        seeds_xy = np.stack([rng.uniform(-W, W, n_polys), rng.uniform(-H, H, n_polys)], axis=-1)
    s = np.asarray(seeds_xy, dtype=np.float64)
    n = len(s)
    mirrors = [s * [1, 1]]
    mirrors.append(np.stack([2 * W - s[:, 0], s[:, 1]], -1))
    mirrors.append(np.stack([-2 * W - s[:, 0], s[:, 1]], -1))
    mirrors.append(np.stack([s[:, 0], 2 * H - s[:, 1]], -1))
    mirrors.append(np.stack([s[:, 0], -2 * H - s[:, 1]], -1))
    vor = Voronoi(np.concatenate(mirrors))
    verts = vor.vertices.copy()
    # clamp numerically-on-the-boundary vertices onto it exactly
    for ax, lim in ((0, W), (1, H)):
        c = verts[:, ax]
        c[np.abs(c - lim) < 1e-6] = lim
        c[np.abs(c + lim) < 1e-6] = -lim

    ridge_of = {}
    for (pa, pb), rv in zip(vor.ridge_points, vor.ridge_vertices):
        if pa >= n and pb >= n:
            continue
        if -1 in rv:
            continue
        key = (min(rv), max(rv))
        ridge_of[key] = (pa < n and pb < n)

    rings = []
    for k in range(n):
        reg = vor.regions[vor.point_region[k]]
        idx = np.array(reg)
        ang = np.arctan2(verts[idx, 1] - s[k, 1], verts[idx, 0] - s[k, 0])
        idx = idx[np.argsort(ang)]
        rings.append([(int(idx[t]), int(idx[(t + 1) % len(idx)])) for t in range(len(idx))])

    # per-edge subdivision counts hitting each polygon's vertex range
    edges = {}
    for ring in rings:
        for a, b in ring:
            key = (min(a, b), max(a, b))
            edges.setdefault(key, 0)
    targets = np.exp(rng.uniform(math.log(vmin), math.log(vmax), n))
    for k, ring in enumerate(rings):
        per = max(targets[k] / len(ring), 1.0)
        for a, b in ring:
            key = (min(a, b), max(a, b))
            want = max(int(round(per)) - 1, 0)
            cur = edges[key]
            edges[key] = want if cur == 0 else min(cur, want)

    def total(k):
        return sum(edges[(min(a, b), max(a, b))] + 1 for a, b in rings[k])

    users = {}
    for k, ring in enumerate(rings):
        for a, b in ring:
            users.setdefault((min(a, b), max(a, b)), []).append(k)
    for _ in range(200):
        bad = False
        for k in range(n):
            t = total(k)
            if t < vmin:
                bad = True
                for a, b in sorted(rings[k], key=lambda e: edges[(min(e), max(e))]):
                    key = (min(a, b), max(a, b))
                    if all(total(o) < vmax for o in users[key] if o != k):
                        edges[key] += min(vmin - t, max(1, (vmin - t) // len(rings[k]) + 1))
                        break
            elif t > vmax:
                bad = True
                for a, b in sorted(rings[k], key=lambda e: -edges[(min(e), max(e))]):
                    key = (min(a, b), max(a, b))
                    if edges[key] > 0 and all(total(o) > vmin for o in users[key] if o != k):
                        edges[key] -= min(edges[key], t - vmax)
                        break
        if not bad:
            break

    amp = {key: jitter for key in edges}
    sub_rng = np.random.default_rng(seed + 7919)
    noise = {key: sub_rng.uniform(-1.0, 1.0, edges[key]) for key in edges}

    def edge_points(key):
        a, b = key
        kk = edges[key]
        pa, pb = verts[a], verts[b]
        if kk == 0:
            return np.zeros((0, 2))
        t = np.arange(1, kk + 1) / (kk + 1)
        base = pa[None, :] + t[:, None] * (pb - pa)[None, :]
        if not ridge_of.get(key, False):     # box boundary: no jitter
            return base
        d = pb - pa
        L = float(np.hypot(d[0], d[1]))
        if L == 0.0:
            return base
        nrm = np.array([-d[1], d[0]]) / L
        seg = L / (kk + 1)
        return base + (noise[key] * amp[key] * seg)[:, None] * nrm[None, :]

    def ring_xy(k):
        pts = []
        for a, b in rings[k]:
            key = (min(a, b), max(a, b))
            ep = edge_points(key)
            if a > b:
                ep = ep[::-1]
            pts.append(verts[a][None, :])
            pts.append(ep)
        return np.concatenate(pts)

    out = [None] * n
    todo = list(range(n))
    converged = False
    for _ in range(12):
        nxt = set()
        for k in todo:
            r = ring_xy(k)
            if _segments_cross(r):
                for a, b in rings[k]:
                    key = (min(a, b), max(a, b))
                    amp[key] *= 0.5
                    nxt.update(users[key])
            else:
                out[k] = r
        if not nxt:
            converged = True
            break
        todo = sorted(nxt)
    # Every polygon touched by an amplitude change is re-checked above, so on
    # convergence out[k] is ring_xy(k) at the final amplitudes and simple;
    # otherwise re-check them all.
    if not converged:
        for k in range(n):
            r = ring_xy(k)
            if _segments_cross(r):
                raise RuntimeError(f"polygon {k} is not simple after jitter reduction")
            out[k] = r
    return [np.ascontiguousarray(box.to_latlng(r)) for r in out]


# ---------------------------------------------------------------------------
# the five workloads
# ---------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    polygons: list
    points: np.ndarray
    eps_m: float
    train: np.ndarray | None = None


def c1_tiny(n_points: int = 100_000) -> Workload:
    """5 concave polygons (8-64 vertices) tiling a 40 km box; uniform
    points (seed 0); eps = 10 m."""
    polys = voronoi_tiling(5, BOX_C1, seed=1, vmin=8, vmax=64)
    pts = points_uniform(n_points, BOX_C1, seed=0)
    return Workload("c1-tiny-5polys", polys, pts, 10.0)


def c2_city_polygons() -> list:
    return voronoi_tiling(300, BOX_CITY, seed=2, vmin=20, vmax=400)


def c2_city(n_points: int = 100_000_000, n_train: int | None = None) -> Workload:
    """300 Voronoi polygons (20-400 vertices) over a 45x50 km box; mixture
    points (seed 3); eps = 4 m; exact index trained on a 1 % sample (seed 4)."""
    polys = c2_city_polygons()
    pts = points_mixture(n_points, BOX_CITY, seed=3)
    if n_train is None:
        n_train = max(n_points // 100, 1000)
    train = points_mixture(n_train, BOX_CITY, seed=4, dist_seed=3)
    return Workload("c2-city-300polys", polys, pts, 4.0, train)


def scale_about_centroid(polys: list, seed: int, lo: float, hi: float) -> list:
    """Each polygon scaled about its vertex centroid (in local metres) by a
    factor drawn from U[lo, hi]: a homothety keeps a simple ring simple, and
    factors above 1 make neighbours of a tiling overlap, below 1 open gaps."""
    rng = np.random.default_rng([seed, 3])
    f = rng.uniform(lo, hi, len(polys))
    out = []
    for k, p in enumerate(polys):
        c = p.mean(axis=0)
        out.append(np.ascontiguousarray(c + f[k] * (p - c)))
    return out


def c3_fine_polygons(n_polys: int = 40_000, seed: int = 5) -> list:
    """n_polys small polygons (4-60 vertices) from a Voronoi tessellation of
    the city box over a density-skewed seed field (the mixture), each scaled
    about its centroid by U[0.85, 1.25] so that a point hits 0-3 polygons."""
    box = BOX_CITY
    rng = np.random.default_rng([seed, 2])
    seeds = mixture_xy(n_polys, box, mixture_params(box, seed), rng)
    polys = voronoi_tiling(n_polys, box, seed=seed, vmin=4, vmax=60, seeds_xy=seeds)
    return scale_about_centroid(polys, seed, 0.85, 1.25)


def c3_fine(n_points: int = 100_000_000, n_polys: int = 40_000, n_train: int | None = None) -> Workload:
    """Fine polygons (c3_fine_polygons) with mixture points (seed 6, the
    polygon field's clusters); eps = 1 m (also run at 10 m); exact index
    trained on a 1 % sample (seed 7)."""
    polys = c3_fine_polygons(n_polys)
    pts = points_mixture(n_points, BOX_CITY, seed=6, dist_seed=5)
    if n_train is None:
        n_train = max(n_points // 100, 1000)
    train = points_mixture(n_train, BOX_CITY, seed=7, dist_seed=5)
    return Workload(f"c3-fine-{n_polys}polys", polys, pts, 1.0, train)


@dataclass
class Job:
    """One (polygon set, point batch) job of the batched form."""
    polygons: list
    points: np.ndarray
    exact: bool
    eps_m: float
    train: np.ndarray | None


def batched_jobs(m: int = 64, seed: int = 11, polys: tuple[int, int] = (5, 40_000),
                 points: tuple[int, int] = (1_000, 10_000_000), exact_every: int = 2) -> list:
    """m jobs with polygon counts and point counts drawn log-uniform from the
    given ranges (per-job seeds).  A set of at most 16 polygons is built as
    the tiny workload (8-64 vertices, 40 km box, uniform points), one of at
    most 1000 as the city one (20-400 vertices, mixture points), a larger one
    as the fine one (4-60 vertices, skewed seed field, overlaps).  Every
    exact_every-th job is exact (trained on 1 % of its own points' field),
    the others approximate with eps 4 m."""
    rng = np.random.default_rng([seed, 4])
    n_polys = np.exp(rng.uniform(math.log(polys[0]), math.log(polys[1]), m)).round().astype(int)
    n_pts = np.exp(rng.uniform(math.log(points[0]), math.log(points[1]), m)).round().astype(int)
    jobs = []
    for j in range(m):
        s = 1000 * seed + j
        k = int(n_polys[j])
        if k <= 16:
            box = BOX_C1
            pl = voronoi_tiling(k, box, seed=s, vmin=8, vmax=64)
            pts = points_uniform(int(n_pts[j]), box, seed=s + 1)
            tr = points_uniform(max(int(n_pts[j]) // 100, 100), box, seed=s + 2)
        elif k <= 1000:
            box = BOX_CITY
            pl = voronoi_tiling(k, box, seed=s, vmin=20, vmax=400)
            pts = points_mixture(int(n_pts[j]), box, seed=s + 1)
            tr = points_mixture(max(int(n_pts[j]) // 100, 100), box, seed=s + 2, dist_seed=s + 1)
        else:
            box = BOX_CITY
            pl = c3_fine_polygons(k, seed=s)
            pts = points_mixture(int(n_pts[j]), box, seed=s + 1, dist_seed=s)
            tr = points_mixture(max(int(n_pts[j]) // 100, 100), box, seed=s + 2, dist_seed=s)
        exact = exact_every > 0 and j % exact_every == exact_every - 1
        jobs.append(Job(pl, pts, exact, 4.0, tr if exact else None))
    return jobs


# ---------------------------------------------------------------------------
# polygons with holes
# ---------------------------------------------------------------------------

def _seg_dist(p: np.ndarray, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Planar distances from point p (2,) to the segments a[i]-b[i]."""
    d = b - a
    t = np.clip(((p - a) * d).sum(-1) / np.maximum((d * d).sum(-1), 1e-300), 0.0, 1.0)
    q = a + t[:, None] * d
    return np.hypot(*(p - q).T)


def _inside(p: np.ndarray, ring: np.ndarray) -> bool:
    """Planar even-odd test (generator use only: it picks hole centres well
    away from every edge)."""
    a, b = ring, np.roll(ring, -1, axis=0)
    cross = ((a[:, 1] > p[1]) != (b[:, 1] > p[1]))
    with np.errstate(divide="ignore", invalid="ignore"):
        x = a[:, 0] + (p[1] - a[:, 1]) * (b[:, 0] - a[:, 0]) / (b[:, 1] - a[:, 1])
    return bool(np.count_nonzero(cross & (x > p[0])) % 2)


def with_holes(polys: list, seed: int, frac: float = 0.35, max_holes: int = 3, vmin: int = 6,
               vmax: int = 16) -> list:
    """A copy of polys where a fraction of the polygons get 1..max_holes holes:
    jittered regular rings of vmin..vmax vertices, each centred on a random
    interior point and sized to a third of its clearance from the outer ring
    and the holes placed before it, listed in the opposite orientation.  A
    polygon with holes is returned as [outer, hole, ...]; the others as
    before.  Planar geometry in local metres (the polygons are a few km
    across, so the thirds leave ample room for the curvature of the
    geodesic edges)."""
    rng = np.random.default_rng(seed)
    out = []
    for P in polys:
        P = np.asarray(P, dtype=np.float64)
        if rng.random() >= frac:
            out.append(P)
            continue
        lat0 = float(P[:, 0].mean())
        kx = 111195.0 * np.cos(np.radians(lat0))
        xy = np.stack([(P[:, 1] - P[:, 1].mean()) * kx, (P[:, 0] - lat0) * 111195.0], -1)
        a, b = xy, np.roll(xy, -1, axis=0)
        holes_xy = []
        want = int(rng.integers(1, max_holes + 1))
        lo, hi = xy.min(0), xy.max(0)
        for _ in range(200):
            if len(holes_xy) == want:
                break
            c = rng.uniform(lo, hi)
            if not _inside(c, xy):
                continue
            clear = float(_seg_dist(c, a, b).min())
            for h in holes_xy:
                clear = min(clear, float(_seg_dist(c, h, np.roll(h, -1, axis=0)).min()))
                if _inside(c, h):
                    clear = 0.0
            r = clear / 3.0
            if r < 20.0:          # metres: too tight a spot
                continue
            m = int(rng.integers(vmin, vmax + 1))
            ang = np.linspace(0.0, 2 * np.pi, m, endpoint=False) + rng.uniform(0, 2 * np.pi)
            rad = r * rng.uniform(0.7, 1.0, m)
            ring = c + np.stack([rad * np.cos(ang), rad * np.sin(ang)], -1)
            holes_xy.append(ring[::-1])
        if not holes_xy:
            out.append(P)
            continue
        to_ll = lambda q: np.stack([q[:, 1] / 111195.0 + lat0, q[:, 0] / kx + P[:, 1].mean()], -1)
        out.append([P] + [np.ascontiguousarray(to_ll(h)) for h in holes_xy])
    return out


def c2_city_holes_polygons() -> list:
    """The city polygons, a third of them with one to three holes (seed 8)."""
    return with_holes(c2_city_polygons(), seed=8)


# ---------------------------------------------------------------------------
# polygons across cube faces
# ---------------------------------------------------------------------------

# A 40 km box centred on the cube edge between faces 0 (+x) and 1 (+y) at
# the equator, and one on the corner of faces 0, 1 and 2 (lat 35.26, lng 45).
BOX_EDGE = Box(40.0, 40.0, lat0=0.0, lng0=45.0)
BOX_CORNER = Box(40.0, 40.0, lat0=35.2643896827547, lng0=45.0)


def crossface_tiling(box: Box, n_polys: int = 40, seed: int = 12) -> list:
    """A Voronoi tiling (8-64 vertices per polygon) of a box that straddles
    cube faces: the polygons across the face boundaries span two or three
    faces."""
    return voronoi_tiling(n_polys, box, seed=seed, vmin=8, vmax=64)
