"""CPU oracle for the adaptive geospatial join probe (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The product path never does: it shares no code
with the oracle and must fail loudly when its own CUDA library is missing.

The arithmetic lives in ``oracle.c`` (plain C, FP64, no fused multiply-add);
this module only marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-pthread", "-std=c11"]


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (gcc, seconds)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        d, i64, u64, i32 = C.c_double, C.c_int64, C.c_uint64, C.c_int
        P = C.c_void_p
        sig = {
            "or_sincosd": (None, [d, P, P]),
            "or_point_valid": (i32, [d, d]),
            "or_face_uv": (i32, [d, d, P, P]),
            "or_uv_to_st": (d, [d]),
            "or_st_to_uv": (d, [d]),
            "or_id_from_face_ij": (u64, [i32, C.c_uint32, C.c_uint32]),
            "or_id_level": (i32, [u64]),
            "or_id_parent": (u64, [u64, i32]),
            "or_id_range_min": (u64, [u64]),
            "or_id_range_max": (u64, [u64]),
            "or_id_decode": (i32, [u64, P, P, P, P]),
            "or_cell_id": (u64, [d, d]),
            "or_cell_ids": (None, [P, i64, P]),
            "or_cell_uv_rect": (i32, [u64, P]),
            "or_uv_dist_m": (d, [i32, d, d, d, d]),
            "or_cell_diag_m": (d, [u64]),
            "or_ring_covers_uv": (i32, [P, i64, d, d]),
            "or_ring_relate_uv": (i32, [P, i64, d, d]),
            "or_rings_relate_uv": (i32, [P, P, i64, d, d]),
            "or_polyset_set_contains": (None, [P, i32]),
            "or_polyset_new": (P, [P, P, i64, i32]),
            "or_polyset_new_rings": (P, [P, P, P, i64, i32]),
            "or_polyset_free": (None, [P]),
            "or_polyset_face": (i32, [P, i64]),
            "or_polygon_covers": (i32, [P, i64, d, d]),
            "or_point_hits_brute": (i64, [P, d, d, P]),
            "or_join_exact_count": (u64, [P, P, i64, P, i32]),
            "or_join_exact_fill": (None, [P, P, i64, P, P, i32]),
            "or_join_approx_count": (u64, [P, i64, P, P, P, i64, P, i32]),
            "or_join_approx_fill": (None, [P, i64, P, P, P, i64, P, P, i32]),
            "or_logical_find": (i64, [P, i64, u64]),
            "or_dist_point_polygon_m": (d, [P, i64, d, d]),
            "or_check_covering": (None, [P, P, i64, P, P, d, d, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return C.c_void_p(a.ctypes.data)


def sincosd(d: float) -> tuple[float, float]:
    lib = _load()
    s, c = C.c_double(), C.c_double()
    lib.or_sincosd(float(d), C.byref(s), C.byref(c))
    return s.value, c.value


def face_uv(lat: float, lng: float) -> tuple[int, float, float]:
    lib = _load()
    u, v = C.c_double(), C.c_double()
    f = lib.or_face_uv(float(lat), float(lng), C.byref(u), C.byref(v))
    return f, u.value, v.value


def uv_to_st(u: float) -> float:
    return _load().or_uv_to_st(float(u))


def st_to_uv(s: float) -> float:
    return _load().or_st_to_uv(float(s))


def id_from_face_ij(face: int, i: int, j: int) -> int:
    return int(_load().or_id_from_face_ij(face, i, j))


def id_level(cid: int) -> int:
    return int(_load().or_id_level(cid))


def id_parent(cid: int, level: int) -> int:
    return int(_load().or_id_parent(cid, level))


def id_range(cid: int) -> tuple[int, int]:
    lib = _load()
    return int(lib.or_id_range_min(cid)), int(lib.or_id_range_max(cid))


def id_decode(cid: int) -> tuple[int, int, int, int]:
    lib = _load()
    f, l, i, j = C.c_int(), C.c_int(), C.c_uint32(), C.c_uint32()
    rc = lib.or_id_decode(cid, C.byref(f), C.byref(l), C.byref(i), C.byref(j))
    if rc != 0:
        raise ValueError("bad cell id")
    return f.value, l.value, i.value, j.value


def cell_id(lat: float, lng: float) -> int:
    return int(_load().or_cell_id(float(lat), float(lng)))


def cell_ids(points: np.ndarray) -> np.ndarray:
    pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 2)
    out = np.zeros(len(pts), dtype=np.uint64)
    _load().or_cell_ids(_ptr(pts), len(pts), _ptr(out))
    return out


def cell_uv_rect(cid: int) -> tuple[int, np.ndarray]:
    r = np.zeros(4, dtype=np.float64)
    f = _load().or_cell_uv_rect(cid, _ptr(r))
    return f, r


def cell_diag_m(cid: int) -> float:
    return float(_load().or_cell_diag_m(cid))


def uv_dist_m(face: int, u0: float, v0: float, u1: float, v1: float) -> float:
    return float(_load().or_uv_dist_m(face, u0, v0, u1, v1))


def ring_covers_uv(uv: np.ndarray, pu: float, pv: float) -> bool:
    a = np.ascontiguousarray(uv, dtype=np.float64).reshape(-1, 2)
    return bool(_load().or_ring_covers_uv(_ptr(a), len(a), float(pu), float(pv)))


def ring_relate_uv(uv: np.ndarray, pu: float, pv: float) -> int:
    """0 exterior, 1 on the boundary, 2 interior of the ring."""
    a = np.ascontiguousarray(uv, dtype=np.float64).reshape(-1, 2)
    return int(_load().or_ring_relate_uv(_ptr(a), len(a), float(pu), float(pv)))


def _rings(p):
    """A polygon as a list of (V,2) rings: an array is one ring, a list or
    tuple of arrays is the outer ring followed by its holes."""
    if isinstance(p, (list, tuple)):
        return [np.asarray(r, dtype=np.float64).reshape(-1, 2) for r in p]
    return [np.asarray(p, dtype=np.float64).reshape(-1, 2)]


def rings_relate_uv(rings, pu: float, pv: float) -> int:
    """Relation of a point to a polygon given as uv rings [outer, hole, ...]:
    0 exterior, 1 boundary (on an edge of any ring), 2 interior."""
    rs = [np.asarray(r, dtype=np.float64).reshape(-1, 2) for r in rings]
    uv = np.ascontiguousarray(np.concatenate(rs))
    off = np.zeros(len(rs) + 1, dtype=np.int64)
    for q, r in enumerate(rs):
        off[q + 1] = off[q] + len(r)
    return int(_load().or_rings_relate_uv(_ptr(uv), _ptr(off), len(rs), float(pu), float(pv)))


def flatten_polygons(polys) -> tuple[np.ndarray, np.ndarray]:
    """list of (V,2) (lat,lng) arrays -> (latlng (N,2) f64, offsets (P+1,) i64).
    Every polygon must be a single ring (see flatten_rings for holes)."""
    off = np.zeros(len(polys) + 1, dtype=np.int64)
    for k, p in enumerate(polys):
        off[k + 1] = off[k] + len(p)
    if len(polys):
        ll = np.ascontiguousarray(np.concatenate([np.asarray(p, dtype=np.float64).reshape(-1, 2) for p in polys]))
    else:
        ll = np.zeros((0, 2), dtype=np.float64)
    return ll, off


def flatten_rings(polys) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Polygons (each an array = one ring, or a list [outer, hole, ...]) ->
    (latlng (N,2), ring vertex offsets (R+1,), polygon ring offsets (P+1,))."""
    rings = [_rings(p) for p in polys]
    pr = np.zeros(len(polys) + 1, dtype=np.int64)
    for k, rs in enumerate(rings):
        pr[k + 1] = pr[k] + len(rs)
    flat = [r for rs in rings for r in rs]
    rv = np.zeros(len(flat) + 1, dtype=np.int64)
    for q, r in enumerate(flat):
        rv[q + 1] = rv[q] + len(r)
    ll = np.ascontiguousarray(np.concatenate(flat)) if flat else np.zeros((0, 2), dtype=np.float64)
    return ll, rv, pr


class PolySet:
    """Polygons prepared in face (u,v) with a uniform-grid prefilter."""

    def __init__(self, polys, grid_n: int = 64, contains: bool = False):
        """polys: each an (V,2) (lat,lng) ring or a list [outer, hole, ...] of
        rings.  contains: join by ST_Contains (boundary points excluded)
        instead of ST_Covers (= ST_Intersects for a point)."""
        self._lib = _load()
        self.latlng, self.ring_off, self.poly_ring_off = flatten_rings(polys)
        self.n = len(polys)
        self._h = self._lib.or_polyset_new_rings(_ptr(self.latlng), _ptr(self.ring_off), _ptr(self.poly_ring_off),
                                                 self.n, int(grid_n))
        self._lib.or_polyset_set_contains(self._h, 1 if contains else 0)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.or_polyset_free(h)
            self._h = None

    def face(self, k: int) -> int:
        return int(self._lib.or_polyset_face(self._h, k))

    def covers(self, k: int, lat: float, lng: float) -> bool:
        return bool(self._lib.or_polygon_covers(self._h, k, float(lat), float(lng)))

    def hits_brute(self, lat: float, lng: float) -> list[int]:
        out = np.zeros(max(self.n, 1), dtype=np.uint32)
        m = self._lib.or_point_hits_brute(self._h, float(lat), float(lng), _ptr(out))
        return [int(x) for x in out[:m]]

    def dist_m(self, k: int, lat: float, lng: float) -> float:
        return float(self._lib.or_dist_point_polygon_m(self._h, k, float(lat), float(lng)))

    def join_exact(self, points: np.ndarray, threads: int = 0) -> tuple[np.ndarray, np.ndarray]:
        """Exact join by brute force (grid-prefiltered). CSR (offsets u64, ids u32)."""
        pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 2)
        n = len(pts)
        offs = np.zeros(n + 1, dtype=np.uint64)
        nnz = int(self._lib.or_join_exact_count(self._h, _ptr(pts), n, _ptr(offs), threads))
        ids = np.zeros(max(nnz, 1), dtype=np.uint32)
        self._lib.or_join_exact_fill(self._h, _ptr(pts), n, _ptr(offs), _ptr(ids), threads)
        return offs, ids[:nnz]

    def count_exact(self, points: np.ndarray, threads: int = 0) -> np.ndarray:
        """Aggregation query of §V (count(*) group by polygon) for the exact
        join: how often each polygon occurs in the brute-force CSR."""
        _, ids = self.join_exact(points, threads)
        return np.bincount(ids, minlength=self.n).astype(np.uint64)

    def check_covering(self, cells, ref_off, refs, eps_m: float = 0.0, cand_margin: float = 1e-11) -> dict:
        cells = np.ascontiguousarray(cells, dtype=np.uint64)
        ref_off = np.ascontiguousarray(ref_off, dtype=np.uint64)
        refs = np.ascontiguousarray(refs, dtype=np.uint32)
        rep = np.zeros(5, dtype=np.int64)
        self._lib.or_check_covering(self._h, _ptr(cells), len(cells), _ptr(ref_off), _ptr(refs),
                                    float(eps_m), float(cand_margin), _ptr(rep))
        keys = ["overlapping_cells", "true_ref_not_inside", "cand_ref_misses", "cand_diag_ge_eps", "bad_ref"]
        return dict(zip(keys, (int(x) for x in rep)))


def join_approx_logical(cells, ref_off, refs, points: np.ndarray, threads: int = 0):
    """Approximate join read off a logical covering by sorted-vector binary
    search: every reference of the unique cell holding the point's id."""
    lib = _load()
    cells = np.ascontiguousarray(cells, dtype=np.uint64)
    ref_off = np.ascontiguousarray(ref_off, dtype=np.uint64)
    refs = np.ascontiguousarray(refs, dtype=np.uint32)
    pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 2)
    n = len(pts)
    offs = np.zeros(n + 1, dtype=np.uint64)
    nnz = int(lib.or_join_approx_count(_ptr(cells), len(cells), _ptr(ref_off), _ptr(refs), _ptr(pts), n,
                                       _ptr(offs), threads))
    ids = np.zeros(max(nnz, 1), dtype=np.uint32)
    lib.or_join_approx_fill(_ptr(cells), len(cells), _ptr(ref_off), _ptr(refs), _ptr(pts), n, _ptr(offs),
                            _ptr(ids), threads)
    return offs, ids[:nnz]


def logical_find(cells, cid: int) -> int:
    cells = np.ascontiguousarray(cells, dtype=np.uint64)
    return int(_load().or_logical_find(_ptr(cells), len(cells), cid))


def count_approx_logical(cells, ref_off, refs, points: np.ndarray, n_polys: int, threads: int = 0) -> np.ndarray:
    """Aggregation query (§V) for the approximate join read off a logical
    covering: how often each polygon occurs in that CSR."""
    _, ids = join_approx_logical(cells, ref_off, refs, points, threads)
    return np.bincount(ids, minlength=n_polys).astype(np.uint64)
