"""ctypes binding of libagj.so (include/agj.h).

Argument marshalling only: every step of the join runs in the library's
CUDA kernels.  PyTorch supplies device memory and streams.  There is no
fallback: if the native library cannot be built or loaded, importing the
binding raises.
"""
from __future__ import annotations

import ctypes as C
import threading

import numpy as np

from . import build as _build

AGJ_OK, AGJ_EINVAL, AGJ_EUNSUPPORTED, AGJ_EBUDGET, AGJ_ENOMEM, AGJ_ECUDA, AGJ_ETIMEOUT, AGJ_EBUSY, \
    AGJ_ECAPACITY, AGJ_EDEVICE = range(10)
APPROX, EXACT, AUTO = 0, 1, 2
COVERS, INTERSECTS, CONTAINS = 0, 1, 2          # join predicates of the exact join (agj_predicate)


class AgjError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = _lib.agj_strerror(status).decode() if _lib else str(status)
        extra = ""
        if _lib is not None:
            e = _lib.agj_last_error()
            extra = e.decode() if e else ""
        super().__init__(f"{what}: {msg} ({status}) {extra}".strip())


class Polygon(C.Structure):
    _fields_ = [("n_vertices", C.c_uint32), ("n_rings", C.c_uint32), ("latlng", C.c_void_p),
                ("ring_ends", C.c_void_p)]


def _polygon_rings(p):
    """A polygon as its rings: an (V,2) array is one ring; a list or tuple of
    arrays is the outer ring followed by its holes."""
    if isinstance(p, (list, tuple)):
        return [np.ascontiguousarray(r, dtype=np.float64).reshape(-1, 2) for r in p]
    return [np.ascontiguousarray(p, dtype=np.float64).reshape(-1, 2)]


class BuildOpts(C.Structure):
    _fields_ = [("max_cover_cells", C.c_uint32), ("max_cover_level", C.c_uint32),
                ("max_interior_cells", C.c_uint32), ("max_interior_level", C.c_uint32),
                ("memory_budget_bytes", C.c_uint64), ("train_latlng", C.c_void_p), ("n_train", C.c_uint64),
                ("max_train_level", C.c_uint32), ("n_threads", C.c_uint32), ("host_only", C.c_uint32),
                ("no_fast_ids", C.c_uint32), ("no_pip_bands", C.c_uint32), ("predicate", C.c_uint32)]


class Stats(C.Structure):
    _fields_ = [("mode", C.c_uint32), ("n_polys", C.c_uint32), ("n_cells", C.c_uint64),
                ("n_cand_cells", C.c_uint64), ("n_nodes", C.c_uint64), ("n_lut_words", C.c_uint64),
                ("device_bytes", C.c_uint64), ("max_refs", C.c_uint32), ("max_cand_refs", C.c_uint32),
                ("max_depth", C.c_uint32), ("max_level", C.c_uint32), ("build_seconds", C.c_double),
                ("fast_ids", C.c_uint32), ("predicate", C.c_uint32), ("fast_err_cells", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class PairsC(C.Structure):
    _fields_ = [("offsets", C.c_void_p), ("ids", C.c_void_p), ("ids_capacity", C.c_uint64),
                ("scratch", C.c_void_p), ("scratch_bytes", C.c_uint64), ("status", C.c_void_p)]


class Requirements(C.Structure):
    _fields_ = [("ids_capacity", C.c_uint64), ("scratch_bytes", C.c_uint64)]


class ServerOpts(C.Structure):
    _fields_ = [("n_slots", C.c_uint32), ("max_step_requests", C.c_uint32), ("max_step_points", C.c_uint64),
                ("hbm_budget_bytes", C.c_uint64), ("max_pending", C.c_uint64), ("points_per_lane", C.c_uint32),
                ("ctas_per_sm", C.c_uint32), ("flags", C.c_uint32), ("max_refs", C.c_uint32),
                ("hbm_reserve_bytes", C.c_uint64)]


class RequestResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("reserved", C.c_uint32), ("nnz", C.c_uint64), ("t_submit_ns", C.c_uint64),
                ("t_start_ns", C.c_uint64), ("t_done_ns", C.c_uint64), ("step", C.c_uint64)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("rejected", C.c_uint64),
                ("points", C.c_uint64), ("steps", C.c_uint64), ("step_requests_max", C.c_uint64),
                ("n_slots", C.c_uint32), ("host_reads", C.c_uint32), ("device_bytes", C.c_uint64),
                ("p50_us", C.c_double), ("p99_us", C.c_double), ("mean_us", C.c_double), ("max_us", C.c_double),
                ("memory_waits", C.c_uint64), ("peak_bytes_in_use", C.c_uint64), ("index_bytes", C.c_uint64),
                ("n_indexes", C.c_uint32), ("reserved", C.c_uint32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class LoadSpec(C.Structure):
    _fields_ = [("rate", C.c_double), ("n_requests", C.c_uint64), ("zipf_alpha", C.c_double),
                ("max_points", C.c_uint32), ("n_sets", C.c_uint32), ("exact_fraction", C.c_double),
                ("approx_index", C.c_void_p), ("exact_index", C.c_void_p), ("pools", C.c_void_p),
                ("pool_points", C.c_void_p), ("seed", C.c_uint64), ("warmup_requests", C.c_uint64)]


class LoadResult(C.Structure):
    _fields_ = [("requests", C.c_uint64), ("points", C.c_uint64), ("rejected", C.c_uint64),
                ("seconds", C.c_double), ("offered_rate", C.c_double), ("achieved_rate", C.c_double),
                ("points_per_s", C.c_double), ("p50_us", C.c_double), ("p99_us", C.c_double),
                ("mean_us", C.c_double), ("max_us", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class BatchOpts(C.Structure):
    _fields_ = [("points_per_lane", C.c_uint32), ("ctas_per_sm", C.c_uint32), ("no_graph", C.c_uint32),
                ("reserved", C.c_uint32)]


_lib = None
_lock = threading.Lock()


def lib():
    """The loaded native library (built in-tree on first use)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build()
        L = C.CDLL(path)
        P, u32, u64, i32, d = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int, C.c_double
        sig = {
            "agj_strerror": (C.c_char_p, [i32]),
            "agj_last_error": (C.c_char_p, []),
            "agj_build": (i32, [P, u32, d, i32, P, P, P]),
            "agj_free": (None, [P]),
            "agj_index_stats": (i32, [P, P]),
            "agj_index_logical": (i32, [P, P, P, P, P, P]),
            "agj_index_trie": (i32, [P, P, P, P]),
            "agj_supercover": (i32, [P, P, u64, P, P, P, P, P]),
            "agj_lut_encode": (i32, [P, P, u64, P, P, P]),
            "agj_join_requirements": (i32, [P, u64, P]),
            "agj_pairs_alloc": (i32, [P, u64, P, P]),
            "agj_pairs_free": (i32, [P, P]),
            "agj_join": (i32, [P, P, u64, P, P]),
            "agj_join_timed": (i32, [P, P, u64, P, P, P]),
            "agj_join_check": (i32, [P, P, P]),
            "agj_join_host": (i32, [P, P, u64, P, P, P, P, u64, P, P]),
            "agj_cell_ids": (i32, [P, u64, P, P]),
            "agj_selftest_scan_timeout": (i32, [P]),
            "agj_selftest_ready_timeout": (i32, [P]),
            "agj_cell_ids_host": (i32, [P, u64, P]),
            "agj_fast_ids_host": (i32, [P, P, u64, P, P]),
            "agj_covers_certified_host": (i32, [P, P, P, u64, P]),
            "agj_batch_create": (i32, [P, P, u32, P, P]),
            "agj_batch_run": (i32, [P, P, P, P]),
            "agj_batch_device_bytes": (u64, [P]),
            "agj_batch_free": (None, [P]),
            "agj_join_batched": (i32, [P, P, P, u32, P, P]),
            "agj_server_create": (i32, [P, u32, P, P]),
            "agj_server_submit": (i32, [P, u32, P, u64, P, P, u64, P]),
            "agj_server_add_index": (i32, [P, P, P]),
            "agj_server_poll": (i32, [P, u64, i32, P]),
            "agj_server_drain": (i32, [P]),
            "agj_server_get_stats": (i32, [P, i32, P]),
            "agj_server_destroy": (None, [P]),
            "agj_server_load": (i32, [P, P, P]),
            "agj_plain_load": (i32, [P, u32, P, P]),
            "agj_count_scratch_bytes": (u64, [P, u64]),
            "agj_join_count": (i32, [P, P, u64, P, P, i32, P, P, u64]),
            "agj_join_count_timed": (i32, [P, P, u64, P, P, i32, P, P, u64, P]),
            "agj_measure_fp64_rate": (i32, [P, P]),
            "agj_train_online": (i32, [P, P, u64, u64, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def _check(rc: int, what: str):
    if rc != AGJ_OK:
        raise AgjError(rc, what)


def _np_ptr(a: np.ndarray):
    return C.c_void_p(a.ctypes.data)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class Index:
    """An adaptive geospatial join index resident on the current CUDA device."""

    def __init__(self, polygons, mode: int = APPROX, precision_m: float = 10.0, train=None,
                 budget_bytes: int = 0, threads: int = 0, max_cover_cells: int = 0, max_interior_cells: int = 0,
                 max_interior_level: int = 0, host_only: bool = False, fast_ids: bool = True, pip_bands: bool = True,
                 predicate: int = COVERS, stream=None):
        L = lib()
        # polygons: each an (V,2) (lat,lng) ring, or [outer, hole, ...]
        rings = [_polygon_rings(p) for p in polygons]
        self._polys = [np.ascontiguousarray(np.concatenate(rs)) for rs in rings]
        self._ring_ends = [np.cumsum([len(r) for r in rs]).astype(np.uint32) for rs in rings]
        arr = (Polygon * max(len(self._polys), 1))()
        for k, p in enumerate(self._polys):
            arr[k].n_vertices = len(p)
            arr[k].latlng = p.ctypes.data
            arr[k].n_rings = len(rings[k])
            arr[k].ring_ends = self._ring_ends[k].ctypes.data
        opts = BuildOpts()
        opts.memory_budget_bytes = int(budget_bytes)
        opts.n_threads = int(threads)
        opts.max_cover_cells = int(max_cover_cells)
        opts.max_interior_cells = int(max_interior_cells)
        opts.max_interior_level = int(max_interior_level)
        opts.host_only = 1 if host_only else 0
        opts.no_fast_ids = 0 if fast_ids else 1
        opts.no_pip_bands = 0 if pip_bands else 1
        opts.predicate = int(predicate)
        self._train = None
        if train is not None:
            self._train = np.ascontiguousarray(train, dtype=np.float64).reshape(-1, 2)
            opts.train_latlng = self._train.ctypes.data
            opts.n_train = len(self._train)
        h = C.c_void_p()
        rc = L.agj_build(arr, len(self._polys), float(precision_m), int(mode), C.byref(opts),
                         C.c_void_p(0) if host_only else _stream_ptr(stream), C.byref(h))
        _check(rc, "agj_build")
        self._h = h
        self.mode = self.stats()["mode"]      # AUTO resolves to APPROX or EXACT
        self.precision_m = precision_m

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().agj_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def stats(self) -> dict:
        s = Stats()
        _check(lib().agj_index_stats(self._h, C.byref(s)), "agj_index_stats")
        return s.as_dict()

    def logical(self):
        """(cells u64[m], ref_off u64[m+1], refs u32[]) of the super covering."""
        L = lib()
        m, r = C.c_uint64(), C.c_uint64()
        _check(L.agj_index_logical(self._h, None, None, None, C.byref(m), C.byref(r)), "agj_index_logical")
        cells = np.zeros(m.value, dtype=np.uint64)
        off = np.zeros(m.value + 1, dtype=np.uint64)
        refs = np.zeros(max(r.value, 1), dtype=np.uint32)
        _check(L.agj_index_logical(self._h, _np_ptr(cells), _np_ptr(off), _np_ptr(refs), None, None),
               "agj_index_logical")
        return cells, off, refs[:r.value]

    def trie(self):
        """(nodes u64[n_nodes*256], lut u32[], face_table u64[18])."""
        st = self.stats()
        nodes = np.zeros(max(st["n_nodes"] * 256, 1), dtype=np.uint64)
        lut = np.zeros(max(st["n_lut_words"], 1), dtype=np.uint32)
        ft = np.zeros(18, dtype=np.uint64)
        _check(lib().agj_index_trie(self._h, _np_ptr(nodes), _np_ptr(lut), _np_ptr(ft)), "agj_index_trie")
        return nodes[:st["n_nodes"] * 256], lut[:st["n_lut_words"]], ft

    def fast_ids_host(self, points: np.ndarray):
        """(ids u64, certified levels u8; 255 = outside the window) of the
        certified fast cell-id step, computed on the host."""
        pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 2)
        ids = np.zeros(len(pts), dtype=np.uint64)
        lv = np.zeros(len(pts), dtype=np.uint8)
        _check(lib().agj_fast_ids_host(self._h, _np_ptr(pts), len(pts), _np_ptr(ids), _np_ptr(lv)),
               "agj_fast_ids_host")
        return ids, lv

    def covers_certified_host(self, points: np.ndarray, polys: np.ndarray) -> np.ndarray:
        """Certified FP32 refine decisions (1, 0, -1 undecided) on the host."""
        pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 2)
        pl = np.ascontiguousarray(polys, dtype=np.uint32)
        out = np.zeros(len(pts), dtype=np.int8)
        _check(lib().agj_covers_certified_host(self._h, _np_ptr(pts), _np_ptr(pl), len(pts), _np_ptr(out)),
               "agj_covers_certified_host")
        return out

    def requirements(self, n: int) -> tuple[int, int]:
        r = Requirements()
        _check(lib().agj_join_requirements(self._h, int(n), C.byref(r)), "agj_join_requirements")
        return int(r.ids_capacity), int(r.scratch_bytes)


class Pairs:
    """CSR output buffers (torch device tensors) for joins of up to n points."""

    def __init__(self, index: Index, n: int, device=None):
        import torch
        cap, scratch = index.requirements(n)
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.n_max = int(n)
        self.offsets = torch.empty(n + 1, dtype=torch.int32, device=dev)
        self.ids = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
        self.scratch = torch.empty(max(scratch, 256), dtype=torch.uint8, device=dev)
        self.status = torch.zeros(4, dtype=torch.int64, device=dev)
        self.c = PairsC()
        self.c.offsets = self.offsets.data_ptr()
        self.c.ids = self.ids.data_ptr()
        self.c.ids_capacity = cap
        self.c.scratch = self.scratch.data_ptr()
        self.c.scratch_bytes = scratch
        self.c.status = self.status.data_ptr()
        self.n = 0

    def check(self, stream=None) -> int:
        nnz = C.c_uint64()
        _check(lib().agj_join_check(C.byref(self.c), _stream_ptr(stream), C.byref(nnz)), "agj_join (device status)")
        return int(nnz.value)

    def fallbacks(self) -> int:
        """Points of the last join whose walk recomputed the FP64 cell id."""
        return int(self.scratch[16:24].cpu().view(torch_int64()).item())

    def refine_fallbacks(self) -> int:
        """Candidates of the last exact join whose refine test ran in FP64."""
        return int(self.scratch[24:32].cpu().view(torch_int64()).item())

    def to_host(self, stream=None):
        """(offsets u32[n+1], ids u32[nnz]) as numpy, after a status check."""
        nnz = self.check(stream)
        off = self.offsets[: self.n + 1].cpu().numpy().view(np.uint32)
        ids = self.ids[:nnz].cpu().numpy().view(np.uint32)
        return off, ids


def torch_int64():
    import torch
    return torch.int64


def join(index: Index, points, pairs: Pairs | None = None, stream=None) -> Pairs:
    """Joins device points (torch float64 (n,2) {lat,lng}) against the index."""
    import torch
    assert points.is_cuda and points.dtype == torch.float64 and points.is_contiguous()
    n = points.shape[0]
    if pairs is None or pairs.n_max < n:
        pairs = Pairs(index, n, device=points.device)
    pairs.n = n
    rc = lib().agj_join(index.handle, C.c_void_p(points.data_ptr()), n, _stream_ptr(stream), C.byref(pairs.c))
    _check(rc, "agj_join")
    return pairs


def join_timed(index: Index, points, pairs: Pairs, events, stream=None) -> Pairs:
    """agj_join recording four torch.cuda.Event objects at the stage
    boundaries (see include/agj.h, agj_join_timed)."""
    arr = (C.c_void_p * 4)(*[C.c_void_p(e.cuda_event) for e in events])
    pairs.n = points.shape[0]
    _check(lib().agj_join_timed(index.handle, C.c_void_p(points.data_ptr()), points.shape[0], _stream_ptr(stream),
                                C.byref(pairs.c), arr), "agj_join_timed")
    return pairs


def join_host(index: Index, points: np.ndarray, pairs: Pairs, staging, h_offsets: np.ndarray, h_ids: np.ndarray,
              stream=None) -> int:
    """End-to-end join from host memory into host CSR arrays; returns nnz."""
    pts = points
    n = pts.shape[0]
    nnz = C.c_uint64()
    pairs.n = n
    rc = lib().agj_join_host(index.handle, C.c_void_p(pts.ctypes.data if isinstance(pts, np.ndarray) else pts.data_ptr()),
                             n, C.c_void_p(staging.data_ptr()), C.byref(pairs.c),
                             C.c_void_p(h_offsets.ctypes.data if isinstance(h_offsets, np.ndarray) else h_offsets.data_ptr()),
                             C.c_void_p(h_ids.ctypes.data if isinstance(h_ids, np.ndarray) else h_ids.data_ptr()),
                             int(h_ids.shape[0]), C.byref(nnz), _stream_ptr(stream))
    _check(rc, "agj_join_host")
    return int(nnz.value)


class Counts:
    """Aggregation-mode buffers (torch device tensors) for joins of up to n
    points: counts (int64 per polygon, read as uint64), status (4 words) and
    the work space."""

    def __init__(self, index: Index, n: int, device=None):
        import torch
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.n_max = int(n)
        self.n_polys = int(index.stats()["n_polys"])
        self.counts = torch.zeros(max(self.n_polys, 1), dtype=torch.int64, device=dev)
        self.status = torch.zeros(4, dtype=torch.int64, device=dev)
        self.scratch_bytes = int(lib().agj_count_scratch_bytes(index.handle, int(n)))
        self.scratch = torch.empty(max(self.scratch_bytes, 256), dtype=torch.uint8, device=dev)

    def to_host(self) -> np.ndarray:
        """counts (uint64 per polygon) after a status check."""
        st = self.status.cpu().numpy().view(np.uint64)
        if st[1]:
            raise AgjError(AGJ_EDEVICE, f"agj_join_count (device status {int(st[1])})")
        return self.counts[: self.n_polys].cpu().numpy().view(np.uint64)

    def fallbacks(self) -> int:
        return int(self.scratch[16:24].cpu().view(torch_int64()).item())


def join_count(index: Index, points, counts: Counts | None = None, accumulate: bool = False, stream=None,
               events=None) -> Counts:
    """Aggregation mode (agj_join_count): per-polygon counts of the join of
    device points (torch float64 (n,2)) with the index."""
    import torch
    assert points.is_cuda and points.dtype == torch.float64 and points.is_contiguous()
    n = points.shape[0]
    if counts is None or counts.n_max < n:
        counts = Counts(index, n, device=points.device)
    args = (index.handle, C.c_void_p(points.data_ptr()), n, _stream_ptr(stream), C.c_void_p(counts.counts.data_ptr()),
            1 if accumulate else 0, C.c_void_p(counts.status.data_ptr()), C.c_void_p(counts.scratch.data_ptr()),
            counts.scratch_bytes)
    if events is None:
        _check(lib().agj_join_count(*args), "agj_join_count")
    else:
        arr = (C.c_void_p * 4)(*[C.c_void_p(e.cuda_event) for e in events])
        _check(lib().agj_join_count_timed(*args, arr), "agj_join_count_timed")
    return counts


def train_online(index: Index, points, budget_bytes: int = 0, stream=None) -> None:
    """Trains an exact index from device points (agj_train_online)."""
    import torch
    assert points.is_cuda and points.dtype == torch.float64 and points.is_contiguous()
    _check(lib().agj_train_online(index.handle, C.c_void_p(points.data_ptr()), points.shape[0], int(budget_bytes),
                                  _stream_ptr(stream)), "agj_train_online")


def measure_fp64_rate(stream=None) -> float:
    """FP64 FMA throughput of the current device in flop/s (agj_measure_fp64_rate)."""
    r = C.c_double()
    _check(lib().agj_measure_fp64_rate(_stream_ptr(stream), C.byref(r)), "agj_measure_fp64_rate")
    return float(r.value)


class Batch:
    """A batched-join plan (agj_batch_create) for fixed (index, point count)
    jobs; run() joins one point batch per job into one Pairs per job."""

    def __init__(self, indexes, ns, points_per_lane: int = 0, ctas_per_sm: int = 0, graph: bool = True):
        m = len(indexes)
        assert len(ns) == m
        self.indexes = list(indexes)
        self.ns = [int(x) for x in ns]
        self.opts = (int(points_per_lane), int(ctas_per_sm), bool(graph))
        hs = (C.c_void_p * max(m, 1))(*[ix.handle for ix in self.indexes])
        nn = (C.c_uint64 * max(m, 1))(*self.ns)
        o = BatchOpts(int(points_per_lane), int(ctas_per_sm), 0 if graph else 1, 0)
        h = C.c_void_p()
        _check(lib().agj_batch_create(hs, nn, m, C.byref(o), C.byref(h)), "agj_batch_create")
        self._h = h

    def device_bytes(self) -> int:
        return int(lib().agj_batch_device_bytes(self._h))

    def pairs(self, device=None) -> list:
        """One Pairs per job, sized for that job."""
        return [Pairs(ix, n, device=device) for ix, n in zip(self.indexes, self.ns)]

    def run(self, points, pairs: list, stream=None) -> list:
        import torch
        m = len(self.indexes)
        assert len(points) == m and len(pairs) == m
        for p, n in zip(points, self.ns):
            assert p.is_cuda and p.dtype == torch.float64 and p.is_contiguous() and p.shape[0] == n
        pp = (C.c_void_p * max(m, 1))(*[C.c_void_p(p.data_ptr()) for p in points])
        arr = (PairsC * max(m, 1))(*[q.c for q in pairs])
        for q, n in zip(pairs, self.ns):
            q.n = n
        _check(lib().agj_batch_run(self._h, pp, _stream_ptr(stream), arr), "agj_batch_run")
        return pairs

    def close(self):
        if getattr(self, "_h", None):
            lib().agj_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def join_batched(indexes, points, pairs: list | None = None, stream=None) -> list:
    """One-shot batched join (agj_join_batched): synchronises the stream."""
    m = len(indexes)
    if pairs is None:
        pairs = [Pairs(ix, p.shape[0], device=p.device) for ix, p in zip(indexes, points)]
    hs = (C.c_void_p * max(m, 1))(*[ix.handle for ix in indexes])
    pp = (C.c_void_p * max(m, 1))(*[C.c_void_p(p.data_ptr()) for p in points])
    nn = (C.c_uint64 * max(m, 1))(*[int(p.shape[0]) for p in points])
    arr = (PairsC * max(m, 1))(*[q.c for q in pairs])
    for q, p in zip(pairs, points):
        q.n = int(p.shape[0])
    _check(lib().agj_join_batched(hs, pp, nn, m, _stream_ptr(stream), arr), "agj_join_batched")
    return pairs


class Server:
    """The served form (agj_server_*): continuous batching of host point
    requests over resident indexes."""

    def __init__(self, indexes, n_slots: int = 0, max_step_requests: int = 0, max_step_points: int = 0,
                 hbm_budget_bytes: int = 0, max_pending: int = 0, points_per_lane: int = 0, ctas_per_sm: int = 0,
                 stage_points: bool = False, max_refs: int = 0, hbm_reserve_bytes: int = 0):
        self.indexes = list(indexes)
        hs = (C.c_void_p * len(self.indexes))(*[ix.handle for ix in self.indexes])
        o = ServerOpts(n_slots, max_step_requests, max_step_points, hbm_budget_bytes, max_pending, points_per_lane,
                       ctas_per_sm, 1 if stage_points else 0, max_refs, hbm_reserve_bytes)
        h = C.c_void_p()
        _check(lib().agj_server_create(hs, len(self.indexes), C.byref(o), C.byref(h)), "agj_server_create")
        self._h = h
        self._live = {}

    def add_index(self, index: "Index") -> int:
        """Admits an index (agj_server_add_index): a host-only index is uploaded
        if it fits the free device memory less the reserve.  Returns its id."""
        k = C.c_uint32()
        _check(lib().agj_server_add_index(self._h, index.handle, C.byref(k)), "agj_server_add_index")
        self.indexes.append(index)
        return int(k.value)

    def submit(self, index_id: int, points: np.ndarray, keep: bool = True) -> int:
        """Queues a request; with keep, its CSR is returned by poll()."""
        pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 2)
        n = pts.shape[0]
        t = C.c_uint64()
        if keep:
            cap = n * max(self.indexes[index_id].stats()["max_refs"], 1)
            off = np.empty(n + 1, dtype=np.uint32)
            ids = np.empty(max(cap, 1), dtype=np.uint32)
            rc = lib().agj_server_submit(self._h, index_id, _np_ptr(pts), n, _np_ptr(off), _np_ptr(ids), cap,
                                         C.byref(t))
        else:
            off = ids = None
            rc = lib().agj_server_submit(self._h, index_id, _np_ptr(pts), n, None, None, 0, C.byref(t))
        _check(rc, "agj_server_submit")
        self._live[int(t.value)] = (pts, off, ids)
        return int(t.value)

    def poll(self, ticket: int, wait: bool = True):
        """(offsets, ids, result dict) of a kept request, or None while it runs."""
        r = RequestResult()
        rc = lib().agj_server_poll(self._h, ticket, 1 if wait else 0, C.byref(r))
        if rc == 7 and not wait:      # AGJ_EBUSY
            return None
        _check(rc, "agj_server_poll")
        pts, off, ids = self._live.pop(ticket)
        res = {k: getattr(r, k) for k, _ in r._fields_ if k != "reserved"}
        _check(r.status, "served request")
        return off, ids[: r.nnz].copy(), res

    def drain(self):
        _check(lib().agj_server_drain(self._h), "agj_server_drain")
        for t in [t for t, v in self._live.items() if v[1] is None]:
            self._live.pop(t)

    def stats(self, reset: bool = False) -> dict:
        st = ServerStats()
        _check(lib().agj_server_get_stats(self._h, 1 if reset else 0, C.byref(st)), "agj_server_get_stats")
        return st.as_dict()

    def load(self, spec: "LoadSpecPy") -> dict:
        res = LoadResult()
        _check(lib().agj_server_load(self._h, C.byref(spec.c), C.byref(res)), "agj_server_load")
        return res.as_dict()

    def close(self):
        if getattr(self, "_h", None):
            lib().agj_server_destroy(self._h)
            self._h = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class LoadSpecPy:
    """agj_load_spec with the arrays it points to kept alive."""

    def __init__(self, rate: float, n_requests: int, pools, approx_index, exact_index=None, zipf_alpha: float = 1.2,
                 max_points: int = 65536, exact_fraction: float = 0.0, seed: int = 0, warmup_requests: int = 0):
        self.pools = [np.ascontiguousarray(p, dtype=np.float64).reshape(-1, 2) for p in pools]
        n_sets = len(self.pools)
        self._ptrs = (C.c_void_p * n_sets)(*[p.ctypes.data for p in self.pools])
        self._counts = (C.c_uint64 * n_sets)(*[p.shape[0] for p in self.pools])
        self._approx = (C.c_uint32 * n_sets)(*approx_index)
        self._exact = (C.c_uint32 * n_sets)(*(exact_index if exact_index is not None else [0xFFFFFFFF] * n_sets))
        self.c = LoadSpec(rate, n_requests, zipf_alpha, max_points, n_sets, exact_fraction,
                          C.cast(self._approx, C.c_void_p), C.cast(self._exact, C.c_void_p),
                          C.cast(self._ptrs, C.c_void_p), C.cast(self._counts, C.c_void_p), seed, warmup_requests)


def plain_load(indexes, spec: LoadSpecPy) -> dict:
    """The spec's arrivals served one request at a time by agj_join_host."""
    hs = (C.c_void_p * len(indexes))(*[ix.handle for ix in indexes])
    res = LoadResult()
    _check(lib().agj_plain_load(hs, len(indexes), C.byref(spec.c), C.byref(res)), "agj_plain_load")
    return res.as_dict()


def supercover(cells, refs):
    """The super-covering merge (§III-B) of (cell, ref) pairs, in order."""
    L = lib()
    cells = np.ascontiguousarray(cells, dtype=np.uint64)
    refs = np.ascontiguousarray(refs, dtype=np.uint32)
    m, r = C.c_uint64(), C.c_uint64()
    _check(L.agj_supercover(_np_ptr(cells), _np_ptr(refs), len(cells), None, None, None, C.byref(m), C.byref(r)),
           "agj_supercover")
    oc = np.zeros(max(m.value, 1), dtype=np.uint64)
    oo = np.zeros(m.value + 1, dtype=np.uint64)
    orf = np.zeros(max(r.value, 1), dtype=np.uint32)
    _check(L.agj_supercover(_np_ptr(cells), _np_ptr(refs), len(cells), _np_ptr(oc), _np_ptr(oo), _np_ptr(orf),
                            None, None), "agj_supercover")
    return oc[:m.value], oo, orf[:r.value]


def lut_encode(lists):
    """Lookup-table encoding (§III-C) of reference lists -> (words, offsets)."""
    L = lib()
    flat = np.array([r for lst in lists for r in lst], dtype=np.uint32)
    off = np.zeros(len(lists) + 1, dtype=np.uint64)
    off[1:] = np.cumsum([len(x) for x in lists])
    nw = C.c_uint64()
    _check(L.agj_lut_encode(_np_ptr(flat), _np_ptr(off), len(lists), None, None, C.byref(nw)), "agj_lut_encode")
    words = np.zeros(max(nw.value, 1), dtype=np.uint32)
    offs = np.zeros(max(len(lists), 1), dtype=np.uint64)
    _check(L.agj_lut_encode(_np_ptr(flat), _np_ptr(off), len(lists), _np_ptr(words), _np_ptr(offs), None),
           "agj_lut_encode")
    return words[:nw.value], offs[:len(lists)]


def cell_ids(points, stream=None, out=None):
    """Device cell ids (FP64 spec) of torch float64 (n,2) points, as int64 bit patterns."""
    import torch
    if out is None:
        out = torch.empty(points.shape[0], dtype=torch.int64, device=points.device)
    assert out.is_cuda and out.dtype == torch.int64 and out.numel() >= points.shape[0]
    rc = lib().agj_cell_ids(C.c_void_p(points.data_ptr()), points.shape[0], C.c_void_p(out.data_ptr()),
                            _stream_ptr(stream))
    _check(rc, "agj_cell_ids")
    return out


def cell_ids_host(points: np.ndarray) -> np.ndarray:
    """Host cell ids with the same spec (library host code)."""
    pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 2)
    out = np.zeros(len(pts), dtype=np.uint64)
    _check(lib().agj_cell_ids_host(_np_ptr(pts), len(pts), _np_ptr(out)), "agj_cell_ids_host")
    return out
