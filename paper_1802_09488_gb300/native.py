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
APPROX, EXACT = 0, 1


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
    _fields_ = [("n_vertices", C.c_uint32), ("latlng", C.c_void_p)]


class BuildOpts(C.Structure):
    _fields_ = [("max_cover_cells", C.c_uint32), ("max_cover_level", C.c_uint32),
                ("max_interior_cells", C.c_uint32), ("max_interior_level", C.c_uint32),
                ("memory_budget_bytes", C.c_uint64), ("train_latlng", C.c_void_p), ("n_train", C.c_uint64),
                ("max_train_level", C.c_uint32), ("n_threads", C.c_uint32), ("host_only", C.c_uint32),
                ("no_fast_ids", C.c_uint32)]


class Stats(C.Structure):
    _fields_ = [("mode", C.c_uint32), ("n_polys", C.c_uint32), ("n_cells", C.c_uint64),
                ("n_cand_cells", C.c_uint64), ("n_nodes", C.c_uint64), ("n_lut_words", C.c_uint64),
                ("device_bytes", C.c_uint64), ("max_refs", C.c_uint32), ("max_cand_refs", C.c_uint32),
                ("max_depth", C.c_uint32), ("max_level", C.c_uint32), ("build_seconds", C.c_double),
                ("fast_ids", C.c_uint32), ("reserved", C.c_uint32), ("fast_err_cells", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class PairsC(C.Structure):
    _fields_ = [("offsets", C.c_void_p), ("ids", C.c_void_p), ("ids_capacity", C.c_uint64),
                ("scratch", C.c_void_p), ("scratch_bytes", C.c_uint64), ("status", C.c_void_p)]


class Requirements(C.Structure):
    _fields_ = [("ids_capacity", C.c_uint64), ("scratch_bytes", C.c_uint64)]


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
            "agj_cell_ids_host": (i32, [P, u64, P]),
            "agj_fast_ids_host": (i32, [P, P, u64, P, P]),
            "agj_covers_certified_host": (i32, [P, P, P, u64, P]),
            "agj_batch_create": (i32, [P, P, u32, P, P]),
            "agj_batch_run": (i32, [P, P, P, P]),
            "agj_batch_device_bytes": (u64, [P]),
            "agj_batch_free": (None, [P]),
            "agj_join_batched": (i32, [P, P, P, u32, P, P]),
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
                 max_interior_level: int = 0, host_only: bool = False, fast_ids: bool = True, stream=None):
        L = lib()
        self._polys = [np.ascontiguousarray(p, dtype=np.float64).reshape(-1, 2) for p in polygons]
        arr = (Polygon * max(len(self._polys), 1))()
        for k, p in enumerate(self._polys):
            arr[k].n_vertices = len(p)
            arr[k].latlng = p.ctypes.data
        opts = BuildOpts()
        opts.memory_budget_bytes = int(budget_bytes)
        opts.n_threads = int(threads)
        opts.max_cover_cells = int(max_cover_cells)
        opts.max_interior_cells = int(max_interior_cells)
        opts.max_interior_level = int(max_interior_level)
        opts.host_only = 1 if host_only else 0
        opts.no_fast_ids = 0 if fast_ids else 1
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
        self.mode = mode
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


def cell_ids(points, stream=None):
    """Device cell ids (FP64 spec) of torch float64 (n,2) points, as int64 bit patterns."""
    import torch
    out = torch.empty(points.shape[0], dtype=torch.int64, device=points.device)
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
