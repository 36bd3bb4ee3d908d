"""Thin ctypes binding of libsdb.so (C ABI in include/sdb.h).

Argument marshalling only: every step of the method runs in the CUDA
library.  Device arrays are passed as torch CUDA tensors (their data
pointers), streams as torch streams; PyTorch provides device memory and
streams, nothing else.  If libsdb.so is missing the import fails: there is no
fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsdb.so")

SDB_OK, SDB_EINVAL, SDB_ENOMEM, SDB_ECUDA, SDB_ETIMEOUT, SDB_EBUSY = range(6)
LOOKUP_BINARY, LOOKUP_LEARNED, LOOKUP_RADIX_SPLINE, LOOKUP_TABLE, LOOKUP_TABLE_LEARNED = 0, 1, 2, 3, 4
COVER_BOUNDARY_FLAGS, COVER_NONCONSERVATIVE = 1, 2


class SdbError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"sdb status {status}: {msg}")
        self.status = status


class _Polys(C.Structure):
    _fields_ = [("n_polygons", C.c_uint32), ("ring_off", C.c_void_p), ("x", C.c_void_p),
                ("y", C.c_void_p)]


class _MultiPolys(C.Structure):
    _fields_ = [("n_polygons", C.c_uint32), ("n_rings", C.c_uint32),
                ("poly_ring_off", C.c_void_p), ("ring_off", C.c_void_p), ("x", C.c_void_p),
                ("y", C.c_void_p)]


def _polys_arg(polys, keep):
    """(struct, is_multi) for a polygon set; numpy arrays kept alive in keep.
    A set with poly_ring_off holds polygons of several rings."""
    arrs = [np.ascontiguousarray(a, np.uint32) for a in (polys.ring_off, polys.x, polys.y)]
    keep.extend(arrs)
    pro = getattr(polys, "poly_ring_off", None)
    if pro is None:
        return _Polys(len(arrs[0]) - 1, _np_ptr(arrs[0]), _np_ptr(arrs[1]), _np_ptr(arrs[2])), False
    pro = np.ascontiguousarray(pro, np.uint32)
    keep.append(pro)
    return _MultiPolys(len(pro) - 1, len(arrs[0]) - 1, _np_ptr(pro), _np_ptr(arrs[0]),
                       _np_ptr(arrs[1]), _np_ptr(arrs[2])), True


class CoveringInfo(C.Structure):
    _fields_ = [("grid_bits", C.c_uint32), ("finest_shift", C.c_uint32),
                ("finest_level", C.c_uint32), ("n_polygons", C.c_uint32),
                ("n_ranges", C.c_uint64), ("n_list_ids", C.c_uint64), ("n_cells", C.c_uint64),
                ("device_bytes", C.c_uint64), ("index_leaf_bits", C.c_uint32),
                ("boundary_flags", C.c_uint32), ("table_bits", C.c_uint32),
                ("table_mixed", C.c_uint64), ("table_sub_bits", C.c_uint32),
                ("table_sub_mixed", C.c_uint64), ("index_root_bits", C.c_uint32)]


class Query(C.Structure):
    _fields_ = [("x0", C.c_uint32), ("y0", C.c_uint32), ("x1", C.c_uint32), ("y1", C.c_uint32),
                ("eps", C.c_uint64), ("poly_off", C.c_uint32), ("poly_cnt", C.c_uint32)]


class BatchInfo(C.Structure):
    _fields_ = [("n_queries", C.c_uint32), ("n_pairs", C.c_uint32), ("out_len", C.c_uint64),
                ("n_ranges", C.c_uint64), ("max_ranges", C.c_uint64), ("n_cells", C.c_uint64),
                ("candidates", C.c_uint64), ("n_tiles", C.c_uint64), ("tile", C.c_uint32),
                ("points_per_thread", C.c_uint32), ("lookup", C.c_uint32),
                ("indexed_queries", C.c_uint32), ("n_leaves", C.c_uint64)]


BATCH_PERSISTENT, BATCH_PER_QUERY, BATCH_GRAPH = 0, 1, 2


class ServerConfig(C.Structure):
    _fields_ = [("workers", C.c_uint32), ("max_batch", C.c_uint32), ("cache_bytes", C.c_uint64),
                ("use_cache", C.c_uint32), ("per_query", C.c_uint32), ("tile", C.c_uint32),
                ("points_per_thread", C.c_uint32), ("lookup", C.c_uint32)]


class TicketInfo(C.Structure):
    _fields_ = [("latency_ms", C.c_double), ("queue_ms", C.c_double), ("batch_size", C.c_uint32),
                ("cache_hit", C.c_uint32), ("ranges", C.c_uint64)]


class ServerStats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("submitted", "completed", "batches", "cache_hits",
                                          "cache_misses", "evictions", "cache_bytes",
                                          "cache_entries", "peak_bytes")]

_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        P, U32, U64, I = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int
        sig = {
            "sdb_finest_level": ([U32, U64, P, P], I),
            "sdb_build_covering": ([P, U32, U64, P, P], I),
            "sdb_build_covering_ex": ([P, U32, U64, U32, P, P], I),
            "sdb_build_covering_multi": ([P, U32, U64, U32, P, P], I),
            "sdb_build_coverings": ([P, U32, P, U32, U32, P, P], I),
            "sdb_join_aggregate_multi": ([P, P, P, U64, P, U32, I, P, P, P], I),
            "sdb_raster_join_multi": ([P, U32, U64, P, P, P, U64, U32, P, P, P], I),
            "sdb_join_aggregate_range": ([P, P, P, U64, P, I, P, P, P, P, P, P], I),
            "sdb_result_bounds": ([P, P, P, P, P, U32, P, P, P, P, P], I),
            "sdb_covering_get_info": ([P, P], I),
            "sdb_covering_build_index": ([P, U32, P], I),
            "sdb_covering_build_index_ex": ([P, U32, U32, P], I),
            "sdb_covering_build_table": ([P, U32, P], I),
            "sdb_trace_enable": ([C.c_int], I),
            "sdb_trace_read": ([P, U32, P], I),
            "sdb_join_aggregate": ([P, P, P, U64, P, I, P, P, P], I),
            "sdb_join_aggregate_host": ([P, P, P, U64, P, U32, I, P, P, P], I),
            "sdb_covering_fallbacks": ([P, P, P], I),
            "sdb_covering_export": ([P, P, P, P], I),
            "sdb_covering_free": ([P], None),
            "sdb_status_string": ([I], C.c_char_p),
            "sdb_last_error": ([], C.c_char_p),
            "sdb_launch_count": ([], U64),
            "sdb_memory_stats": ([P, P], I),
            "sdb_covering_index_stats": ([P, P, P], I),
            "sdb_points_create": ([P, P, P, U64, U32, P, P], I),
            "sdb_points_free": ([P], None),
            "sdb_points_build_index": ([P, U32, U32, P], I),
            "sdb_raster_join": ([P, U32, U64, P, P, P, U64, U32, P, P, P], I),
            "sdb_points_aggregate": ([P, P, I, P, P, P], I),
            "sdb_points_index_stats": ([P, P, P, P, P], I),
            "sdb_batch_create": ([P, P, P, U32, P, U64, P, P], I),
            "sdb_batch_get_info": ([P, P], I),
            "sdb_batch_query_ranges": ([P, P], I),
            "sdb_batch_run": ([P, I, P, P, P], I),
            "sdb_batch_autotune": ([P, P, P, P], I),
            "sdb_batch_set_tuning": ([P, U32, U32, P], I),
            "sdb_batch_set_lookup": ([P, I, P], I),
            "sdb_batch_fallbacks": ([P, P, P], I),
            "sdb_batch_free": ([P], None),
            "sdb_server_create": ([P, P, P, P], I),
            "sdb_server_submit": ([P, P, P, P], I),
            "sdb_server_wait": ([P, U64, U32, P, P, P], I),
            "sdb_server_get_stats": ([P, P], I),
            "sdb_server_destroy": ([P], None),
            "sdb_join_aggregate_host_noalloc": ([P, P, P, U64, P, I, P, P, P], I),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(st: int):
    if st != SDB_OK:
        raise SdbError(st, lib().sdb_last_error().decode(errors="replace"))


def _np_ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _dptr(t, itemsize: int):
    """Device pointer of a contiguous CUDA tensor with the given element size
    (uint32/int32 point arrays: 4; uint64/int64 outputs: 8)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("device arrays must be contiguous CUDA tensors")
    if t.element_size() != itemsize:
        raise ValueError(f"expected {itemsize}-byte elements, got {t.dtype}")
    return C.c_void_p(t.data_ptr())


def finest_level(grid_bits: int, eps: int) -> tuple[int, int]:
    """(k, F): finest side 2^k, finest level F (Sec. 2.2)."""
    k, F = C.c_uint32(), C.c_uint32()
    _check(lib().sdb_finest_level(grid_bits, int(eps), C.byref(k), C.byref(F)))
    return k.value, F.value


class Covering:
    """Device-resident covering (owns the library handle)."""

    def __init__(self, handle: int):
        self._h = C.c_void_p(handle)

    @property
    def handle(self):
        return self._h

    def info(self) -> CoveringInfo:
        inf = CoveringInfo()
        _check(lib().sdb_covering_get_info(self._h, C.byref(inf)))
        return inf

    def free(self):
        if self._h and self._h.value:
            lib().sdb_covering_free(self._h)
            self._h = C.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def build_covering(polys, grid_bits: int, eps: int, stream=None, flags: int = 0) -> Covering:
    """sdb_build_covering_ex (or _multi for polygons of several rings): polys has
    ring_off/x/y (and poly_ring_off) uint32 numpy arrays; flags 0,
    COVER_BOUNDARY_FLAGS (result ranges) or COVER_NONCONSERVATIVE."""
    keep = []
    sp, multi = _polys_arg(polys, keep)
    out = C.c_void_p()
    fn = lib().sdb_build_covering_multi if multi else lib().sdb_build_covering_ex
    _check(fn(C.byref(sp), grid_bits, int(eps), int(flags), _stream(stream), C.byref(out)))
    return Covering(out.value)


def raster_join(polys, grid_bits: int, eps: int, x, y, attr, count, sum_=None, tile_bits: int = 0,
                stream=None):
    """sdb_raster_join (Bounded Raster Join) on device tensors; polys as for
    build_covering."""
    keep = []
    sp, multi = _polys_arg(polys, keep)
    n = x.numel() if x is not None else 0
    fn = lib().sdb_raster_join_multi if multi else lib().sdb_raster_join
    _check(fn(C.byref(sp), grid_bits, int(eps), _dptr(x, 4), _dptr(y, 4), _dptr(attr, 4), n,
              tile_bits, _dptr(count, 8), _dptr(sum_, 8), _stream(stream)))


def build_coverings(polys, grid_bits: int, eps_list, stream=None, flags: int = 0):
    """sdb_build_coverings: one covering per eps, built in one pass."""
    keep = []
    sp, multi = _polys_arg(polys, keep)
    if multi:
        return [build_covering(polys, grid_bits, e, stream, flags) for e in eps_list]
    eps = np.ascontiguousarray(eps_list, np.uint64)
    outs = (C.c_void_p * len(eps))()
    _check(lib().sdb_build_coverings(C.byref(sp), grid_bits, _np_ptr(eps), len(eps), int(flags),
                                     _stream(stream), outs))
    return [Covering(o) for o in outs]


def covering_build_index(cov: Covering, leaf_bits: int, stream=None, root_bits=None):
    if root_bits is None:
        _check(lib().sdb_covering_build_index(cov.handle, leaf_bits, _stream(stream)))
    else:
        _check(lib().sdb_covering_build_index_ex(cov.handle, leaf_bits, root_bits,
                                                 _stream(stream)))


def covering_build_table(cov: Covering, table_bits: int, stream=None):
    _check(lib().sdb_covering_build_table(cov.handle, table_bits, _stream(stream)))


def join_aggregate(x, y, attr, cov: Covering, lookup: int, count, sum_=None, stream=None):
    """sdb_join_aggregate on device tensors (uint32 x/y, int32 attr, int64 outputs)."""
    n = x.numel() if x is not None else 0
    _check(lib().sdb_join_aggregate(_dptr(x, 4), _dptr(y, 4), _dptr(attr, 4), n, cov.handle,
                                    lookup, _dptr(count, 8), _dptr(sum_, 8), _stream(stream)))


def join_aggregate_multi(x, y, attr, covs, lookup: int, count, sum_=None, stream=None):
    """sdb_join_aggregate_multi: one pass over the points for several coverings;
    count / sum_ are int64 device tensors of shape (len(covs), P)."""
    n = x.numel() if x is not None else 0
    arr = (C.c_void_p * len(covs))(*[c.handle.value for c in covs])
    _check(lib().sdb_join_aggregate_multi(_dptr(x, 4), _dptr(y, 4), _dptr(attr, 4), n, arr,
                                          len(covs), lookup, _dptr(count, 8), _dptr(sum_, 8),
                                          _stream(stream)))


def join_aggregate_range(x, y, attr, cov: Covering, lookup: int, count, bcount, sum_=None,
                         bsum=None, babs=None, stream=None):
    """sdb_join_aggregate_range on device tensors (int64 outputs of P entries):
    COUNT/SUM plus the boundary partials bounding the exact answers."""
    n = x.numel() if x is not None else 0
    _check(lib().sdb_join_aggregate_range(_dptr(x, 4), _dptr(y, 4), _dptr(attr, 4), n, cov.handle,
                                          lookup, _dptr(count, 8), _dptr(sum_, 8),
                                          _dptr(bcount, 8), _dptr(bsum, 8), _dptr(babs, 8),
                                          _stream(stream)))


def result_bounds(count, bcount, sum_=None, bsum=None, babs=None, stream=None):
    """sdb_result_bounds on the range join's device outputs (int64 tensors of
    P entries): returns device tensors (count_lo, count_hi, sum_lo, sum_hi), the
    sum pair None for COUNT only."""
    import torch
    P = count.numel()
    new = lambda: torch.empty(P, dtype=torch.int64, device=count.device)  # noqa: E731
    c_lo, c_hi = new(), new()
    s_lo, s_hi = (new(), new()) if sum_ is not None else (None, None)
    _check(lib().sdb_result_bounds(_dptr(count, 8), _dptr(sum_, 8), _dptr(bcount, 8),
                                   _dptr(bsum, 8), _dptr(babs, 8), P, _dptr(c_lo, 8),
                                   _dptr(c_hi, 8), _dptr(s_lo, 8), _dptr(s_hi, 8),
                                   _stream(stream)))
    return c_lo, c_hi, s_lo, s_hi


def join_aggregate_host(x, y, attr, covs, lookup: int, stream=None):
    """sdb_join_aggregate_host on numpy arrays; returns (count, sum) of shape
    (len(covs), P) as uint64 / int64 numpy arrays."""
    x = np.ascontiguousarray(x, np.uint32)
    y = np.ascontiguousarray(y, np.uint32)
    a = None if attr is None else np.ascontiguousarray(attr, np.int32)
    P = covs[0].info().n_polygons
    arr = (C.c_void_p * len(covs))(*[c.handle.value for c in covs])
    cnt = np.zeros((len(covs), P), np.uint64)
    sm = None if a is None else np.zeros((len(covs), P), np.int64)
    _check(lib().sdb_join_aggregate_host(_np_ptr(x), _np_ptr(y), _np_ptr(a), len(x), arr,
                                         len(covs), lookup, _np_ptr(cnt), _np_ptr(sm),
                                         _stream(stream)))
    return cnt, sm


def join_aggregate_host_ptrs(x_ptr: int, y_ptr: int, attr_ptr: int | None, n: int, covs,
                             lookup: int, count_ptr: int, sum_ptr: int | None, stream=None):
    """sdb_join_aggregate_host on raw host pointers (e.g. pinned torch tensors)."""
    arr = (C.c_void_p * len(covs))(*[c.handle.value for c in covs])
    _check(lib().sdb_join_aggregate_host(C.c_void_p(x_ptr), C.c_void_p(y_ptr),
                                         C.c_void_p(attr_ptr) if attr_ptr else None, n, arr,
                                         len(covs), lookup, C.c_void_p(count_ptr),
                                         C.c_void_p(sum_ptr) if sum_ptr else None,
                                         _stream(stream)))


def join_aggregate_host_noalloc(x, y, attr, cov: Covering, lookup: int, stream=None):
    """sdb_join_aggregate_host_noalloc on numpy arrays: the host-buffer join for
    callers that cannot allocate device memory (see include/sdb.h); returns
    (count, sum) of shape (P,) as uint64 / int64 numpy arrays."""
    x = np.ascontiguousarray(x, np.uint32)
    y = np.ascontiguousarray(y, np.uint32)
    a = None if attr is None else np.ascontiguousarray(attr, np.int32)
    P = cov.info().n_polygons
    cnt = np.zeros(P, np.uint64)
    sm = None if a is None else np.zeros(P, np.int64)
    _check(lib().sdb_join_aggregate_host_noalloc(_np_ptr(x), _np_ptr(y), _np_ptr(a), len(x),
                                                 cov.handle, lookup, _np_ptr(cnt), _np_ptr(sm),
                                                 _stream(stream)))
    return cnt, sm


def covering_fallbacks(cov: Covering, stream=None) -> int:
    v = C.c_uint64()
    _check(lib().sdb_covering_fallbacks(cov.handle, _stream(stream), C.byref(v)))
    return v.value


def covering_index_stats(cov: Covering) -> tuple[float, int]:
    """(range-weighted mean window, max window) of the learned index."""
    m, x = C.c_double(), C.c_uint32()
    _check(lib().sdb_covering_index_stats(cov.handle, C.byref(m), C.byref(x)))
    return m.value, x.value


def covering_export(cov: Covering):
    """(start uint64[R+1], list_off uint32[R+1], list_ids uint32[nids])."""
    inf = cov.info()
    start = np.empty(inf.n_ranges + 1, np.uint64)
    loff = np.empty(inf.n_ranges + 1, np.uint32)
    ids = np.empty(max(inf.n_list_ids, 1), np.uint32)
    _check(lib().sdb_covering_export(cov.handle, _np_ptr(start), _np_ptr(loff), _np_ptr(ids)))
    return start, loff, ids[:inf.n_list_ids]


class _TraceStat(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("count", C.c_uint64), ("total_ms", C.c_double)]


def trace_enable(on: bool = True):
    """Start (dropping earlier records) or stop recording per-phase device time."""
    _check(lib().sdb_trace_enable(1 if on else 0))


def trace_read() -> dict:
    """{phase name: (intervals, total ms)} of the recorded phases."""
    n = C.c_uint32(0)
    _check(lib().sdb_trace_read(None, 0, C.byref(n)))
    buf = (_TraceStat * max(1, n.value))()
    _check(lib().sdb_trace_read(C.cast(buf, C.c_void_p), n.value, C.byref(n)))
    return {buf[i].name.decode(): (int(buf[i].count), float(buf[i].total_ms))
            for i in range(min(n.value, len(buf)))}


def memory_stats() -> tuple[int, int]:
    """(used, reserved) bytes of the library's device memory pool on the
    current device."""
    u, r = C.c_uint64(), C.c_uint64()
    _check(lib().sdb_memory_stats(C.byref(u), C.byref(r)))
    return int(u.value), int(r.value)


def launch_count() -> int:
    """Kernels launched by libsdb.so in this process so far."""
    return int(lib().sdb_launch_count())


class Points:
    """Resident, Hilbert-ordered point set (owns the library handle)."""

    def __init__(self, handle: int):
        self._h = C.c_void_p(handle)

    @property
    def handle(self):
        return self._h

    def free(self):
        if self._h and self._h.value:
            lib().sdb_points_free(self._h)
            self._h = C.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def points_create(x, y, attr, grid_bits: int, stream=None) -> Points:
    """sdb_points_create from device tensors (4-byte elements)."""
    out = C.c_void_p()
    _check(lib().sdb_points_create(_dptr(x, 4), _dptr(y, 4), _dptr(attr, 4), x.numel(), grid_bits,
                                   _stream(stream), C.byref(out)))
    return Points(out.value)


def points_build_index(pts: Points, radix_bits: int = 25, spline_error: int = 32, stream=None):
    """sdb_points_build_index: prefix sums + RadixSpline over the resident keys."""
    _check(lib().sdb_points_build_index(pts.handle, radix_bits, spline_error, _stream(stream)))


def points_aggregate(pts: Points, cov: Covering, lookup: int, count, sum_=None, stream=None):
    """sdb_points_aggregate into int64 device tensors of P entries."""
    _check(lib().sdb_points_aggregate(pts.handle, cov.handle, lookup, _dptr(count, 8),
                                      _dptr(sum_, 8), _stream(stream)))


def points_index_stats(pts: Points, stream=None):
    """(spline points, largest interpolation error, fallbacks of the last spline run)."""
    a, b, c = C.c_uint64(), C.c_uint64(), C.c_uint64()
    _check(lib().sdb_points_index_stats(pts.handle, C.byref(a), C.byref(b), C.byref(c),
                                        _stream(stream)))
    return a.value, b.value, c.value


class Batch:
    """Prepared batch of viewport queries (owns the library handle; keeps the
    point set it was built on alive)."""

    def __init__(self, handle: int, points: Points):
        self._h = C.c_void_p(handle)
        self.points = points

    @property
    def handle(self):
        return self._h

    def info(self) -> BatchInfo:
        inf = BatchInfo()
        _check(lib().sdb_batch_get_info(self._h, C.byref(inf)))
        return inf

    def query_ranges(self) -> np.ndarray:
        r = np.zeros(self.info().n_queries, np.uint32)
        _check(lib().sdb_batch_query_ranges(self._h, _np_ptr(r)))
        return r

    def free(self):
        if self._h and self._h.value:
            lib().sdb_batch_free(self._h)
            self._h = C.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def batch_create(points: Points, polys, queries, subset_ids, stream=None) -> Batch:
    """sdb_batch_create.  queries: a sequence of (x0, y0, x1, y1, eps, poly_off,
    poly_cnt) tuples or a numpy structured/2-D array with those columns."""
    off = np.ascontiguousarray(polys.ring_off, np.uint32)
    x = np.ascontiguousarray(polys.x, np.uint32)
    y = np.ascontiguousarray(polys.y, np.uint32)
    sp = _Polys(len(off) - 1, _np_ptr(off), _np_ptr(x), _np_ptr(y))
    qs = (Query * len(queries))(*[Query(*[int(v) for v in q]) for q in queries])
    ids = np.ascontiguousarray(subset_ids, np.uint32)
    out = C.c_void_p()
    _check(lib().sdb_batch_create(points.handle, C.byref(sp), qs, len(queries), _np_ptr(ids),
                                  len(ids), _stream(stream), C.byref(out)))
    return Batch(out.value, points)


def batch_run(batch: Batch, mode: int, count, sum_=None, stream=None):
    _check(lib().sdb_batch_run(batch.handle, mode, _dptr(count, 8), _dptr(sum_, 8),
                               _stream(stream)))


def batch_autotune(batch: Batch, stream=None) -> tuple[int, int]:
    t, p = C.c_uint32(), C.c_uint32()
    _check(lib().sdb_batch_autotune(batch.handle, _stream(stream), C.byref(t), C.byref(p)))
    return t.value, p.value


def batch_set_tuning(batch: Batch, tile: int, points_per_thread: int, stream=None):
    _check(lib().sdb_batch_set_tuning(batch.handle, tile, points_per_thread, _stream(stream)))


def batch_set_lookup(batch: Batch, lookup: int, stream=None):
    """sdb_batch_set_lookup: LOOKUP_BINARY or LOOKUP_LEARNED for later runs."""
    _check(lib().sdb_batch_set_lookup(batch.handle, lookup, _stream(stream)))


def batch_fallbacks(batch: Batch, stream=None) -> int:
    v = C.c_uint64()
    _check(lib().sdb_batch_fallbacks(batch.handle, _stream(stream), C.byref(v)))
    return int(v.value)


class Server:
    """Continuous-batching query server (owns the library handle)."""

    def __init__(self, handle: int, points: Points, P: int):
        self._h = C.c_void_p(handle)
        self.points = points
        self.n_polygons = P

    @staticmethod
    def prepare(query, subset_ids):
        """The marshalled arguments of one submit (the query record and its
        subset ids), for callers that submit at high rates."""
        ids = np.ascontiguousarray(subset_ids, np.uint32)
        q = Query(*[int(v) for v in query])
        q.poly_off = 0
        q.poly_cnt = len(ids)
        return (q, ids, C.byref(q), _np_ptr(ids))

    def submit_prepared(self, prep) -> int:
        """Queue a query marshalled by prepare(); returns a ticket."""
        t = C.c_uint64()
        _check(lib().sdb_server_submit(self._h, prep[2], prep[3], C.byref(t)))
        return t.value

    def submit(self, query, subset_ids) -> int:
        """Queue (x0, y0, x1, y1, eps, _, poly_cnt) with its subset ids; returns a ticket."""
        return self.submit_prepared(self.prepare(query, subset_ids))

    def wait(self, ticket: int, poly_cnt: int, timeout_ms: int = 60_000):
        """(count, sum, TicketInfo) of a ticket; raises SdbError(SDB_ETIMEOUT) on timeout."""
        cnt = np.zeros(max(poly_cnt, 1), np.uint64)
        sm = np.zeros(max(poly_cnt, 1), np.int64)
        info = TicketInfo()
        _check(lib().sdb_server_wait(self._h, ticket, timeout_ms, _np_ptr(cnt), _np_ptr(sm),
                                     C.byref(info)))
        return cnt[:poly_cnt], sm[:poly_cnt], info

    def stats(self) -> ServerStats:
        st = ServerStats()
        _check(lib().sdb_server_get_stats(self._h, C.byref(st)))
        return st

    def destroy(self):
        if self._h and self._h.value:
            lib().sdb_server_destroy(self._h)
            self._h = C.c_void_p(0)

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def server_create(points: Points, polys, *, workers=4, max_batch=256, cache_bytes=40 << 30,
                  use_cache=True, per_query=False, tile=0, points_per_thread=0,
                  lookup=LOOKUP_BINARY) -> Server:
    off = np.ascontiguousarray(polys.ring_off, np.uint32)
    x = np.ascontiguousarray(polys.x, np.uint32)
    y = np.ascontiguousarray(polys.y, np.uint32)
    sp = _Polys(len(off) - 1, _np_ptr(off), _np_ptr(x), _np_ptr(y))
    cfg = ServerConfig(workers, max_batch, cache_bytes, int(use_cache), int(per_query), tile,
                       points_per_thread, lookup)
    out = C.c_void_p()
    _check(lib().sdb_server_create(points.handle, C.byref(sp), C.byref(cfg), C.byref(out)))
    return Server(out.value, points, len(off) - 1)


def status_string(st: int) -> str:
    return lib().sdb_status_string(st).decode()
