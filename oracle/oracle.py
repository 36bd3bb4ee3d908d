"""ctypes wrapper around the C++ oracle (``sdb_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg use it; the CUDA library and its binding never do.

Every function here is argument marshalling; the arithmetic lives in the C++
file, which cites the paper section it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import platform
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sdb_oracle.cpp")
LIB = os.path.join(HERE, "liboracle.so")

HILBERT, ZORDER = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (g++, plain C++17)."""
    stamp = LIB + ".arch"
    arch = platform.machine()
    if not os.path.exists(stamp) or open(stamp).read().strip() != arch:
        force = True
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread",
                               SRC, "-o", tmp])
        os.replace(tmp, LIB)
        with open(stamp, "w") as f:
            f.write(arch)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        P, U32, U64, I64, I32 = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int64, C.c_int
        L.orc_finest_k.argtypes = [U64, U32, C.POINTER(C.c_uint32)]
        L.orc_finest_k.restype = I32
        L.orc_curve_many.argtypes = [I32, U32, U64, P, P, P]
        L.orc_classify_many.argtypes = [P, P, P, P, U32, U64, P, P, I64, P]
        L.orc_cover.argtypes = [U32, P, P, P, P, U32, U64, I32, I32]
        L.orc_cover.restype = P
        L.orc_cover_sizes.argtypes = [P, P, P, P, P, P]
        L.orc_cover_export.argtypes = [P, P, P, P]
        L.orc_cover_free.argtypes = [P]
        L.orc_join_o1.argtypes = [P, U64, P, P, P, P, P, P, P, P, I32]
        L.orc_join_o2.argtypes = [U32, P, P, P, P, U32, U64, U64, P, P, P, P, P, P, P, P, P,
                                  I64, I32, I32]
        L.orc_join_o2.restype = I32
        L.orc_point_index_aggregate.argtypes = [P, U64, P, P, P, P, P, I32]
        L.orc_join_exact.argtypes = [U32, P, P, P, P, U32, U64, P, P, P, P, P, P, I64, I32]
        L.orc_near_boundary.argtypes = [P, P, P, P, U32, U32, U32, U64]
        L.orc_near_boundary.restype = I32
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _u32(a):
    return np.ascontiguousarray(a, dtype=np.uint32)


def _shape(polys):
    """(n_polygons, poly_ring_off or None, ring_off, x, y) of a polygon set; a set
    with poly_ring_off holds polygons of several rings (outer rings and holes,
    even-odd region)."""
    pro = getattr(polys, "poly_ring_off", None)
    pro = None if pro is None else _u32(pro)
    return polys.n, pro, _u32(polys.ring_off), _u32(polys.x), _u32(polys.y)


def finest_k(eps: int, grid_bits: int):
    """(k, F) with finest side 2^k and finest level F = B - k, or None if eps < sqrt(2)."""
    k = C.c_uint32()
    if lib().orc_finest_k(int(eps), int(grid_bits), C.byref(k)) != 0:
        return None
    return k.value, grid_bits - k.value


def curve(order: int, x, y, which: int = HILBERT) -> np.ndarray:
    x, y = _u32(x), _u32(y)
    out = np.empty(len(x), np.uint64)
    lib().orc_curve_many(which, order, len(x), _p(x), _p(y), _p(out))
    return out


def classify(polys, j: int, x0, y0, side: int) -> np.ndarray:
    """0 exterior / 1 interior / 2 boundary for closed squares against polygon j."""
    x0 = np.ascontiguousarray(x0, np.int64)
    y0 = np.ascontiguousarray(y0, np.int64)
    out = np.empty(len(x0), np.uint8)
    _, pro, off, vx, vy = _shape(polys)
    lib().orc_classify_many(_p(pro), _p(off), _p(vx), _p(vy), j, len(x0), _p(x0), _p(y0), side,
                            _p(out))
    return out


@dataclass
class Covering:
    start: np.ndarray     # uint64 [R+1]
    list_off: np.ndarray  # uint32 [R+1]
    list_ids: np.ndarray  # uint32
    n_records: int
    F: int
    k: int
    grid_bits: int
    n_polygons: int
    which: int
    flagged: bool = False
    _h: int = 0

    @property
    def R(self) -> int:
        return len(self.start) - 1

    def free(self):
        if self._h:
            lib().orc_cover_free(self._h)
            self._h = 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def join(self, x, y, attr=None):
        """O1: per-point ordered lookup in the canonical covering."""
        x, y = _u32(x), _u32(y)
        a = None if attr is None else np.ascontiguousarray(attr, np.int32)
        cnt = np.zeros(self.n_polygons, np.uint64)
        sm = np.zeros(self.n_polygons, np.int64)
        lib().orc_join_o1(self._h, len(x), _p(x), _p(y), _p(a), _p(cnt), _p(sm), None, None,
                          None, self.which)
        return cnt, sm

    def point_index_aggregate(self, x, y, attr=None):
        """Sec. 3 point indexing: sorted full-resolution keys + prefix sums,
        two lower bounds per covering range.  Equals join() exactly."""
        x, y = _u32(x), _u32(y)
        a = None if attr is None else np.ascontiguousarray(attr, np.int32)
        cnt = np.zeros(self.n_polygons, np.uint64)
        sm = np.zeros(self.n_polygons, np.int64)
        lib().orc_point_index_aggregate(self._h, len(x), _p(x), _p(y), _p(a), _p(cnt), _p(sm),
                                        self.which)
        return cnt, sm

    def join_range(self, x, y, attr=None):
        """O1 on a flagged covering (Sec. 6): (count, sum, bcount, bsum, babs)."""
        x, y = _u32(x), _u32(y)
        a = None if attr is None else np.ascontiguousarray(attr, np.int32)
        P = self.n_polygons
        out = [np.zeros(P, np.uint64), np.zeros(P, np.int64), np.zeros(P, np.uint64),
               np.zeros(P, np.int64), np.zeros(P, np.uint64)]
        lib().orc_join_o1(self._h, len(x), _p(x), _p(y), _p(a), *[_p(o) for o in out], self.which)
        return tuple(out)


def cover(polys, eps: int, which: int = HILBERT, grid_bits: int | None = None,
          flagged: bool = False, noncons: bool = False) -> Covering:
    """O1: recursive quadtree covering of every polygon, swept into canonical ranges
    (flagged: list entries carry bit 31 on boundary cells, Sec. 6; noncons: a
    finest boundary cell is kept only when its centre is in the polygon, Sec. 2.2)."""
    B = polys.grid_bits if grid_bits is None else grid_bits
    P, pro, off, vx, vy = _shape(polys)
    h = lib().orc_cover(P, _p(pro), _p(off), _p(vx), _p(vy), B, int(eps), which,
                        int(flagged) | (2 if noncons else 0))
    if not h:
        raise ValueError("invalid covering arguments")
    R, nids, nrec = C.c_uint64(), C.c_uint64(), C.c_uint64()
    F, k = C.c_uint32(), C.c_uint32()
    lib().orc_cover_sizes(h, C.byref(R), C.byref(nids), C.byref(nrec), C.byref(F), C.byref(k))
    start = np.empty(R.value + 1, np.uint64)
    loff = np.empty(R.value + 1, np.uint32)
    ids = np.empty(nids.value, np.uint32)
    lib().orc_cover_export(h, _p(start), _p(loff), _p(ids))
    return Covering(start, loff, ids, nrec.value, F.value, k.value, B, P, which,
                    bool(flagged), h)


def join_o2(polys, eps: int, pts, *, threads: int = 1, member: bool = False, only: int = -1,
            grid_bits: int | None = None, boundary_sums: bool = False, noncons: bool = False):
    """O2: per point, the definitional test 'closed finest cell meets closed polygon'.

    Returns (count, sum, boundary_count[, boundary_sum, boundary_abs][, member])."""
    B = polys.grid_bits if grid_bits is None else grid_bits
    P = polys.n
    x, y = _u32(pts.x), _u32(pts.y)
    a = None if pts.attr is None else np.ascontiguousarray(pts.attr, np.int32)
    cnt = np.zeros(P, np.uint64)
    sm = np.zeros(P, np.int64)
    bnd = np.zeros(P, np.uint64)
    bs = np.zeros(P, np.int64) if boundary_sums else None
    ba = np.zeros(P, np.uint64) if boundary_sums else None
    mem = np.zeros(len(x), np.uint8) if member else None
    _, pro, off, vx, vy = _shape(polys)
    rc = lib().orc_join_o2(P, _p(pro), _p(off), _p(vx), _p(vy), B,
                           int(eps), len(x), _p(x), _p(y), _p(a), _p(cnt), _p(sm), _p(bnd),
                           _p(bs), _p(ba), _p(mem), only, threads, 2 if noncons else 0)
    if rc != 0:
        raise ValueError("invalid O2 arguments")
    out = (cnt, sm, bnd) + ((bs, ba) if boundary_sums else ())
    return out + (mem,) if member else out


def range_bounds(count, sm, bcount, bsum, babs):
    """Sec. 6 on a conservative covering: the exact COUNT lies in
    [count - bcount, count]; the exact SUM is sum minus the attribute sum of the
    false positives, a subset of the boundary points, so it lies in
    [sum - pos, sum - neg] with pos = (babs + bsum) / 2 >= 0 and
    neg = (bsum - babs) / 2 <= 0 (the boundary points' positive and negative parts)."""
    count, sm = np.asarray(count, np.int64), np.asarray(sm, np.int64)
    bcount, bsum, babs = (np.asarray(bcount, np.int64), np.asarray(bsum, np.int64),
                          np.asarray(babs, np.int64))
    pos, neg = (babs + bsum) // 2, (bsum - babs) // 2
    return count - bcount, count, sm - pos, sm - neg


def join_exact(polys, pts, *, threads: int = 1, member: bool = False, only: int = -1):
    """Exact closed point-in-polygon join (points on the boundary count)."""
    P = polys.n
    x, y = _u32(pts.x), _u32(pts.y)
    a = None if pts.attr is None else np.ascontiguousarray(pts.attr, np.int32)
    cnt = np.zeros(P, np.uint64)
    sm = np.zeros(P, np.int64)
    mem = np.zeros(len(x), np.uint8) if member else None
    _, pro, off, vx, vy = _shape(polys)
    lib().orc_join_exact(P, _p(pro), _p(off), _p(vx), _p(vy),
                         polys.grid_bits, len(x), _p(x), _p(y), _p(a), _p(cnt), _p(sm), _p(mem),
                         only, threads)
    return (cnt, sm, mem) if member else (cnt, sm)


def near_boundary(polys, j: int, px: int, py: int, eps: int) -> bool:
    """Exact: is (px, py) within distance eps of polygon j's boundary?"""
    _, pro, off, vx, vy = _shape(polys)
    return bool(lib().orc_near_boundary(_p(pro), _p(off), _p(vx), _p(vy), j, int(px), int(py),
                                        int(eps)))
