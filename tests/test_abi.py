"""Host-side checks of the C ABI: every declared entry point is exported, and
argument validation answers with status codes before touching the GPU."""
import ctypes as C
import os
import re

import numpy as np

from paper_2010_12548_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(sdb_[a-z0-9_]+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(sdblib):
    names = declared()
    assert len(names) >= 10
    L = sdblib.lib()
    for n in sorted(names):
        assert hasattr(L, n), n


def test_finest_level_matches_oracle(sdblib, orc):
    rng = np.random.default_rng(1)
    for B in (1, 4, 16, 24, 28, 30):
        for eps in [2, 3, 4, 5, 45, 46, 64, 4096] + list(rng.integers(2, 2 ** 33, 50)):
            k, F = sdblib.finest_level(B, int(eps))
            ko, Fo = orc.finest_k(int(eps), B)
            assert (k, F) == (ko, Fo), (B, eps)


def _status(sdblib, fn, *args):
    return getattr(sdblib.lib(), fn)(*args)


def test_invalid_arguments_rejected_on_host(sdblib):
    L = sdblib.lib()
    k, F = C.c_uint32(), C.c_uint32()
    assert L.sdb_finest_level(0, 64, C.byref(k), C.byref(F)) == sdblib.SDB_EINVAL
    assert L.sdb_finest_level(31, 64, C.byref(k), C.byref(F)) == sdblib.SDB_EINVAL
    assert L.sdb_finest_level(16, 1, C.byref(k), C.byref(F)) == sdblib.SDB_EINVAL
    assert b"eps" in L.sdb_last_error()

    def build(off, x, y, B=8, eps=4):
        P = W.Polygons(np.array(off, np.uint32), np.array(x, np.uint32), np.array(y, np.uint32), B)
        try:
            sdblib.build_covering(P, B, eps, stream=0)
        except sdblib.SdbError as e:
            return e.status, str(e)
        return 0, ""

    st, msg = build([0, 2], [1, 2], [1, 2])
    assert st == sdblib.SDB_EINVAL and "fewer than 3" in msg
    st, msg = build([0, 3], [1, 2, 300], [1, 2, 3])
    assert st == sdblib.SDB_EINVAL and "outside the grid" in msg
    st, msg = build([0, 3], [1, 2, 3], [1, 5, 3], eps=1)
    assert st == sdblib.SDB_EINVAL
    st, msg = build([0, 3], [1, 2, 3], [1, 5, 3], B=31)
    assert st == sdblib.SDB_EINVAL
    st, msg = build([1, 4], [1, 2, 3, 4], [1, 5, 3, 4])
    assert st == sdblib.SDB_EINVAL
    assert L.sdb_build_covering(None, 8, 4, None, None) == sdblib.SDB_EINVAL
    out = C.c_void_p()
    assert L.sdb_build_covering_ex(None, 8, 4, 4, None, C.byref(out)) == sdblib.SDB_EINVAL
    assert b"flags" in L.sdb_last_error()
    assert L.sdb_build_covering_ex(None, 8, 4, 3, None, C.byref(out)) == sdblib.SDB_EINVAL
    assert b"conservative" in L.sdb_last_error()
    assert L.sdb_build_covering_multi(None, 8, 4, 0, None, C.byref(out)) == sdblib.SDB_EINVAL
    assert L.sdb_join_aggregate_range(None, None, None, 0, None, 0, None, None, None, None, None,
                                      None) == sdblib.SDB_EINVAL
    assert L.sdb_join_aggregate(None, None, None, 0, None, 0, None, None, None) == sdblib.SDB_EINVAL
    assert L.sdb_covering_build_index(None, 12, None) == sdblib.SDB_EINVAL
    assert L.sdb_covering_build_index_ex(None, 12, 0, None) == sdblib.SDB_EINVAL
    assert L.sdb_covering_build_table(None, 20, None) == sdblib.SDB_EINVAL
    assert L.sdb_trace_read(None, 0, None) == sdblib.SDB_EINVAL
    # tracing with nothing recorded needs no device
    sdblib.trace_enable(True)
    assert sdblib.trace_read() == {}
    sdblib.trace_enable(False)
    assert L.sdb_join_aggregate_host(None, None, None, 0, None, 0, 0, None, None, None) == \
        sdblib.SDB_EINVAL
    for s in range(6):
        assert sdblib.status_string(s)
    L.sdb_covering_free(None)
