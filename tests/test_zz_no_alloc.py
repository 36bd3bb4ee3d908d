"""The allocation-free host-buffer join (sdb_join_aggregate_host_noalloc).

It serves callers that cannot allocate device memory while calling in
(services that reserve their whole memory budget when they start, plugins in a
process whose own allocator owns the device).  Its results must equal the
regular host-buffer entry point's, bit for bit, on consecutive calls that reuse
the same fixed device array, for every covering lookup; and once the first call
has set the array up, further calls must leave the device's free memory and the
library's memory pool untouched.  This file is collected last.
"""
import numpy as np
import pytest

from paper_2010_12548_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_join_matches_host_join(cuda, sdblib):
    # more points than one staging chunk (2^20), so the chunk loop is exercised
    w = W.tiny_stars(2_500_003)
    cov = sdblib.build_covering(w.polygons, w.grid_bits, w.eps[0])
    sdblib.covering_build_index(cov, 8)
    sdblib.covering_build_table(cov, 12)
    lookups = (sdblib.LOOKUP_BINARY, sdblib.LOOKUP_LEARNED, sdblib.LOOKUP_TABLE)
    half = w.points.n // 2
    want = {}
    for lookup in lookups:
        c, s = sdblib.join_aggregate_host(w.points.x, w.points.y, w.points.attr, [cov], lookup)
        ch, _ = sdblib.join_aggregate_host(w.points.x[:half], w.points.y[:half], None, [cov],
                                           lookup)
        want[lookup] = (c[0], s[0], ch[0])
    # the first call on the device sets the fixed array up (and loads the
    # kernels); after it nothing may be allocated
    sdblib.join_aggregate_host_noalloc(w.points.x[:10], w.points.y[:10], w.points.attr[:10], cov,
                                       sdblib.LOOKUP_BINARY)
    cuda.cuda.synchronize()
    free0 = cuda.cuda.mem_get_info()[0]
    pool0 = sdblib.memory_stats()
    for lookup in lookups:
        want_c, want_s, want_half = want[lookup]
        for _ in range(2):  # the array keeps the previous call's contents
            got_c, got_s = sdblib.join_aggregate_host_noalloc(w.points.x, w.points.y,
                                                              w.points.attr, cov, lookup)
            assert np.array_equal(got_c, want_c) and np.array_equal(got_s, want_s)
        # count only, on a different number of points
        got_c, _ = sdblib.join_aggregate_host_noalloc(w.points.x[:half], w.points.y[:half], None,
                                                      cov, lookup)
        assert np.array_equal(got_c, want_half)
    cuda.cuda.synchronize()
    assert cuda.cuda.mem_get_info()[0] == free0
    assert sdblib.memory_stats() == pool0


def test_noalloc_rejects_too_many_polygons(cuda, sdblib):
    n = 65_537  # one more than the fixed maximum
    k = np.arange(n, dtype=np.uint32)
    cx, cy = (k % 512) * 8, (k // 512) * 8
    x = np.stack([cx, cx + 4, cx], 1).ravel()
    y = np.stack([cy, cy, cy + 4], 1).ravel()
    P = W.Polygons(np.arange(0, 3 * n + 1, 3, dtype=np.uint32), x, y, 12)
    cov = sdblib.build_covering(P, 12, 2 ** 13)
    with pytest.raises(sdblib.SdbError) as e:
        sdblib.join_aggregate_host_noalloc(np.zeros(4, np.uint32), np.zeros(4, np.uint32),
                                           None, cov, sdblib.LOOKUP_BINARY)
    assert e.value.status == sdblib.SDB_EINVAL and "maximum" in str(e.value)
