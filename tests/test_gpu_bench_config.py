"""Parity of the configuration the benchmark times.

The benchmark builds the 263-zone tiling's coverings for the whole eps sweep
{2^12, 2^10, 2^8, 2^6} in one pass (sdb_build_coverings: four queries, about
117M packed records, 40-bit keys) and joins 100M mobility points against each
with the learned lookup (cell table of 2^22 buckets in front of a learned
index of 2^16 leaves under one root line).  Here, on exactly those inputs and in exactly those
launches:

* every swept covering equals the covering built for its eps alone, entry for
  entry;
* on a fixed 4M-point sample of the benchmark's points every lookup (binary
  search, learned index, cell table, table + learned) on every swept covering
  equals the oracle's definitional test (O2) per polygon, COUNT and SUM;
* on all 100M points the four lookups give identical results with no learned
  fallback, and the per-polygon counts add up to the points the covering can
  hold (every point of the square grid lies in at least one zone).
"""
import os

import numpy as np
import pytest

from paper_2010_12548_gb300 import workloads as W

pytestmark = pytest.mark.gpu

import bench  # noqa: E402  (the benchmark's own constants: leaf and table bits)


def dev(torch, a):
    a = np.ascontiguousarray(a)
    return torch.from_numpy(a.view(np.int32) if a.dtype.itemsize == 4 else a).cuda()


@pytest.fixture(scope="module")
def timed(cuda, sdblib):
    """The benchmark's workload and its swept coverings, with every lookup
    structure built as the benchmark builds it."""
    w = W.mobility_zones(100_000_000)
    covs = sdblib.build_coverings(w.polygons, 24, w.eps)
    for c in covs:
        sdblib.covering_build_table(c, bench.TABLE_BITS)
        sdblib.covering_build_index(c, bench.LEAF_BITS, root_bits=bench.LEAF_ROOT_BITS)
    return w, covs


def lookups(sdb):
    return (sdb.LOOKUP_BINARY, sdb.LOOKUP_LEARNED, sdb.LOOKUP_TABLE, sdb.LOOKUP_TABLE_LEARNED)


def join(torch, sdb, cov, x, y, a, lookup, P):
    cnt = torch.full((P,), 7, dtype=torch.int64, device="cuda")
    sm = torch.full((P,), 7, dtype=torch.int64, device="cuda")
    sdb.join_aggregate(x, y, a, cov, lookup, cnt, sm)
    torch.cuda.synchronize()
    return cnt.cpu().numpy().view(np.uint64), sm.cpu().numpy()


def test_sweep_equals_single_builds(cuda, sdblib, timed):
    w, covs = timed
    assert sum(c.info().n_cells for c in covs) > 100_000_000  # the sweep's record count
    for c, eps in zip(covs, w.eps):
        one = sdblib.build_covering(w.polygons, 24, eps)
        for a, b in zip(sdblib.covering_export(c), sdblib.covering_export(one)):
            assert np.array_equal(a, b), eps
        ia, ib = c.info(), one.info()
        assert (ia.n_ranges, ia.n_list_ids, ia.n_cells) == (ib.n_ranges, ib.n_list_ids,
                                                            ib.n_cells), eps
        one.free()


def test_sampled_points_vs_definitional_oracle(cuda, sdblib, orc, timed):
    torch = cuda
    w, covs = timed
    P = w.polygons.n
    idx = np.arange(0, w.points.n, 25)  # a fixed 4M-point sample
    pts = w.points.take(idx)
    x, y, a = dev(torch, pts.x), dev(torch, pts.y), dev(torch, pts.attr)
    threads = os.cpu_count() or 1
    for c, eps in zip(covs, w.eps):
        want_c, want_s, _ = orc.join_o2(w.polygons, eps, pts, threads=threads)
        for lookup in lookups(sdblib):
            got_c, got_s = join(torch, sdblib, c, x, y, a, lookup, P)
            assert np.array_equal(got_c, want_c), (eps, lookup)
            assert np.array_equal(got_s, want_s), (eps, lookup)


def test_full_size_lookups_agree(cuda, sdblib, timed):
    torch = cuda
    w, covs = timed
    P = w.polygons.n
    x, y, a = dev(torch, w.points.x), dev(torch, w.points.y), dev(torch, w.points.attr)
    for c, eps in zip(covs, w.eps):
        ref = join(torch, sdblib, c, x, y, a, sdblib.LOOKUP_BINARY, P)
        # a tiling of the whole grid: every point is counted at least once
        assert int(ref[0].sum()) >= w.points.n
        for lookup in lookups(sdblib)[1:]:
            got = join(torch, sdblib, c, x, y, a, lookup, P)
            assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), (eps,
                                                                                      lookup)
            if lookup in (sdblib.LOOKUP_LEARNED, sdblib.LOOKUP_TABLE_LEARNED):
                assert sdblib.covering_fallbacks(c) == 0, (eps, lookup)
