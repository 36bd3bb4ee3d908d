"""The large learned-index configuration at full size.

1B points on [0,2^28)^2 (70% from 64 Gaussian clusters, 30% uniform, fare
attributes), the 40,000-cell jittered Voronoi tiling, and the finest eps a
single covering build reaches on it (2^9: about 2.1e9 raster cells and 5.3e8
ranges; eps = 2^5 would need about 3.4e10).  In the launches the benchmark
times (all 1B points at once):

* binary search, the learned index alone (2^16 leaves under one root line), the cell table and the
  table + learned lookup give identical per-polygon COUNT and SUM, with no
  learned fallback;
* every point is counted at least once (the polygons tile the whole grid);
* per polygon, the counts at eps 2^9 are at most those at eps 2^10 (the finer
  raster's cells nest inside the coarser one's);
* on a fixed 2M-point sample the results equal the oracle's definitional test;
* tiled by the 32 x 32 quadtree cells of level 5 (viewport queries over the
  Hilbert-ordered resident points, 32 tiles a batch), the per-polygon sums of
  the tiles' answers equal the single covering's join at eps 2^9 over all 1B
  points, and at eps 2^5 itself equal the definitional test on the sample.
"""
import os

import numpy as np
import pytest

from paper_2010_12548_gb300 import workloads as W

pytestmark = pytest.mark.gpu

import bench  # noqa: E402  (the benchmark's leaf and table bits, its eps sweep)

N = 1_000_000_000


def dev(torch, a):
    a = np.ascontiguousarray(a)
    return torch.from_numpy(a.view(np.int32) if a.dtype.itemsize == 4 else a).cuda()


def join(torch, sdb, cov, x, y, a, lookup, P):
    cnt = torch.full((P,), 7, dtype=torch.int64, device="cuda")
    sm = torch.full((P,), 7, dtype=torch.int64, device="cuda")
    sdb.join_aggregate(x, y, a, cov, lookup, cnt, sm)
    torch.cuda.synchronize()
    return cnt.cpu().numpy().view(np.uint64), sm.cpu().numpy()


def test_config3_full_size(cuda, sdblib, orc):
    torch = cuda
    T = W.tracts40k_tiling()
    pts = W.resident_points(N)
    P = T.n
    x, y, a = dev(torch, pts.x), dev(torch, pts.y), dev(torch, pts.attr)
    eps = bench.C3_EPS_SWEEP[-1]
    cov = sdblib.build_covering(T, 28, eps)
    inf = cov.info()
    assert inf.n_cells > 2_000_000_000 and inf.n_ranges > 500_000_000
    sdblib.covering_build_table(cov, bench.TABLE_BITS)
    sdblib.covering_build_index(cov, bench.LEAF_BITS, root_bits=bench.LEAF_ROOT_BITS)
    ref = join(torch, sdblib, cov, x, y, a, sdblib.LOOKUP_BINARY, P)
    assert int(ref[0].sum()) >= N
    for lookup in (sdblib.LOOKUP_LEARNED, sdblib.LOOKUP_TABLE, sdblib.LOOKUP_TABLE_LEARNED):
        got = join(torch, sdblib, cov, x, y, a, lookup, P)
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), lookup
        if lookup != sdblib.LOOKUP_TABLE:
            assert sdblib.covering_fallbacks(cov) == 0, lookup
    # the sample against the definitional test
    idx = np.arange(0, N, N // 2_000_000)
    sp = pts.take(idx)
    sx, sy, sa = dev(torch, sp.x), dev(torch, sp.y), dev(torch, sp.attr)
    want_c, want_s, _ = orc.join_o2(T, eps, sp, threads=os.cpu_count() or 1)
    for lookup in (sdblib.LOOKUP_BINARY, sdblib.LOOKUP_TABLE_LEARNED):
        got = join(torch, sdblib, cov, sx, sy, sa, lookup, P)
        assert np.array_equal(got[0], want_c) and np.array_equal(got[1], want_s), lookup
    cov.free()
    # nesting against the next coarser eps
    coarse = sdblib.build_covering(T, 28, 2 * eps)
    sdblib.covering_build_table(coarse, bench.TABLE_BITS)
    cc = join(torch, sdblib, coarse, x, y, a, sdblib.LOOKUP_TABLE, P)
    assert (ref[0] <= cc[0]).all()
    coarse.free()
    # tiled: the tiles' answers add up to the single covering's at eps 2^9 ...
    p = sdblib.points_create(x, y, a, 28)
    qb = W.tile_queries(T, 28, bench.C3_TILE_LEVEL, eps)
    lks = (sdblib.LOOKUP_LEARNED, sdblib.LOOKUP_BINARY)
    tot, st = bench.tiled_join(sdblib, torch, torch.device("cuda"), None, T, p, qb, lks,
                               timing=False)
    p.free()
    assert st["fallbacks"] == 0
    for lk in lks:
        assert np.array_equal(tot[lk][0].cpu().numpy().view(np.uint64), ref[0]), lk
        assert np.array_equal(tot[lk][1].cpu().numpy(), ref[1]), lk
    # ... and at eps 2^5 equal the definitional test on the sample
    e5 = bench.C3_TILED_EPS
    sp5 = sdblib.points_create(sx, sy, sa, 28)
    qb5 = W.tile_queries(T, 28, bench.C3_TILE_LEVEL, e5)
    tot5, _ = bench.tiled_join(sdblib, torch, torch.device("cuda"), None, T, sp5, qb5, lks,
                               timing=False)
    want_c, want_s, _ = orc.join_o2(T, e5, sp, threads=os.cpu_count() or 1)
    for lk in lks:
        assert np.array_equal(tot5[lk][0].cpu().numpy().view(np.uint64), want_c), lk
        assert np.array_equal(tot5[lk][1].cpu().numpy(), want_s), lk
