"""The cell-table lookup (a direct-mapped first level over the finest cell ids,
the role of ACT's upper levels in Sec. 3) vs the CPU oracle.

The table only changes how a point's range is found, so every join through it
must equal the oracle's O1 join bit for bit: coarse tables (most buckets meet
several ranges, so most points go through the per-warp queue), fine tables (one
id per bucket, no mixed bucket), both aggregation paths, COUNT only, the
result-range join, the host-buffer joins, and the full-size workload against
the other lookups.  Every case runs twice: with a binary search inside mixed
buckets (LOOKUP_TABLE) and with the learned index's window cut to the bucket's
(LOOKUP_TABLE_LEARNED), which must also report no fallback.
"""
import numpy as np
import pytest

from paper_2010_12548_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TABLE = 3  # LOOKUP_TABLE
TABLE_LEARNED = 4  # LOOKUP_TABLE_LEARNED
LOOKUPS = (TABLE, TABLE_LEARNED)


def build_table(sdb, cov, bits, lookup, leaf_bits=8):
    """The cell table, plus the learned index the second lookup needs."""
    sdb.covering_build_table(cov, bits)
    if lookup == TABLE_LEARNED:
        sdb.covering_build_index(cov, leaf_bits)


def no_fallback(sdb, cov, lookup):
    if lookup == TABLE_LEARNED:
        assert sdb.covering_fallbacks(cov) == 0


def dev(torch, a):
    a = np.ascontiguousarray(a)
    return torch.from_numpy(a.view(np.int32) if a.dtype.itemsize == 4 else a).cuda()


def join(torch, sdb, cov, pts, lookup=TABLE, with_sum=True, x=None, y=None, a=None):
    P = cov.info().n_polygons
    x = dev(torch, pts.x) if x is None else x
    y = dev(torch, pts.y) if y is None else y
    a = (dev(torch, pts.attr) if a is None else a) if with_sum else None
    cnt = torch.full((P,), 7, dtype=torch.int64, device="cuda")  # the call zeroes it
    sm = torch.full((P,), 7, dtype=torch.int64, device="cuda") if with_sum else None
    sdb.join_aggregate(x, y, a, cov, lookup, cnt, sm)
    torch.cuda.synchronize()
    return cnt.cpu().numpy().view(np.uint64), (sm.cpu().numpy() if with_sum else None)


def signed_points(seed, n, B):
    rng = np.random.default_rng(seed)
    a = rng.integers(-2 ** 31, 2 ** 31, n, dtype=np.int64).astype(np.int32)
    a[:3] = [-2 ** 31, 2 ** 31 - 1, 0]
    return W.Points(rng.integers(0, 2 ** B, n, dtype=np.uint32),
                    rng.integers(0, 2 ** B, n, dtype=np.uint32), a, B)


@pytest.mark.parametrize("lookup", LOOKUPS)
@pytest.mark.parametrize("B,eps,seed", [(8, 3, 1), (10, 2, 2), (12, 9, 3), (16, 64, 4),
                                        (16, 700, 5), (12, 2 ** 13, 6), (20, 40, 7)])
def test_table_stars_vs_oracle(cuda, sdblib, orc, B, eps, seed, lookup):
    """Overlapping stars (lists of several polygons), tables from 2^8 buckets
    to one id per bucket; extreme attributes stress the packed accumulators."""
    rng = np.random.default_rng(seed)
    G = 2 ** B
    P = W.star_polygons(rng, 9, B, nverts=(3, 16), radius=(G / 16, G / 4))
    oc = orc.cover(P, eps)
    cov = sdblib.build_covering(P, B, eps)
    pts = signed_points(seed, 50_021, B)
    pts.x[::101] = G + 3  # outside the grid
    want = oc.join(pts.x, pts.y, pts.attr)
    for tb in sorted({8, 11, 16, 2 * oc.F, 26}):
        if tb < 8 or tb > 26:
            continue
        build_table(sdblib, cov, tb, lookup, leaf_bits=4 + tb % 9)
        inf = cov.info()
        assert inf.table_bits == min(tb & ~1, 2 * oc.F)  # whole levels
        if inf.table_bits == 2 * oc.F:
            assert inf.table_mixed == 0  # one id per bucket
        cnt, sm = join(cuda, sdblib, cov, pts, lookup)
        assert np.array_equal(cnt, want[0]) and np.array_equal(sm, want[1]), tb
        no_fallback(sdblib, cov, lookup)
        cnt, _ = join(cuda, sdblib, cov, pts, lookup, with_sum=False)
        assert np.array_equal(cnt, want[0]), tb


@pytest.mark.parametrize("lookup", LOOKUPS)
def test_table_mostly_mixed(cuda, sdblib, orc, lookup):
    """A 2^8-bucket table over many small polygons: nearly every point lies in
    a mixed bucket, so the per-warp queues fill and drain on every tile."""
    rng = np.random.default_rng(11)
    P = W.star_polygons(rng, 400, 16, nverts=(3, 10), radius=(300, 1500))
    oc = orc.cover(P, 20)
    cov = sdblib.build_covering(P, 16, 20)
    build_table(sdblib, cov, 8, lookup, leaf_bits=12)
    assert cov.info().table_mixed >= 150
    pts = signed_points(12, 300_007, 16)
    want = oc.join(pts.x, pts.y, pts.attr)
    cnt, sm = join(cuda, sdblib, cov, pts, lookup)
    assert np.array_equal(cnt, want[0]) and np.array_equal(sm, want[1])
    no_fallback(sdblib, cov, lookup)
    # every point on one vertex (a boundary cell, in a mixed bucket): all lanes
    # queue and add to the same accumulators, at the extreme attribute
    vx, vy = int(P.x[P.ring_off[0]]), int(P.y[P.ring_off[0]])
    one = W.Points(np.full(200_000, vx, np.uint32), np.full(200_000, vy, np.uint32),
                   np.full(200_000, -2 ** 31, np.int32), 16)
    want = oc.join(one.x, one.y, one.attr)
    assert want[0][0] == 200_000
    cnt, sm = join(cuda, sdblib, cov, one, lookup)
    assert np.array_equal(cnt, want[0]) and np.array_equal(sm, want[1])
    one.attr[:] = 2 ** 31 - 1
    want = oc.join(one.x, one.y, one.attr)
    cnt, sm = join(cuda, sdblib, cov, one, lookup)
    assert np.array_equal(cnt, want[0]) and np.array_equal(sm, want[1])


def test_table_zones(cuda, sdblib, orc):
    """The 263-zone tiling at eps 2^12 and 2^10, 1M mobility points."""
    T = W.zones263_tiling()
    pts = W.mobility_points(W.BASE_SEED + 7, 1_000_003, 24, 32)
    for eps in (2 ** 12, 2 ** 10):
        oc = orc.cover(T, eps)
        cov = sdblib.build_covering(T, 24, eps)
        want = oc.join(pts.x, pts.y, pts.attr)
        for tb in (10, 16, 22):
            for lookup, lb in ((TABLE, 0), (TABLE_LEARNED, 12), (TABLE_LEARNED, 16)):
                build_table(sdblib, cov, tb, lookup, leaf_bits=lb)
                cnt, sm = join(cuda, sdblib, cov, pts, lookup)
                assert np.array_equal(cnt, want[0]) and np.array_equal(sm, want[1]), (eps, tb, lb)
                no_fallback(sdblib, cov, lookup)


@pytest.mark.parametrize("lookup", LOOKUPS)
def test_table_edge_cases_and_errors(cuda, sdblib, orc, lookup):
    torch = cuda
    TABLE = lookup  # noqa: N806  (every call below goes through this lookup)
    B, eps = 12, 9
    rng = np.random.default_rng(77)
    P = W.star_polygons(rng, 9, B, nverts=(3, 12), radius=(256, 800))
    oc = orc.cover(P, eps)
    cov = sdblib.build_covering(P, B, eps)
    build_table(sdblib, cov, 10, lookup, leaf_bits=5)
    base = signed_points(3, 5000, B)
    base.x[::97] = 2 ** B + 5
    base.y[::89] = 2 ** 31
    for n in (0, 1, 2, 3, 4, 5, 31, 32, 33, 127, 128, 129, 1003, 5000):
        pts = base.take(np.arange(n))
        want = oc.join(pts.x, pts.y, pts.attr)
        cnt, sm = join(torch, sdblib, cov, pts, lookup)
        assert np.array_equal(cnt, want[0]) and np.array_equal(sm, want[1]), n
    # unaligned device pointers take the scalar path
    x = dev(torch, np.concatenate([[0], base.x]).astype(np.uint32))[1:]
    y = dev(torch, np.concatenate([[0], base.y]).astype(np.uint32))[1:]
    a = dev(torch, np.concatenate([[0], base.attr]).astype(np.int32))[1:]
    want = oc.join(base.x, base.y, base.attr)
    cnt, sm = join(torch, sdblib, cov, base, lookup, x=x, y=y, a=a)
    assert np.array_equal(cnt, want[0]) and np.array_equal(sm, want[1])
    # the finest level 0: one cell, one bucket
    big = sdblib.build_covering(P, B, 2 ** 13)
    build_table(sdblib, big, 8, lookup, leaf_bits=4)
    assert big.info().table_bits == 0
    want = orc.cover(P, 2 ** 13).join(base.x, base.y, base.attr)
    cnt, sm = join(torch, sdblib, big, base, lookup)
    assert np.array_equal(cnt, want[0]) and np.array_equal(sm, want[1])
    # the host-buffer joins
    cnt, sm = sdblib.join_aggregate_host(base.x, base.y, base.attr, [cov, big], TABLE)
    assert np.array_equal(cnt[1], want[0]) and np.array_equal(sm[1], want[1])
    cnt, sm = sdblib.join_aggregate_host_noalloc(base.x, base.y, base.attr, cov, TABLE)
    w2 = oc.join(base.x, base.y, base.attr)
    assert np.array_equal(cnt, w2[0]) and np.array_equal(sm, w2[1])
    # argument errors are caught on the host
    z = torch.zeros(P.n, dtype=torch.int64, device="cuda")
    fresh = sdblib.build_covering(P, B, eps)
    for call in (lambda: sdblib.join_aggregate(x, y, None, fresh, TABLE, z),
                 lambda: sdblib.covering_build_table(fresh, 7),
                 lambda: sdblib.covering_build_table(fresh, 27),
                 lambda: sdblib.join_aggregate(x, y, None, cov, 5, z),
                 lambda: sdblib.join_aggregate_multi(x, y, None, [cov, fresh], TABLE,
                                                     torch.zeros((2, P.n), dtype=torch.int64,
                                                                 device="cuda"))):
        with pytest.raises(sdblib.SdbError) as e:
            call()
        assert e.value.status == sdblib.SDB_EINVAL


@pytest.mark.parametrize("lookup", LOOKUPS)
def test_table_global_aggregation_and_range(cuda, sdblib, orc, lookup):
    """P > 2048 (global atomics) and the result-range join through the table."""
    torch = cuda
    TABLE = lookup  # noqa: N806
    rng = np.random.default_rng(5)
    P = W.star_polygons(rng, 3000, 16, nverts=(3, 8), radius=(200, 900))
    pts = signed_points(6, 200_000, 16)
    oc = orc.cover(P, 40)
    cov = sdblib.build_covering(P, 16, 40)
    build_table(sdblib, cov, 12, lookup, leaf_bits=10)
    want = oc.join(pts.x, pts.y, pts.attr)
    cnt, sm = join(torch, sdblib, cov, pts, lookup)
    assert np.array_equal(cnt, want[0]) and np.array_equal(sm, want[1])
    no_fallback(sdblib, cov, lookup)
    for n_poly, seed in ((1500, 7), (7, 8)):  # global and shared range accumulators
        S = W.star_polygons(np.random.default_rng(seed), n_poly, 16, nverts=(3, 12),
                            radius=(200, 4000))
        ofl = orc.cover(S, 300, flagged=True)
        fl = sdblib.build_covering(S, 16, 300, flags=1)
        build_table(sdblib, fl, 10, lookup, leaf_bits=7)
        want = ofl.join_range(pts.x, pts.y, pts.attr)
        out = [torch.full((S.n,), 7, dtype=torch.int64, device="cuda") for _ in range(5)]
        sdblib.join_aggregate_range(dev(torch, pts.x), dev(torch, pts.y), dev(torch, pts.attr),
                                    fl, TABLE, out[0], out[2], out[1], out[3], out[4])
        torch.cuda.synchronize()
        got = [o.cpu().numpy() for o in out]
        for i, (g, w) in enumerate(zip(got, want)):
            assert np.array_equal(g.view(np.uint64) if i in (0, 2, 4) else g, w), (n_poly, i)


def test_table_full_size(cuda, sdblib):
    """100M mobility points, the 263-zone tiling at eps 2^6 and 2^10: the table
    lookup (several table sizes) equals the learned and binary-search lookups."""
    torch = cuda
    w = W.mobility_zones(100_000_000)
    T, pts = w.polygons, w.points
    x, y, a = dev(torch, pts.x), dev(torch, pts.y), dev(torch, pts.attr)
    for eps in (2 ** 6, 2 ** 10):
        cov = sdblib.build_covering(T, 24, eps)
        sdblib.covering_build_index(cov, 20 if eps == 64 else 14)
        ref = join(torch, sdblib, cov, pts, sdblib.LOOKUP_LEARNED, x=x, y=y, a=a)
        bs = join(torch, sdblib, cov, pts, sdblib.LOOKUP_BINARY, x=x, y=y, a=a)
        assert np.array_equal(ref[0], bs[0]) and np.array_equal(ref[1], bs[1])
        for tb in (18, 22, 24):
            sdblib.covering_build_table(cov, tb)
            for lookup in LOOKUPS:
                got = join(torch, sdblib, cov, pts, lookup, x=x, y=y, a=a)
                assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), (eps,
                                                                                          tb)
                no_fallback(sdblib, cov, lookup)


@pytest.mark.parametrize("lookup", LOOKUPS)
def test_table_sweep_join_equals_separate(cuda, sdblib, orc, lookup):
    """One pass over the points for several coverings through their tables (the
    combined top level where every covering holds the same polygon, each table
    elsewhere) equals one join per covering and the oracle; more coverings than
    one pass takes, coverings without a common top level, ragged n, COUNT only."""
    torch = cuda
    T = W.zones263_tiling()
    pts = W.mobility_points(W.BASE_SEED + 12, 300_007, 24, 32)
    eps_list = [1024, 2 ** 14, 64, 4096, 256]
    covs = [sdblib.build_covering(T, 24, e) for e in eps_list]
    for c in covs:
        build_table(sdblib, c, 22, lookup, leaf_bits=14)
    x, y, a = dev(torch, pts.x), dev(torch, pts.y), dev(torch, pts.attr)
    E, P = len(covs), T.n
    for n in (pts.n, 1001, 0):
        cnt = torch.full((E, P), 7, dtype=torch.int64, device="cuda")
        sm = torch.full((E, P), 7, dtype=torch.int64, device="cuda")
        sdblib.join_aggregate_multi(x[:n], y[:n], a[:n], covs, lookup, cnt, sm)
        torch.cuda.synchronize()
        for e, c in enumerate(covs):
            want = join(torch, sdblib, c, pts, lookup, x=x[:n], y=y[:n], a=a[:n])
            assert np.array_equal(cnt[e].cpu().numpy().view(np.uint64), want[0]), (n, e)
            assert np.array_equal(sm[e].cpu().numpy(), want[1]), (n, e)
            no_fallback(sdblib, c, lookup)
    want = orc.cover(T, 4096).join(pts.x, pts.y, pts.attr)
    cnt = torch.zeros((E, P), dtype=torch.int64, device="cuda")
    sdblib.join_aggregate_multi(x, y, None, covs, lookup, cnt)
    torch.cuda.synchronize()
    assert np.array_equal(cnt[3].cpu().numpy().view(np.uint64), want[0])
    # top levels of different levels (a 2^8-bucket table has its top at level 4):
    # no combined level, every point asks the tables
    small = sdblib.build_covering(T, 24, 2 ** 13)
    build_table(sdblib, small, 8, lookup, leaf_bits=6)
    pair = [small, covs[2]]
    cnt = torch.zeros((2, P), dtype=torch.int64, device="cuda")
    sm = torch.zeros((2, P), dtype=torch.int64, device="cuda")
    sdblib.join_aggregate_multi(x, y, a, pair, lookup, cnt, sm)
    torch.cuda.synchronize()
    for e, c in enumerate(pair):
        want = join(torch, sdblib, c, pts, lookup, x=x, y=y, a=a)
        assert np.array_equal(cnt[e].cpu().numpy().view(np.uint64), want[0]), e
        assert np.array_equal(sm[e].cpu().numpy(), want[1]), e
