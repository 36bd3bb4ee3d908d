"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer results, so the bar is bit-exact: canonical coverings, per-polygon
counts and int64 sums.  The learned and cell-table lookups must equal binary
search.
"""
import json
import os

import numpy as np
import pytest

from paper_2010_12548_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def dev(torch, a):
    a = np.ascontiguousarray(a)
    return torch.from_numpy(a.view(np.int32) if a.dtype.itemsize == 4 else a).cuda()


def gpu_join(torch, sdb, cov, pts, lookup=0, with_sum=True, x=None, y=None, a=None):
    P = cov.info().n_polygons
    x = dev(torch, pts.x) if x is None else x
    y = dev(torch, pts.y) if y is None else y
    a = (dev(torch, pts.attr) if a is None else a) if with_sum else None
    cnt = torch.full((P,), 7, dtype=torch.int64, device="cuda")  # the call must zero it
    sm = torch.full((P,), 7, dtype=torch.int64, device="cuda") if with_sum else None
    sdb.join_aggregate(x, y, a, cov, lookup, cnt, sm)
    torch.cuda.synchronize()
    return cnt.cpu().numpy().view(np.uint64), (sm.cpu().numpy() if with_sum else None)


def assert_same_covering(sdb, cov, oc):
    st, lo, ids = sdb.covering_export(cov)
    assert np.array_equal(st, oc.start)
    assert np.array_equal(lo, oc.list_off)
    assert np.array_equal(ids, oc.list_ids)


def polys_of(rings, B):
    off, xs, ys = [0], [], []
    for r in rings:
        xs += [p[0] for p in r]
        ys += [p[1] for p in r]
        off.append(len(xs))
    return W.Polygons(np.array(off, np.uint32), np.array(xs, np.uint32), np.array(ys, np.uint32), B)


def lattice(B):
    g = np.arange(2 ** B, dtype=np.uint32)
    gx, gy = np.meshgrid(g, g)
    return W.Points(gx.ravel(), gy.ravel(), np.ones(gx.size, np.int32), B)


def small_stars(seed, B, n=6, nverts=(3, 12)):
    rng = np.random.default_rng(seed)
    G = 2 ** B
    return W.star_polygons(rng, n, B, nverts=nverts, radius=(G / 16, G / 5))


def test_handworked_golden(cuda, sdblib):
    with open(os.path.join(GOLD, "handworked_b4.json")) as f:
        g = json.load(f)
    B = g["grid_bits"]
    pts = lattice(B)
    for name, ring in g["polygons"].items():
        P = polys_of([ring], B)
        for c in g["cases"]:
            cov = sdblib.build_covering(P, B, c["eps"])
            sdblib.covering_build_index(cov, 4)
            sdblib.covering_build_table(cov, 8)
            for lookup in (0, 1, 3):
                cnt, sm = gpu_join(cuda, sdblib, cov, pts, lookup)
                assert int(cnt[0]) == c[name] and int(sm[0]) == c[name], (name, c, lookup)


@pytest.mark.parametrize("B,eps,seed", [(6, 2, 1), (6, 5, 2), (7, 12, 3), (8, 3, 4), (8, 23, 5),
                                        (10, 2, 6), (10, 40, 7), (12, 9, 8), (16, 64, 9),
                                        (16, 1000, 10), (16, 2 ** 17, 11), (5, 2 ** 10, 12)])
def test_covering_and_join_vs_oracle_small(cuda, sdblib, orc, B, eps, seed):
    P = small_stars(seed, B)
    oc = orc.cover(P, eps)
    cov = sdblib.build_covering(P, B, eps)
    inf = cov.info()
    assert (inf.finest_shift, inf.finest_level) == (oc.k, oc.F)
    assert_same_covering(sdblib, cov, oc)
    rng = np.random.default_rng(seed)
    n = 20_011
    pts = W.Points(rng.integers(0, 2 ** B, n, dtype=np.uint32),
                   rng.integers(0, 2 ** B, n, dtype=np.uint32),
                   rng.integers(-2 ** 31, 2 ** 31, n, dtype=np.int64).astype(np.int32), B)
    want = oc.join(pts.x, pts.y, pts.attr)
    sdblib.covering_build_index(cov, 4 if oc.R < 64 else 8)
    for lookup in (0, 1):
        cnt, sm = gpu_join(cuda, sdblib, cov, pts, lookup)
        assert np.array_equal(cnt, want[0]) and np.array_equal(sm, want[1]), lookup
    assert sdblib.covering_fallbacks(cov) == 0
    for tb in (8, 12, 26):  # coarse buckets (many mixed) up to one id per bucket
        sdblib.covering_build_table(cov, tb)
        assert cov.info().table_bits == min(tb, 2 * oc.F)
        cnt, sm = gpu_join(cuda, sdblib, cov, pts, sdblib.LOOKUP_TABLE)
        assert np.array_equal(cnt, want[0]) and np.array_equal(sm, want[1]), tb


def test_finest_grid_unpacked_records(cuda, sdblib, orc):
    """B = 30 at eps 2 (F = 30): keys of 61 bits leave no room to pack the
    record's value into the key word, so the builder takes the two-array
    record path; coverings and joins still equal the oracle's."""
    rng = np.random.default_rng(21)
    B = 30
    base = W.star_polygons(rng, 5, 12, nverts=(3, 9), radius=(20, 60))
    off = np.uint32(2 ** 29 + 12345)  # small stars somewhere in the middle of the grid
    P = W.Polygons(base.ring_off, base.x + off, base.y + off, B)
    for eps in (2, 3, 40):
        oc = orc.cover(P, eps)
        cov = sdblib.build_covering(P, B, eps)
        assert_same_covering(sdblib, cov, oc)
        n = 30_001
        pts = W.Points((rng.integers(0, 4096, n) + off).astype(np.uint32),
                       (rng.integers(0, 4096, n) + off).astype(np.uint32),
                       rng.integers(-2 ** 31, 2 ** 31, n, dtype=np.int64).astype(np.int32), B)
        want = oc.join(pts.x, pts.y, pts.attr)
        sdblib.covering_build_index(cov, 6)
        sdblib.covering_build_table(cov, 20)
        for lookup in (0, 1, 3):
            cnt, sm = gpu_join(cuda, sdblib, cov, pts, lookup)
            assert np.array_equal(cnt, want[0]) and np.array_equal(sm, want[1]), (eps, lookup)


def test_stars16_workload(cuda, sdblib, orc):
    """100k uniform points, 16 overlapping star polygons, eps = 64 (F = 11)."""
    w = W.tiny_stars()
    oc = orc.cover(w.polygons, 64)
    cov = sdblib.build_covering(w.polygons, 16, 64)
    assert_same_covering(sdblib, cov, oc)
    o1 = oc.join(w.points.x, w.points.y, w.points.attr)
    o2 = orc.join_o2(w.polygons, 64, w.points, threads=4)
    assert np.array_equal(o1[0], o2[0]) and np.array_equal(o1[1], o2[1])
    for leaf_bits in (4, 8, 12):
        sdblib.covering_build_index(cov, leaf_bits)
        for lookup in (0, 1):
            cnt, sm = gpu_join(cuda, sdblib, cov, w.points, lookup)
            assert np.array_equal(cnt, o1[0]) and np.array_equal(sm, o1[1])
        assert sdblib.covering_fallbacks(cov) == 0
    # the root as one line (the plain two-level model) and as 2^6 segments
    for root_bits in (0, 6):
        sdblib.covering_build_index(cov, 8, root_bits=root_bits)
        assert cov.info().index_root_bits == root_bits
        cnt, sm = gpu_join(cuda, sdblib, cov, w.points, 1)
        assert np.array_equal(cnt, o1[0]) and np.array_equal(sm, o1[1])
        assert sdblib.covering_fallbacks(cov) == 0


def test_zones_tiling_coarse_eps(cuda, sdblib, orc):
    """The 263-zone tiling on [0,2^24)^2 at eps 2^12 and 2^10, 1M mobility points."""
    T = W.zones263_tiling()
    pts = W.mobility_points(W.BASE_SEED + 7, 1_000_000, 24, 32)
    for eps in (2 ** 12, 2 ** 10):
        oc = orc.cover(T, eps)
        cov = sdblib.build_covering(T, 24, eps)
        assert_same_covering(sdblib, cov, oc)
        want = oc.join(pts.x, pts.y, pts.attr)
        assert int(want[0].sum()) >= pts.n  # tiling: every point in >= 1 polygon
        sdblib.covering_build_index(cov, 12)
        assert cov.info().index_root_bits == 12
        for lookup in (0, 1):
            cnt, sm = gpu_join(cuda, sdblib, cov, pts, lookup)
            assert np.array_equal(cnt, want[0]) and np.array_equal(sm, want[1])
        assert sdblib.covering_fallbacks(cov) == 0
        sdblib.covering_build_index(cov, 12, root_bits=0)  # one root line
        cnt, sm = gpu_join(cuda, sdblib, cov, pts, 1)
        assert np.array_equal(cnt, want[0]) and np.array_equal(sm, want[1])
        assert sdblib.covering_fallbacks(cov) == 0


def test_edge_cases(cuda, sdblib, orc):
    torch = cuda
    B, eps = 12, 9
    P = small_stars(77, B, n=9)
    oc = orc.cover(P, eps)
    cov = sdblib.build_covering(P, B, eps)
    sdblib.covering_build_index(cov, 6)
    rng = np.random.default_rng(3)
    base = W.Points(rng.integers(0, 2 ** B, 5000, dtype=np.uint32),
                    rng.integers(0, 2 ** B, 5000, dtype=np.uint32),
                    rng.integers(-1000, 1000, 5000).astype(np.int32), B)
    # points outside the grid match nothing
    base.x[::97] = 2 ** B + 5
    base.y[::89] = 2 ** 31
    for n in (0, 1, 2, 3, 4, 5, 127, 128, 129, 1003, 5000):
        pts = base.take(np.arange(n))
        want = oc.join(pts.x, pts.y, pts.attr)
        for lookup in (0, 1):
            cnt, sm = gpu_join(torch, sdblib, cov, pts, lookup)
            assert np.array_equal(cnt, want[0]) and np.array_equal(sm, want[1]), (n, lookup)
            cnt, _ = gpu_join(torch, sdblib, cov, pts, lookup, with_sum=False)
            assert np.array_equal(cnt, want[0])
    # unaligned device pointers (offset by one element) take the scalar path
    x = dev(torch, np.concatenate([[0], base.x]).astype(np.uint32))[1:]
    y = dev(torch, np.concatenate([[0], base.y]).astype(np.uint32))[1:]
    a = dev(torch, np.concatenate([[0], base.attr]).astype(np.int32))[1:]
    want = oc.join(base.x, base.y, base.attr)
    for lookup in (0, 1):
        cnt, sm = gpu_join(torch, sdblib, cov, base, lookup, x=x, y=y, a=a)
        assert np.array_equal(cnt, want[0]) and np.array_equal(sm, want[1])


def test_many_polygons_global_aggregation(cuda, sdblib, orc):
    """P > 2048 takes the global-memory aggregation path."""
    rng = np.random.default_rng(5)
    P = W.star_polygons(rng, 3000, 16, nverts=(3, 8), radius=(200, 900))
    pts = W.uniform_points(rng, 200_000, 16)
    for eps in (40, 300):
        oc = orc.cover(P, eps)
        cov = sdblib.build_covering(P, 16, eps)
        assert_same_covering(sdblib, cov, oc)
        want = oc.join(pts.x, pts.y, pts.attr)
        sdblib.covering_build_index(cov, 10)
        for lookup in (0, 1):
            cnt, sm = gpu_join(cuda, sdblib, cov, pts, lookup)
            assert np.array_equal(cnt, want[0]) and np.array_equal(sm, want[1])


def test_host_join_multi_covering(cuda, sdblib, orc):
    w = W.tiny_stars(300_001)
    covs, wants = [], []
    for eps in (64, 256, 2048):
        oc = orc.cover(w.polygons, eps)
        c = sdblib.build_covering(w.polygons, 16, eps)
        sdblib.covering_build_index(c, 8)
        covs.append(c)
        wants.append(oc.join(w.points.x, w.points.y, w.points.attr))
    for lookup in (0, 1):
        cnt, sm = sdblib.join_aggregate_host(w.points.x, w.points.y, w.points.attr, covs, lookup)
        for i in range(3):
            assert np.array_equal(cnt[i], wants[i][0]) and np.array_equal(sm[i], wants[i][1])


def test_deterministic(cuda, sdblib):
    T = W.zones263_tiling()
    pts = W.mobility_points(W.BASE_SEED + 8, 2_000_000, 24, 32)
    c1 = sdblib.build_covering(T, 24, 2 ** 8)
    c2 = sdblib.build_covering(T, 24, 2 ** 8)
    e1, e2 = sdblib.covering_export(c1), sdblib.covering_export(c2)
    assert all(np.array_equal(a, b) for a, b in zip(e1, e2))
    sdblib.covering_build_index(c1, 12)
    r = [gpu_join(cuda, sdblib, c1, pts, lk) for lk in (0, 1, 0, 1)]
    for a, b in r[1:]:
        assert np.array_equal(a, r[0][0]) and np.array_equal(b, r[0][1])


def test_build_coverings_eps_sweep(cuda, sdblib, orc):
    """Coverings of an eps sweep built in one pass equal the ones built one at
    a time, entry for entry (zone tiling: the joint pass; overlapping stars:
    the per-eps fallback), with boundary flags and non-conservative too."""
    T = W.zones263_tiling()
    for flags in (0, 1, 2):
        covs = sdblib.build_coverings(T, 24, [4096, 1024, 256], flags=flags)
        for c, eps in zip(covs, (4096, 1024, 256)):
            one = sdblib.build_covering(T, 24, eps, flags=flags)
            for a, b in zip(sdblib.covering_export(c), sdblib.covering_export(one)):
                assert np.array_equal(a, b), (flags, eps)
            ia, ib = c.info(), one.info()
            assert (ia.n_ranges, ia.n_list_ids, ia.n_cells) == (ib.n_ranges, ib.n_list_ids,
                                                                ib.n_cells)
    w = W.tiny_stars(10_000)
    covs = sdblib.build_coverings(w.polygons, 16, [2048, 64, 5])
    for c, eps in zip(covs, (2048, 64, 5)):
        assert_same_covering(sdblib, c, orc.cover(w.polygons, eps))


def test_join_multi_equals_separate_joins(cuda, sdblib, orc):
    """One pass over the points for several coverings (an eps sweep, more than
    one group of four, unordered) equals one join per covering; the finest
    covering need not come first; many polygons take global accumulators."""
    torch = cuda
    T = W.zones263_tiling()
    pts = W.mobility_points(W.BASE_SEED + 12, 300_007, 24, 32)
    eps_list = [1024, 2 ** 14, 64, 4096, 256]
    covs = [sdblib.build_covering(T, 24, e) for e in eps_list]
    for c in covs:
        sdblib.covering_build_index(c, 14)
    x, y, a = dev(torch, pts.x), dev(torch, pts.y), dev(torch, pts.attr)
    E, P = len(covs), T.n
    for lookup in (0, 1):
        for n in (pts.n, 1001):
            cnt = torch.full((E, P), 7, dtype=torch.int64, device="cuda")
            sm = torch.full((E, P), 7, dtype=torch.int64, device="cuda")
            sdblib.join_aggregate_multi(x[:n], y[:n], a[:n], covs, lookup, cnt, sm)
            torch.cuda.synchronize()
            for e, c in enumerate(covs):
                want = gpu_join(torch, sdblib, c, pts, lookup, x=x[:n], y=y[:n], a=a[:n])
                assert np.array_equal(cnt[e].cpu().numpy().view(np.uint64), want[0]), (lookup, e)
                assert np.array_equal(sm[e].cpu().numpy(), want[1]), (lookup, e)
    # the oracle on one covering, and unaligned pointers
    want = orc.cover(T, 64).join(pts.x[1:], pts.y[1:], pts.attr[1:])
    cnt = torch.zeros((E, P), dtype=torch.int64, device="cuda")
    sm = torch.zeros((E, P), dtype=torch.int64, device="cuda")
    sdblib.join_aggregate_multi(x[1:], y[1:], a[1:], covs, 1, cnt, sm)
    torch.cuda.synchronize()
    assert np.array_equal(cnt[2].cpu().numpy().view(np.uint64), want[0])
    assert np.array_equal(sm[2].cpu().numpy(), want[1])
    # 3000 polygons x 2 coverings > 2048 accumulators: global atomics
    rng = np.random.default_rng(5)
    S = W.star_polygons(rng, 3000, 16, nverts=(3, 8), radius=(200, 900))
    sp = W.uniform_points(rng, 100_000, 16)
    sc = [sdblib.build_covering(S, 16, e) for e in (40, 300)]
    cnt = torch.zeros((2, S.n), dtype=torch.int64, device="cuda")
    sm = torch.zeros((2, S.n), dtype=torch.int64, device="cuda")
    sdblib.join_aggregate_multi(dev(torch, sp.x), dev(torch, sp.y), dev(torch, sp.attr), sc, 0,
                                cnt, sm)
    torch.cuda.synchronize()
    for e, eps in enumerate((40, 300)):
        want = orc.cover(S, eps).join(sp.x, sp.y, sp.attr)
        assert np.array_equal(cnt[e].cpu().numpy().view(np.uint64), want[0])
        assert np.array_equal(sm[e].cpu().numpy(), want[1])
