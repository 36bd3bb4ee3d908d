"""Result range estimation (Sec. 6) on the GPU vs the CPU oracle.

Boundary-flagged coverings must equal the oracle's flagged coverings entry for
entry (both merge paths), and the range join's five per-polygon outputs (count,
sum, boundary count, boundary sum, boundary magnitude sum) must equal the
oracle's flagged O1 join bit for bit, for both lookups, and the COUNT and SUM
intervals the library derives from them on the device must equal the
oracle's.  At full size (the
263-zone tiling at eps = 2^6 over 100M points) the counts and sums must equal
the plain join's and, on a sample of points, the boundary partials must equal
the definitional O2 test.
"""
import numpy as np
import pytest

from oracle import oracle as ORC
from paper_2010_12548_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FLAG = 1  # COVER_BOUNDARY_FLAGS


def dev(torch, a):
    a = np.ascontiguousarray(a)
    return torch.from_numpy(a.view(np.int32) if a.dtype.itemsize == 4 else a).cuda()


def gpu_range(torch, sdb, cov, pts, lookup, with_sum=True, x=None, y=None, a=None):
    P = cov.info().n_polygons
    x = dev(torch, pts.x) if x is None else x
    y = dev(torch, pts.y) if y is None else y
    a = (dev(torch, pts.attr) if a is None else a) if with_sum else None

    def out():  # the call must zero them
        return torch.full((P,), 7, dtype=torch.int64, device="cuda")
    cnt, bc = out(), out()
    sm, bs, ba = (out(), out(), out()) if with_sum else (None, None, None)
    sdb.join_aggregate_range(x, y, a, cov, lookup, cnt, bc, sm, bs, ba)
    # the Sec. 6 intervals, computed by the library from the device partials
    bounds = sdb.result_bounds(cnt, bc, sm, bs, ba)
    torch.cuda.synchronize()
    u64 = lambda t: t.cpu().numpy().view(np.uint64)  # noqa: E731
    if not with_sum:
        got = u64(cnt), u64(bc)
        lo_c, hi_c = bounds[0].cpu().numpy(), bounds[1].cpu().numpy()
        assert bounds[2] is None and bounds[3] is None
        assert np.array_equal(lo_c, got[0].astype(np.int64) - got[1].astype(np.int64))
        assert np.array_equal(hi_c, got[0].astype(np.int64))
        return got
    got = u64(cnt), sm.cpu().numpy(), u64(bc), bs.cpu().numpy(), u64(ba)
    LAST_BOUNDS[:] = [b.cpu().numpy() for b in bounds]
    return got


# the device intervals of the most recent gpu_range call with sums
LAST_BOUNDS = []


def assert_bounds_match_oracle(orc, want):
    """The library's intervals equal the oracle's, element by element."""
    for g, w in zip(LAST_BOUNDS, orc.range_bounds(*want)):
        assert np.array_equal(g, w)


def assert_same_covering(sdb, cov, oc):
    st, lo, ids = sdb.covering_export(cov)
    assert np.array_equal(st, oc.start)
    assert np.array_equal(lo, oc.list_off)
    assert np.array_equal(ids, oc.list_ids)


def signed_points(seed, n, B):
    rng = np.random.default_rng(seed)
    a = rng.integers(-2 ** 31, 2 ** 31, n, dtype=np.int64).astype(np.int32)
    a[:3] = [-2 ** 31, 2 ** 31 - 1, 0]
    return W.Points(rng.integers(0, 2 ** B, n, dtype=np.uint32),
                    rng.integers(0, 2 ** B, n, dtype=np.uint32), a, B)


def check_range(torch, sdb, cov, oc, pts):
    want = oc.join_range(pts.x, pts.y, pts.attr)
    plain = oc.join(pts.x, pts.y, pts.attr)
    for lookup in (0, 1):
        got = gpu_range(torch, sdb, cov, pts, lookup)
        for g, w in zip(got, want):
            assert np.array_equal(g, w), lookup
        assert_bounds_match_oracle(ORC, want)
        c, b = gpu_range(torch, sdb, cov, pts, lookup, with_sum=False)
        assert np.array_equal(c, want[0]) and np.array_equal(b, want[2])
        # the plain join on a flagged covering: plain results
        P = cov.info().n_polygons
        cnt = torch.zeros(P, dtype=torch.int64, device="cuda")
        sm = torch.zeros(P, dtype=torch.int64, device="cuda")
        sdb.join_aggregate(dev(torch, pts.x), dev(torch, pts.y), dev(torch, pts.attr), cov, lookup,
                           cnt, sm)
        torch.cuda.synchronize()
        assert np.array_equal(cnt.cpu().numpy().view(np.uint64), plain[0])
        assert np.array_equal(sm.cpu().numpy(), plain[1])
    return want


@pytest.mark.parametrize("B,eps,seed", [(8, 3, 1), (10, 2, 2), (12, 9, 3), (16, 64, 4),
                                        (16, 700, 5)])
def test_flagged_overlapping_stars(cuda, sdblib, orc, B, eps, seed):
    """Overlapping stars take the general merge; every output vs the oracle."""
    rng = np.random.default_rng(seed)
    G = 2 ** B
    P = W.star_polygons(rng, 7, B, nverts=(3, 12), radius=(G / 16, G / 5))
    oc = orc.cover(P, eps, flagged=True)
    cov = sdblib.build_covering(P, B, eps, flags=FLAG)
    assert cov.info().boundary_flags == 1
    assert_same_covering(sdblib, cov, oc)
    sdblib.covering_build_index(cov, 6)
    pts = signed_points(seed, 20_011, B)
    want = check_range(cuda, sdblib, cov, oc, pts)
    ex, exs = orc.join_exact(P, pts)
    lo_c, hi_c, lo_s, hi_s = LAST_BOUNDS
    assert ((lo_c <= ex) & (ex <= hi_c)).all() and ((lo_s <= exs) & (exs <= hi_s)).all()


def test_flagged_zones_tiling(cuda, sdblib, orc):
    """The 263-zone tiling (fast merge path) at eps 2^12 and 2^10, 1M points."""
    T = W.zones263_tiling()
    pts = W.mobility_points(W.BASE_SEED + 7, 1_000_003, 24, 32)
    for eps in (2 ** 12, 2 ** 10):
        oc = orc.cover(T, eps, flagged=True)
        cov = sdblib.build_covering(T, 24, eps, flags=FLAG)
        assert_same_covering(sdblib, cov, oc)
        plain = sdblib.build_covering(T, 24, eps)
        assert cov.info().n_ranges >= plain.info().n_ranges
        sdblib.covering_build_index(cov, 12)
        check_range(cuda, sdblib, cov, oc, pts)
        assert sdblib.covering_fallbacks(cov) == 0


def test_range_edge_cases(cuda, sdblib, orc):
    torch = cuda
    B = 12
    rng = np.random.default_rng(9)
    P = W.star_polygons(rng, 9, B, nverts=(3, 12), radius=(256, 800))
    base = signed_points(21, 5000, B)
    base.x[::97] = 2 ** B + 5  # outside the grid: no polygon
    for eps in (9, 2 ** 13):  # 2^13: one cell covers the grid (finest level 0)
        oc = orc.cover(P, eps, flagged=True)
        cov = sdblib.build_covering(P, B, eps, flags=FLAG)
        assert_same_covering(sdblib, cov, oc)
        sdblib.covering_build_index(cov, 4)
        for n in (0, 1, 3, 4, 5, 129, 1003, 5000):
            pts = base.take(np.arange(n))
            want = oc.join_range(pts.x, pts.y, pts.attr)
            for lookup in (0, 1):
                got = gpu_range(torch, sdblib, cov, pts, lookup)
                for g, w in zip(got, want):
                    assert np.array_equal(g, w), (eps, n, lookup)
                assert_bounds_match_oracle(orc, want)
    # argument errors are caught on the host
    plain = sdblib.build_covering(P, B, 9)
    z = torch.zeros(P.n, dtype=torch.int64, device="cuda")
    x = dev(torch, base.x)
    with pytest.raises(sdblib.SdbError) as e:
        sdblib.join_aggregate_range(x, x, None, plain, 0, z, z)
    assert e.value.status == sdblib.SDB_EINVAL
    cov = sdblib.build_covering(P, B, 9, flags=FLAG)
    with pytest.raises(sdblib.SdbError) as e:
        sdblib.join_aggregate_range(x, x, dev(torch, base.attr), cov, 0, z, z, z, None, z)
    assert e.value.status == sdblib.SDB_EINVAL
    with pytest.raises(sdblib.SdbError) as e:
        sdblib.build_covering(P, B, 9, flags=4)
    assert e.value.status == sdblib.SDB_EINVAL
    with pytest.raises(sdblib.SdbError) as e:  # sum arrays given only in part
        sdblib.result_bounds(z, z, z, None, z)
    assert e.value.status == sdblib.SDB_EINVAL


def test_range_many_polygons_global(cuda, sdblib, orc):
    """P > 1024: the range join accumulates in global memory."""
    rng = np.random.default_rng(5)
    P = W.star_polygons(rng, 1500, 16, nverts=(3, 8), radius=(200, 900))
    pts = signed_points(6, 100_000, 16)
    oc = orc.cover(P, 300, flagged=True)
    cov = sdblib.build_covering(P, 16, 300, flags=FLAG)
    assert_same_covering(sdblib, cov, oc)
    sdblib.covering_build_index(cov, 10)
    check_range(cuda, sdblib, cov, oc, pts)


def test_range_full_size_sampled(cuda, sdblib, orc):
    """eps = 2^6 on the 263-zone tiling, 100M mobility points: counts and sums
    equal the plain join's; the boundary partials on a 2M-point sample equal
    the definitional test; the intervals contain the exact sample answers."""
    torch = cuda
    w = W.mobility_zones(100_000_000)
    T, pts = w.polygons, w.points
    eps = 64
    cov = sdblib.build_covering(T, 24, eps, flags=FLAG)
    plain = sdblib.build_covering(T, 24, eps)
    bits = 20
    sdblib.covering_build_index(cov, bits)
    sdblib.covering_build_index(plain, bits)
    x, y, a = dev(torch, pts.x), dev(torch, pts.y), dev(torch, pts.attr)
    P = T.n
    cnt = torch.zeros(P, dtype=torch.int64, device="cuda")
    sm = torch.zeros(P, dtype=torch.int64, device="cuda")
    sdblib.join_aggregate(x, y, a, plain, 1, cnt, sm)
    torch.cuda.synchronize()
    got = gpu_range(torch, sdblib, cov, pts, 1, x=x, y=y, a=a)
    assert np.array_equal(got[0], cnt.cpu().numpy().view(np.uint64))
    assert np.array_equal(got[1], sm.cpu().numpy())
    assert (got[2] <= got[0]).all()
    assert sdblib.covering_fallbacks(cov) == 0
    del x, y, a
    rng = np.random.default_rng(13)
    sample = pts.take(np.sort(rng.choice(pts.n, 2_000_000, replace=False)))
    g = gpu_range(torch, sdblib, cov, sample, 1)
    c2, s2, b2, bs2, ba2 = orc.join_o2(T, eps, sample, threads=16, boundary_sums=True)
    for u, v in zip(g, (c2, s2, b2, bs2, ba2)):
        assert np.array_equal(u, v)
    assert_bounds_match_oracle(orc, (c2, s2, b2, bs2, ba2))
    ex, exs = orc.join_exact(T, sample, threads=16)
    lo_c, hi_c, lo_s, hi_s = LAST_BOUNDS
    assert ((lo_c <= ex) & (ex <= hi_c)).all() and ((lo_s <= exs) & (exs <= hi_s)).all()
