"""Point-indexed aggregation (Sec. 3, "Point Indexing") on the GPU.

Range counting over the resident, Hilbert-sorted points with prefix sums must
equal the oracle's definition (sorted keys, std::lower_bound per range
boundary) and the per-point join exactly, with binary search and with the
RadixSpline lookup; the spline's measured interpolation error must stay
within its bound.
"""
import numpy as np
import pytest

from paper_2010_12548_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


def resident(torch, sdb, pts, B):
    return sdb.points_create(dev(torch, pts.x), dev(torch, pts.y), dev(torch, pts.attr), B)


def aggregate(torch, sdb, p, cov, lookup, with_sum=True):
    P = cov.info().n_polygons
    cnt = torch.full((P,), 7, dtype=torch.int64, device="cuda")  # the call must zero it
    sm = torch.full((P,), 7, dtype=torch.int64, device="cuda") if with_sum else None
    sdb.points_aggregate(p, cov, lookup, cnt, sm)
    torch.cuda.synchronize()
    return cnt.cpu().numpy().view(np.uint64), (sm.cpu().numpy() if with_sum else None)


def signed(rng, pts):
    a = rng.integers(-2 ** 31, 2 ** 31, pts.n, dtype=np.int64).astype(np.int32)
    return W.Points(pts.x, pts.y, a, pts.grid_bits)


@pytest.mark.parametrize("radix_bits,spline_error", [(25, 32), (4, 1), (12, 1000), (18, 3)])
def test_point_index_vs_oracle_stars(cuda, sdblib, orc, radix_bits, spline_error):
    torch = cuda
    w = W.tiny_stars(60_000)
    rng = np.random.default_rng(radix_bits)
    base = signed(rng, w.points)
    # duplicated locations
    pts = W.Points(np.concatenate([base.x, base.x[:3000]]), np.concatenate([base.y, base.y[:3000]]),
                   np.concatenate([base.attr, base.attr[:3000]]), 16)
    p = resident(torch, sdblib, pts, 16)
    cnt0, _ = None, None
    for eps in (2 ** 17, 4096, 300, 64, 5):
        cov = sdblib.build_covering(w.polygons, 16, eps)
        oc = orc.cover(w.polygons, eps)
        want = oc.point_index_aggregate(pts.x, pts.y, pts.attr)
        assert all(np.array_equal(u, v) for u, v in zip(want, oc.join(pts.x, pts.y, pts.attr)))
        cnt0, _ = aggregate(torch, sdblib, p, cov, sdblib.LOOKUP_BINARY, with_sum=False)
        assert np.array_equal(cnt0, want[0]), eps
    sdblib.points_build_index(p, radix_bits, spline_error)
    ns, err, _ = sdblib.points_index_stats(p)
    assert 2 <= ns and err <= spline_error
    for eps in (2 ** 17, 4096, 300, 64, 5):
        cov = sdblib.build_covering(w.polygons, 16, eps, flags=1 if eps == 64 else 0)
        want = orc.cover(w.polygons, eps).point_index_aggregate(pts.x, pts.y, pts.attr)
        for lookup in (sdblib.LOOKUP_BINARY, sdblib.LOOKUP_RADIX_SPLINE):
            got = aggregate(torch, sdblib, p, cov, lookup)
            assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1]), (eps, lookup)


def test_point_index_heavy_duplicates_and_tiny(cuda, sdblib, orc):
    """Points on a coarse lattice (runs of equal keys across chunk borders),
    a single point, and points on the grid's corners."""
    torch = cuda
    rng = np.random.default_rng(4)
    w = W.tiny_stars(10)
    g = rng.integers(0, 16, size=(200_000, 2)) * 4096
    pts = W.Points(g[:, 0].astype(np.uint32), g[:, 1].astype(np.uint32),
                   rng.integers(-1000, 1000, 200_000).astype(np.int32), 16)
    for sub in (pts, pts.take(np.arange(1)),
                W.Points(np.array([0, 65535, 0, 65535], np.uint32),
                         np.array([0, 0, 65535, 65535], np.uint32),
                         np.array([1, 2, 3, 4], np.int32), 16)):
        p = resident(torch, sdblib, sub, 16)
        sdblib.points_build_index(p, 10, 2)
        _, err, _ = sdblib.points_index_stats(p)
        assert err <= 2
        for eps in (2 ** 17, 700, 9):
            cov = sdblib.build_covering(w.polygons, 16, eps)
            want = orc.cover(w.polygons, eps).point_index_aggregate(sub.x, sub.y, sub.attr)
            for lookup in (sdblib.LOOKUP_BINARY, sdblib.LOOKUP_RADIX_SPLINE):
                got = aggregate(torch, sdblib, p, cov, lookup)
                assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


def test_point_index_errors(cuda, sdblib):
    torch = cuda
    w = W.tiny_stars(1000)
    p = resident(torch, sdblib, w.points, 16)
    cov = sdblib.build_covering(w.polygons, 16, 64)
    z = torch.zeros(w.polygons.n, dtype=torch.int64, device="cuda")
    for call in (lambda: sdblib.points_aggregate(p, cov, sdblib.LOOKUP_BINARY, z, z),  # no index
                 lambda: sdblib.points_aggregate(p, cov, sdblib.LOOKUP_RADIX_SPLINE, z),
                 lambda: sdblib.points_aggregate(p, cov, sdblib.LOOKUP_LEARNED, z),
                 lambda: sdblib.points_build_index(p, 31, 32),
                 lambda: sdblib.points_build_index(p, 20, 0)):
        with pytest.raises(sdblib.SdbError) as e:
            call()
        assert e.value.status == sdblib.SDB_EINVAL
    other = sdblib.build_covering(w.polygons, 17, 64)  # other grid bits
    sdblib.points_build_index(p)
    with pytest.raises(sdblib.SdbError) as e:
        sdblib.points_aggregate(p, other, sdblib.LOOKUP_BINARY, z)
    assert e.value.status == sdblib.SDB_EINVAL


def test_point_index_tracts_vs_oracle(cuda, sdblib, orc):
    """The 40,000-polygon tiling on [0,2^28)^2, 2M resident points, eps 2^17."""
    torch = cuda
    T = W.tracts40k_tiling()
    pts = W.mobility_points(W.BASE_SEED + 55, 2_000_000, 28, 64, sigma=(2 ** 20, 2 ** 23))
    p = resident(torch, sdblib, pts, 28)
    sdblib.points_build_index(p, 25, 32)
    eps = 2 ** 17
    cov = sdblib.build_covering(T, 28, eps)
    want = orc.cover(T, eps).join(pts.x, pts.y, pts.attr)
    for lookup in (sdblib.LOOKUP_BINARY, sdblib.LOOKUP_RADIX_SPLINE):
        got = aggregate(torch, sdblib, p, cov, lookup)
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
    assert sdblib.points_index_stats(p)[2] == 0


def test_point_index_full_size(cuda, sdblib):
    """200M resident points and the 40,000-polygon tiling (the paper's
    point-indexing setting): range counting with both lookups equals the
    per-point join over the same points, at three precision levels."""
    torch = cuda
    T, pts, _ = W.lod_workload()
    x, y, a = dev(torch, pts.x), dev(torch, pts.y), dev(torch, pts.attr)
    p = sdblib.points_create(x, y, a, 28)
    sdblib.points_build_index(p, 25, 32)
    ns, err, _ = sdblib.points_index_stats(p)
    assert err <= 32
    P = T.n
    for eps in (2 ** 19, 2 ** 17, 2 ** 16):
        cov = sdblib.build_covering(T, 28, eps)
        sdblib.covering_build_index(cov, 16)
        cnt = torch.zeros(P, dtype=torch.int64, device="cuda")
        sm = torch.zeros(P, dtype=torch.int64, device="cuda")
        sdblib.join_aggregate(x, y, a, cov, sdblib.LOOKUP_LEARNED, cnt, sm)
        torch.cuda.synchronize()
        want = cnt.cpu().numpy().view(np.uint64), sm.cpu().numpy()
        for lookup in (sdblib.LOOKUP_BINARY, sdblib.LOOKUP_RADIX_SPLINE):
            got = aggregate(torch, sdblib, p, cov, lookup)
            assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1]), eps
        assert sdblib.points_index_stats(p)[2] == 0
