"""Bounded Raster Join (Sec. 5.2) restated in CUDA, vs the CPU oracle.

Its answer is the definitional one (a point counts for a polygon when its
closed finest cell meets the closed polygon), computed here by blending the
points into a canvas of finest cells and rasterising every polygon
conservatively; it must equal the oracle's definitional O2 join exactly, for
every tiling of the canvas.
"""
import json
import os

import numpy as np
import pytest

from paper_2010_12548_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


def brj(torch, sdb, polys, B, eps, pts, tile_bits=0, with_sum=True, x=None, y=None, a=None):
    P = polys.n
    x = dev(torch, pts.x) if x is None else x
    y = dev(torch, pts.y) if y is None else y
    a = (dev(torch, pts.attr) if a is None else a) if with_sum else None
    cnt = torch.full((P,), 7, dtype=torch.int64, device="cuda")  # zeroed by the call
    sm = torch.full((P,), 7, dtype=torch.int64, device="cuda") if with_sum else None
    sdb.raster_join(polys, B, eps, x, y, a, cnt, sm, tile_bits)
    torch.cuda.synchronize()
    return cnt.cpu().numpy().view(np.uint64), (sm.cpu().numpy() if with_sum else None)


def polys_of(rings, B):
    off, xs, ys = [0], [], []
    for r in rings:
        xs += [p[0] for p in r]
        ys += [p[1] for p in r]
        off.append(len(xs))
    return W.Polygons(np.array(off, np.uint32), np.array(xs, np.uint32), np.array(ys, np.uint32), B)


def test_raster_handworked_golden(cuda, sdblib):
    with open(os.path.join(GOLD, "handworked_b4.json")) as f:
        g = json.load(f)
    B = g["grid_bits"]
    gx, gy = np.meshgrid(np.arange(2 ** B, dtype=np.uint32), np.arange(2 ** B, dtype=np.uint32))
    pts = W.Points(gx.ravel(), gy.ravel(), np.ones(gx.size, np.int32), B)
    for name, ring in g["polygons"].items():
        P = polys_of([ring], B)
        for c in g["cases"]:
            for tb in (0, 1, 2):
                cnt, sm = brj(cuda, sdblib, P, B, c["eps"], pts, tb)
                assert int(cnt[0]) == c[name] and int(sm[0]) == c[name], (name, c, tb)


@pytest.mark.parametrize("B,eps,seed", [(8, 3, 1), (10, 2, 2), (12, 9, 3), (16, 64, 4),
                                        (16, 700, 5), (12, 2 ** 13, 6)])
def test_raster_overlapping_stars_vs_oracle(cuda, sdblib, orc, B, eps, seed):
    rng = np.random.default_rng(seed)
    G = 2 ** B
    P = W.star_polygons(rng, 9, B, nverts=(3, 16), radius=(G / 16, G / 4))
    n = 30_011
    pts = W.Points(rng.integers(0, G, n, dtype=np.uint32), rng.integers(0, G, n, dtype=np.uint32),
                   rng.integers(-2 ** 31, 2 ** 31, n, dtype=np.int64).astype(np.int32), B)
    pts.x[::101] = G + 3  # outside the grid
    want = orc.join_o2(P, eps, pts)
    F = orc.finest_k(eps, B)[1]
    for tb in sorted({0, 1, 3, max(1, F - 8)}):
        if F - min(F, tb if tb else 13) > 8:
            continue
        cnt, sm = brj(cuda, sdblib, P, B, eps, pts, tb)
        assert np.array_equal(cnt, want[0]) and np.array_equal(sm, want[1]), tb
        cnt, _ = brj(cuda, sdblib, P, B, eps, pts, tb, with_sum=False)
        assert np.array_equal(cnt, want[0])


def test_raster_zones_vs_oracle(cuda, sdblib, orc):
    """The 263-zone tiling on [0,2^24)^2, 1M mobility points, eps 2^12 (one
    tile) and 2^10 (16 tiles), plus a tiling with smaller tiles."""
    T = W.zones263_tiling()
    pts = W.mobility_points(W.BASE_SEED + 9, 1_000_003, 24, 32)
    for eps, tb in ((2 ** 12, 0), (2 ** 10, 0), (2 ** 10, 9)):
        want = orc.cover(T, eps).join(pts.x, pts.y, pts.attr)
        cnt, sm = brj(cuda, sdblib, T, 24, eps, pts, tb)
        assert np.array_equal(cnt, want[0]) and np.array_equal(sm, want[1]), (eps, tb)


def test_raster_edge_cases_and_errors(cuda, sdblib, orc):
    torch = cuda
    rng = np.random.default_rng(7)
    P = W.star_polygons(rng, 5, 12, nverts=(3, 10), radius=(300, 900))
    pts = W.Points(rng.integers(0, 4096, 1000, dtype=np.uint32),
                   rng.integers(0, 4096, 1000, dtype=np.uint32),
                   rng.integers(-9, 9, 1000).astype(np.int32), 12)
    for n in (0, 1, 2, 999):
        sub = pts.take(np.arange(n))
        want = orc.join_o2(P, 9, sub)
        cnt, sm = brj(torch, sdblib, P, 12, 9, sub, 2)
        assert np.array_equal(cnt, want[0]) and np.array_equal(sm, want[1]), n
    x = dev(torch, pts.x)
    z = torch.zeros(P.n, dtype=torch.int64, device="cuda")
    for kw in (dict(eps=9, tile_bits=15), dict(eps=2, tile_bits=1), dict(eps=1, tile_bits=0)):
        with pytest.raises(sdblib.SdbError) as e:
            sdblib.raster_join(P, 12, kw["eps"], x, x, None, z, None, kw["tile_bits"])
        assert e.value.status == sdblib.SDB_EINVAL


def test_raster_full_size(cuda, sdblib):
    """100M mobility points and the 263-zone tiling at eps 2^12 and 2^10: the
    raster join equals the covering join."""
    torch = cuda
    w = W.mobility_zones(100_000_000)
    T, pts = w.polygons, w.points
    x, y, a = dev(torch, pts.x), dev(torch, pts.y), dev(torch, pts.attr)
    for eps in (2 ** 12, 2 ** 10):
        cov = sdblib.build_covering(T, 24, eps)
        cnt = torch.zeros(T.n, dtype=torch.int64, device="cuda")
        sm = torch.zeros(T.n, dtype=torch.int64, device="cuda")
        sdblib.join_aggregate(x, y, a, cov, sdblib.LOOKUP_BINARY, cnt, sm)
        torch.cuda.synchronize()
        got = brj(torch, sdblib, T, 24, eps, pts, 0, x=x, y=y, a=a)
        assert np.array_equal(got[0], cnt.cpu().numpy().view(np.uint64))
        assert np.array_equal(got[1], sm.cpu().numpy())
