"""Non-conservative coverings and polygons of several rings (holes,
multi-polygons) on the GPU vs the CPU oracle.

Coverings must equal the oracle's entry for entry and joins bit for bit; the
raster join on multi-polygons must equal the definitional test.
"""
import json
import os

import numpy as np
import pytest

from paper_2010_12548_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")
NONCONS = 2  # COVER_NONCONSERVATIVE


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


def join(torch, sdb, cov, pts, lookup):
    P = cov.info().n_polygons
    cnt = torch.full((P,), 7, dtype=torch.int64, device="cuda")
    sm = torch.full((P,), 7, dtype=torch.int64, device="cuda")
    sdb.join_aggregate(dev(torch, pts.x), dev(torch, pts.y), dev(torch, pts.attr), cov, lookup,
                       cnt, sm)
    torch.cuda.synchronize()
    return cnt.cpu().numpy().view(np.uint64), sm.cpu().numpy()


def raster(torch, sdb, polys, B, eps, pts, tile_bits=0):
    P = polys.n
    cnt = torch.full((P,), 7, dtype=torch.int64, device="cuda")
    sm = torch.full((P,), 7, dtype=torch.int64, device="cuda")
    sdb.raster_join(polys, B, eps, dev(torch, pts.x), dev(torch, pts.y), dev(torch, pts.attr), cnt,
                    sm, tile_bits)
    torch.cuda.synchronize()
    return cnt.cpu().numpy().view(np.uint64), sm.cpu().numpy()


def same_covering(sdb, cov, oc):
    st, lo, ids = sdb.covering_export(cov)
    return (np.array_equal(st, oc.start) and np.array_equal(lo, oc.list_off)
            and np.array_equal(ids, oc.list_ids))


def lattice(B):
    g = np.arange(2 ** B, dtype=np.uint32)
    gx, gy = np.meshgrid(g, g)
    return W.Points(gx.ravel(), gy.ravel(), np.ones(gx.size, np.int32), B)


def single(rings, B):
    off, xs, ys = [0], [], []
    for r in rings:
        xs += [p[0] for p in r]
        ys += [p[1] for p in r]
        off.append(len(xs))
    return W.Polygons(np.array(off, np.uint32), np.array(xs, np.uint32), np.array(ys, np.uint32), B)


def multi(polys, B):
    pro, roff, xs, ys = [0], [0], [], []
    for rings in polys:
        for r in rings:
            xs += [p[0] for p in r]
            ys += [p[1] for p in r]
            roff.append(len(xs))
        pro.append(len(roff) - 1)
    return W.MultiPolygons(np.array(pro, np.uint32), np.array(roff, np.uint32),
                           np.array(xs, np.uint32), np.array(ys, np.uint32), B)


def test_golden_noncons_and_holes(cuda, sdblib):
    torch = cuda
    cases = [("handworked_b4.json", lambda shape, B: single([shape], B)),
             ("handworked_holes_b4.json", lambda shape, B: multi([shape], B))]
    for fname, make in cases:
        with open(os.path.join(GOLD, fname)) as f:
            g = json.load(f)
        B = g["grid_bits"]
        pts = lattice(B)
        for name, shape in g["polygons"].items():
            P = make(shape, B)
            for c in g["cases"]:
                for flags, want in ((0, c[name]), (NONCONS, c["noncons"][name])):
                    cov = sdblib.build_covering(P, B, c["eps"], flags=flags)
                    sdblib.covering_build_index(cov, 4)
                    for lookup in (0, 1):
                        cnt, sm = join(torch, sdblib, cov, pts, lookup)
                        assert int(cnt[0]) == want and int(sm[0]) == want, (name, c, flags)
                for tb in (0, 1):
                    cnt, sm = raster(torch, sdblib, P, B, c["eps"], pts, tb)
                    assert int(cnt[0]) == c[name] and int(sm[0]) == c[name], (name, c, tb)


@pytest.mark.parametrize("B,eps,seed", [(8, 3, 1), (10, 2, 2), (12, 9, 3), (16, 64, 4),
                                        (16, 700, 5), (12, 2 ** 13, 6)])
def test_noncons_stars_vs_oracle(cuda, sdblib, orc, B, eps, seed):
    rng = np.random.default_rng(seed)
    G = 2 ** B
    P = W.star_polygons(rng, 9, B, nverts=(3, 16), radius=(G / 16, G / 4))
    pts = W.Points(rng.integers(0, G, 20_000, dtype=np.uint32),
                   rng.integers(0, G, 20_000, dtype=np.uint32),
                   rng.integers(-1000, 1000, 20_000).astype(np.int32), B)
    oc = orc.cover(P, eps, noncons=True)
    cov = sdblib.build_covering(P, B, eps, flags=NONCONS)
    assert same_covering(sdblib, cov, oc)
    want = orc.join_o2(P, eps, pts, noncons=True)
    sdblib.covering_build_index(cov, 6)
    for lookup in (0, 1):
        got = join(cuda, sdblib, cov, pts, lookup)
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


def test_noncons_zones(cuda, sdblib, orc):
    T = W.zones263_tiling()
    pts = W.mobility_points(W.BASE_SEED + 11, 1_000_003, 24, 32)
    for eps in (2 ** 12, 2 ** 10):
        oc = orc.cover(T, eps, noncons=True)
        cov = sdblib.build_covering(T, 24, eps, flags=NONCONS)
        assert same_covering(sdblib, cov, oc)
        sdblib.covering_build_index(cov, 12)
        want = oc.join(pts.x, pts.y, pts.attr)
        got = join(cuda, sdblib, cov, pts, 1)
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


@pytest.mark.parametrize("B,eps,seed", [(12, 2, 1), (14, 40, 2), (14, 300, 3), (16, 90, 4),
                                        (12, 2 ** 13, 5)])
def test_multipolygons_vs_oracle(cuda, sdblib, orc, B, eps, seed):
    """Holed and multi-part stars: conservative, flagged and non-conservative
    coverings, both lookups, and the raster join."""
    torch = cuda
    M = W.holed_stars(np.random.default_rng(seed), 12, B,
                      radius=(2 ** (B - 6), 2 ** (B - 5)))
    rng = np.random.default_rng(seed + 100)
    pts = W.Points(rng.integers(0, 2 ** B, 30_000, dtype=np.uint32),
                   rng.integers(0, 2 ** B, 30_000, dtype=np.uint32),
                   rng.integers(-1000, 1000, 30_000).astype(np.int32), B)
    for flags, kw in ((0, {}), (1, {"flagged": True}), (NONCONS, {"noncons": True})):
        oc = orc.cover(M, eps, **kw)
        cov = sdblib.build_covering(M, B, eps, flags=flags)
        assert same_covering(sdblib, cov, oc), flags
        want = orc.join_o2(M, eps, pts, noncons=flags == NONCONS)
        sdblib.covering_build_index(cov, 6)
        for lookup in (0, 1):
            got = join(torch, sdblib, cov, pts, lookup)
            assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1]), flags
    want = orc.join_o2(M, eps, pts)
    F = orc.finest_k(eps, B)[1]
    for tb in sorted({0, max(1, F - 8), min(13, max(1, F - 2))}):
        got = raster(torch, sdblib, M, B, eps, pts, tb)
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1]), tb


def test_noncons_full_size_sampled(cuda, sdblib, orc):
    """eps = 2^6 on the 263-zone tiling: the non-conservative covering joined
    with a 2M-point sample of the 100M points equals the definitional test,
    and over all 100M points never exceeds the conservative counts."""
    torch = cuda
    w = W.mobility_zones(100_000_000)
    T = w.polygons
    cons = sdblib.build_covering(T, 24, 64)
    nc = sdblib.build_covering(T, 24, 64, flags=NONCONS)
    sdblib.covering_build_index(nc, 20)
    sdblib.covering_build_index(cons, 20)
    a = join(torch, sdblib, nc, w.points, 1)
    b = join(torch, sdblib, cons, w.points, 1)
    assert (a[0] <= b[0]).all()
    rng = np.random.default_rng(17)
    sample = w.points.take(np.sort(rng.choice(w.points.n, 2_000_000, replace=False)))
    want = orc.join_o2(T, 64, sample, threads=16, noncons=True)
    got = join(torch, sdblib, nc, sample, 1)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
