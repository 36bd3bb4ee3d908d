"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Nothing here retypes the oracle's formulas: every expected value comes from a
hand derivation (tests/golden), from a different formulation (fan
triangulation + separating axes for star-shaped polygons), from a curve
property, or from an invariant of the conservative raster (Sec. 2.2, Sec. 6).
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2010_12548_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def polys_of(rings, B):
    off, xs, ys = [0], [], []
    for r in rings:
        xs += [p[0] for p in r]
        ys += [p[1] for p in r]
        off.append(len(xs))
    return W.Polygons(np.array(off, np.uint32), np.array(xs, np.uint32), np.array(ys, np.uint32), B)


def lattice(B, attr=1):
    g = np.arange(2 ** B, dtype=np.uint32)
    gx, gy = np.meshgrid(g, g)
    return W.Points(gx.ravel(), gy.ravel(), np.full(gx.size, attr, np.int32), B)


# ---------------------------------------------------------------- Sec. 2.2 side

def test_finest_side_golden(orc):
    with open(os.path.join(GOLD, "finest_side.json")) as f:
        g = json.load(f)
    for c in g["cases"]:
        r = orc.finest_k(c["eps"], c["grid_bits"])
        if c["side"] is None:
            assert r is None, c
        else:
            assert r is not None and 2 ** r[0] == c["side"], (c, r)
            assert r[1] == c["grid_bits"] - r[0]


def test_finest_side_bracket(orc):
    # s*sqrt(2) <= eps < 2s*sqrt(2) whenever the grid does not cap s
    rng = np.random.default_rng(7)
    for eps in list(rng.integers(2, 2 ** 40, 400)) + [2 ** i for i in range(1, 40)]:
        k, _ = orc.finest_k(int(eps), 30) if int(eps) < 2 ** 31 else orc.finest_k(int(eps), 30)
        s = 2 ** k
        assert 2 * s * s <= int(eps) ** 2
        if k < 30:
            assert int(eps) ** 2 < 8 * s * s


# ---------------------------------------------------------------- Sec. 3 curve

@pytest.mark.parametrize("which", [0, 1])
def test_curve_bijection_and_prefix(orc, which):
    for order in range(1, 9):
        n = 2 ** order
        gx, gy = np.meshgrid(np.arange(n), np.arange(n))
        h = orc.curve(order, gx.ravel(), gy.ravel(), which)
        assert np.array_equal(np.sort(h), np.arange(n * n, dtype=np.uint64))
        for L in range(order + 1):
            hl = orc.curve(L, gx.ravel() >> (order - L), gy.ravel() >> (order - L), which)
            assert np.array_equal(h >> np.uint64(2 * (order - L)), hl)


def test_hilbert_adjacency_and_ends(orc):
    assert list(orc.curve(1, [0, 0, 1, 1], [0, 1, 1, 0])) == [0, 1, 2, 3]
    for order in range(1, 9):
        n = 2 ** order
        gx, gy = np.meshgrid(np.arange(n), np.arange(n))
        gx, gy = gx.ravel(), gy.ravel()
        h = orc.curve(order, gx, gy)
        o = np.argsort(h)
        step = np.abs(np.diff(gx[o])) + np.abs(np.diff(gy[o]))
        assert (step == 1).all()  # consecutive ids are 4-neighbours
        assert (gx[o[0]], gy[o[0]]) == (0, 0)
        assert (gx[o[-1]], gy[o[-1]]) == (n - 1, 0)


# ------------------------------------------------- hand-worked counts (golden)

def test_handworked_square_triangle(orc):
    with open(os.path.join(GOLD, "handworked_b4.json")) as f:
        g = json.load(f)
    B = g["grid_bits"]
    pts = lattice(B)
    for name, ring in g["polygons"].items():
        P = polys_of([ring], B)
        assert int(orc.join_exact(P, pts)[0][0]) == g["exact"][name]
        for c in g["cases"]:
            assert 2 ** orc.finest_k(c["eps"], B)[0] == c["side"]
            for which in (0, 1):
                cov = orc.cover(P, c["eps"], which)
                cnt, sm = cov.join(pts.x, pts.y, pts.attr)
                assert int(cnt[0]) == c[name] and int(sm[0]) == c[name], (name, c, which)
            cnt2, sm2, _ = orc.join_o2(P, c["eps"], pts)
            assert int(cnt2[0]) == c[name]


def test_points_outside_grid_ignored(orc):
    P = polys_of([[(0, 0), (15, 0), (15, 15), (0, 15)]], 4)
    pts = W.Points(np.array([0, 16, 3, 2 ** 31], np.uint32), np.array([0, 0, 16, 5], np.uint32),
                   np.array([1, 10, 100, 1000], np.int32), 4)
    cov = orc.cover(P, 2)
    assert cov.join(pts.x, pts.y, pts.attr)[0][0] == 1
    assert orc.join_o2(P, 2, pts)[0][0] == 1


# --------------------------------- star polygons: fan triangulation + SAT pin

def _orient(a, b, c):
    return (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])


def fan(P, j):
    rx, ry = P.ring(j)
    c = tuple(int(v) for v in P.centres[j])
    v = list(zip(rx.tolist(), ry.tolist()))
    return [(c, v[i], v[(i + 1) % len(v)]) for i in range(len(v))]


def tri_meets_square(t, x0, y0, x1, y1):
    xs = [p[0] for p in t]
    ys = [p[1] for p in t]
    if max(xs) < x0 or min(xs) > x1 or max(ys) < y0 or min(ys) > y1:
        return False
    corners = [(x0, y0), (x1, y0), (x1, y1), (x0, y1)]
    for i in range(3):
        a, b, c = t[i], t[(i + 1) % 3], t[(i + 2) % 3]
        sc = _orient(a, b, c)
        if all(_orient(a, b, q) * sc < 0 for q in corners):
            return False
    return True


def tri_has_point(t, p):
    a, b, c = t
    return _orient(a, b, p) >= 0 and _orient(b, c, p) >= 0 and _orient(c, a, p) >= 0


def small_stars(seed, B, n=6):
    rng = np.random.default_rng(seed)
    G = 2 ** B
    return W.star_polygons(rng, n, B, nverts=(3, 12), radius=(G / 16, G / 5))


@pytest.mark.parametrize("B,eps,seed", [(6, 2, 1), (6, 5, 2), (7, 12, 3), (8, 3, 4), (8, 23, 5)])
def test_star_cells_vs_fan_sat(orc, B, eps, seed):
    """O1 and O2 membership equals 'closed cell meets some closed fan triangle'."""
    P = small_stars(seed, B)
    pts = lattice(B)
    k, F = orc.finest_k(eps, B)
    s = 2 ** k
    for j in range(P.n):
        tris = fan(P, j)
        want = np.zeros(pts.n, bool)
        cells = {}
        for i in range(pts.n):
            cx, cy = int(pts.x[i]) >> k, int(pts.y[i]) >> k
            if (cx, cy) not in cells:
                x0, y0 = cx * s, cy * s
                cells[(cx, cy)] = any(tri_meets_square(t, x0, y0, x0 + s, y0 + s) for t in tris)
            want[i] = cells[(cx, cy)]
        _, _, _, mem = orc.join_o2(P, eps, pts, member=True, only=j)
        assert np.array_equal(mem.astype(bool), want), j
        one = P.subset([j])
        cnt, sm = orc.cover(one, eps).join(pts.x, pts.y, pts.attr)
        assert int(cnt[0]) == int(want.sum())


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_exact_pip_vs_fan(orc, seed):
    B = 7
    P = small_stars(seed, B)
    pts = lattice(B)
    for j in range(P.n):
        tris = fan(P, j)
        want = np.array([any(tri_has_point(t, (int(x), int(y))) for t in tris)
                         for x, y in zip(pts.x, pts.y)])
        _, _, mem = orc.join_exact(P, pts, member=True, only=j)
        assert np.array_equal(mem.astype(bool), want)


def test_classify_interior_cells_are_inside(orc):
    """A cell the oracle calls interior lies inside the fan union and touches
    no fan edge on the ring; a cell it calls exterior meets no fan triangle."""
    B = 8
    P = small_stars(21, B, n=4)
    rng = np.random.default_rng(5)
    for j in range(P.n):
        tris = fan(P, j)
        for side in (1, 2, 4, 8, 16):
            x0 = rng.integers(0, 2 ** B - side, 300) // side * side
            y0 = rng.integers(0, 2 ** B - side, 300) // side * side
            cls = orc.classify(P, j, x0, y0, side)
            for a, b, c in zip(x0.tolist(), y0.tolist(), cls.tolist()):
                meets = any(tri_meets_square(t, a, b, a + side, b + side) for t in tris)
                if c == 0:
                    assert not meets
                else:
                    assert meets
                if c == 1:
                    corners = [(a, b), (a + side, b), (a + side, b + side), (a, b + side)]
                    assert all(any(tri_has_point(t, q) for t in tris) for q in corners)


# ---------------------------------------------------- canonical covering form

@pytest.mark.parametrize("which", [0, 1])
def test_covering_is_canonical_and_exact_cell_set(orc, which):
    B = 6
    P = small_stars(31, B, n=5)
    for eps in (2, 6, 23):
        k, F = orc.finest_k(eps, B)
        cov = orc.cover(P, eps, which)
        st, lo, ids = cov.start, cov.list_off, cov.list_ids
        assert st[0] == 0 and st[-1] == 4 ** F
        assert (np.diff(st.astype(np.int64)) > 0).all()
        lists = [tuple(ids[lo[r]:lo[r + 1]]) for r in range(cov.R)]
        for r in range(cov.R):
            assert list(lists[r]) == sorted(set(lists[r]))
            if r:
                assert lists[r] != lists[r - 1]
        # decode: every finest cell's list equals the set of polygons it meets
        n = 2 ** F
        gx, gy = np.meshgrid(np.arange(n), np.arange(n))
        gx, gy = gx.ravel(), gy.ravel()
        h = orc.curve(F, gx, gy, which)
        r_of = np.searchsorted(st, h, side="right") - 1
        s = 2 ** k
        for j in range(P.n):
            cls = orc.classify(P, j, gx * s, gy * s, s)
            inlist = np.array([j in lists[r] for r in r_of])
            assert np.array_equal(inlist, cls != 0)


# ------------------------------------------- result range estimation (Sec. 6)

def test_handworked_boundary_counts(orc):
    """Boundary-cell point counts derived by hand (tests/golden/handworked_b4.json):
    the flagged covering's O1 join and the definitional O2 test both match."""
    with open(os.path.join(GOLD, "handworked_b4.json")) as f:
        g = json.load(f)
    B = g["grid_bits"]
    pts = lattice(B)
    for name, ring in g["polygons"].items():
        P = polys_of([ring], B)
        for c in g["cases"]:
            want = c["boundary"][name]
            for which in (0, 1):
                cov = orc.cover(P, c["eps"], which, flagged=True)
                cnt, sm, bc, bs, ba = cov.join_range(pts.x, pts.y, pts.attr)
                assert int(cnt[0]) == c[name] and int(bc[0]) == want, (name, c, which)
                assert int(bs[0]) == want and int(ba[0]) == want
            assert int(orc.join_o2(P, c["eps"], pts)[2][0]) == want


def _merge_plain(cov):
    """Strip the boundary flags and merge equal neighbours."""
    st, lo, ids = cov.start, cov.list_off, cov.list_ids
    starts, lists = [], []
    for r in range(cov.R):
        lst = tuple(int(e) & 0x7FFFFFFF for e in ids[lo[r]:lo[r + 1]])
        if lists and lists[-1] == lst:
            continue
        starts.append(int(st[r]))
        lists.append(lst)
    return starts + [int(st[-1])], lists


@pytest.mark.parametrize("which", [0, 1])
def test_flagged_covering_cell_by_cell(orc, which):
    """Every finest cell of the flagged covering: polygon j is on its list iff the
    cell meets j, and flagged iff the cell meets j's boundary (classify, a
    separate predicate from the sweep); without flags it is the plain covering."""
    B = 6
    P = small_stars(31, B, n=5)
    for eps in (2, 6, 23):
        k, F = orc.finest_k(eps, B)
        cf = orc.cover(P, eps, which, flagged=True)
        cp = orc.cover(P, eps, which)
        st, lo, ids = cf.start, cf.list_off, cf.list_ids
        lists = [tuple(int(e) for e in ids[lo[r]:lo[r + 1]]) for r in range(cf.R)]
        assert st[0] == 0 and st[-1] == 4 ** F
        for r in range(cf.R):
            polys = [e & 0x7FFFFFFF for e in lists[r]]
            assert polys == sorted(set(polys))
            if r:
                assert lists[r] != lists[r - 1]
        n = 2 ** F
        gx, gy = np.meshgrid(np.arange(n), np.arange(n))
        gx, gy = gx.ravel(), gy.ravel()
        h = orc.curve(F, gx, gy, which)
        r_of = np.searchsorted(st, h, side="right") - 1
        s = 2 ** k
        for j in range(P.n):
            cls = orc.classify(P, j, gx * s, gy * s, s)
            inlist = np.array([j in [e & 0x7FFFFFFF for e in lists[r]] for r in r_of])
            flagged = np.array([(j | 0x80000000) in lists[r] for r in r_of])
            assert np.array_equal(inlist, cls != 0)
            assert np.array_equal(flagged, cls == 2)
        ps, pl = _merge_plain(cf)
        assert ps == [int(v) for v in cp.start]
        assert pl == [tuple(int(e) for e in cp.list_ids[cp.list_off[r]:cp.list_off[r + 1]])
                      for r in range(cp.R)]


def test_range_bounds_signed_attributes(orc):
    """Sec. 6 with signed attributes: the flagged O1 partials equal the
    definitional O2 ones, and the exact COUNT and SUM (exact point-in-polygon
    join) lie in the intervals, whose widths are bcount and babs."""
    w = W.tiny_stars(20_000)
    rng = np.random.default_rng(5)
    attr = rng.integers(-2 ** 31, 2 ** 31, size=w.points.n, dtype=np.int64).astype(np.int32)
    attr[:4] = [-2 ** 31, 2 ** 31 - 1, 0, -1]
    pts = W.Points(w.points.x, w.points.y, attr, w.points.grid_bits)
    P = w.polygons
    ex, exs = orc.join_exact(P, pts)
    for eps in (4096, 512, 64, 8):
        cov = orc.cover(P, eps, flagged=True)
        c, s, bc, bs, ba = cov.join_range(pts.x, pts.y, pts.attr)
        c2, s2, b2, bs2, ba2 = orc.join_o2(P, eps, pts, boundary_sums=True)
        for u, v in ((c, c2), (s, s2), (bc, b2), (bs, bs2), (ba, ba2)):
            assert np.array_equal(u, v), eps
        lo_c, hi_c, lo_s, hi_s = orc.range_bounds(c, s, bc, bs, ba)
        assert ((lo_c <= ex) & (ex <= hi_c)).all()
        assert ((lo_s <= exs) & (exs <= hi_s)).all()
        assert np.array_equal(hi_c - lo_c, bc.astype(np.int64))
        assert np.array_equal(hi_s - lo_s, ba.astype(np.int64))


# ----------------------------------------------- point indexing (Sec. 3)

def test_point_index_handworked(orc):
    """Sorted keys + prefix sums over the covering's ranges give the hand-derived
    counts (tests/golden/handworked_b4.json)."""
    with open(os.path.join(GOLD, "handworked_b4.json")) as f:
        g = json.load(f)
    B = g["grid_bits"]
    pts = lattice(B)
    for name, ring in g["polygons"].items():
        P = polys_of([ring], B)
        for c in g["cases"]:
            for which in (0, 1):
                cnt, sm = orc.cover(P, c["eps"], which).point_index_aggregate(pts.x, pts.y,
                                                                              pts.attr)
                assert int(cnt[0]) == c[name] and int(sm[0]) == c[name], (name, c, which)


@pytest.mark.parametrize("which", [0, 1])
def test_point_index_equals_point_stream(orc, which):
    """Range counting over sorted points (two lower bounds per range) equals the
    per-point lookup join exactly: overlapping stars, duplicated points, points
    outside the grid, signed attributes, several eps (F = 0 included)."""
    w = W.tiny_stars(30_000)
    rng = np.random.default_rng(8)
    x = np.concatenate([w.points.x, w.points.x[:500], [2 ** 16, 3]]).astype(np.uint32)
    y = np.concatenate([w.points.y, w.points.y[:500], [5, 2 ** 20]]).astype(np.uint32)
    a = rng.integers(-2 ** 31, 2 ** 31, len(x), dtype=np.int64).astype(np.int32)
    for eps in (2 ** 17, 4096, 300, 64, 5):
        cov = orc.cover(w.polygons, eps, which)
        want = cov.join(x, y, a)
        got = cov.point_index_aggregate(x, y, a)
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1]), eps
        fl = orc.cover(w.polygons, eps, which, flagged=True).point_index_aggregate(x, y, a)
        assert np.array_equal(fl[0], want[0]) and np.array_equal(fl[1], want[1]), eps


# ------------------------------------- non-conservative raster (Sec. 2.2)

def multi_of(polys, B):
    """MultiPolygons from a list of polygons, each a list of rings."""
    pro, roff, xs, ys = [0], [0], [], []
    for rings in polys:
        for r in rings:
            xs += [p[0] for p in r]
            ys += [p[1] for p in r]
            roff.append(len(xs))
        pro.append(len(roff) - 1)
    return W.MultiPolygons(np.array(pro, np.uint32), np.array(roff, np.uint32),
                           np.array(xs, np.uint32), np.array(ys, np.uint32), B)


def test_noncons_handworked(orc):
    """Hand-derived non-conservative counts (centre rule) of both golden files."""
    for fname, make in (("handworked_b4.json", lambda ring, B: polys_of([ring], B)),
                        ("handworked_holes_b4.json", lambda rings, B: multi_of([rings], B))):
        with open(os.path.join(GOLD, fname)) as f:
            g = json.load(f)
        B = g["grid_bits"]
        pts = lattice(B)
        for name, shape in g["polygons"].items():
            P = make(shape, B)
            for c in g["cases"]:
                want = c["noncons"][name]
                for which in (0, 1):
                    cnt, sm = orc.cover(P, c["eps"], which, noncons=True).join(pts.x, pts.y,
                                                                               pts.attr)
                    assert int(cnt[0]) == want and int(sm[0]) == want, (name, c, which)
                assert int(orc.join_o2(P, c["eps"], pts, noncons=True)[0][0]) == want


def test_noncons_o1_o2_and_eps_bound(orc, stars_small):
    """Non-conservative covering join = definitional test; every false negative
    and false positive lies within eps of the boundary; never more than the
    conservative count."""
    w = stars_small
    P, pts = w.polygons, w.points
    for eps in (64, 200, 1000):
        cons = orc.join_o2(P, eps, pts)[0]
        want = orc.join_o2(P, eps, pts, noncons=True)
        assert (want[0] <= cons).all()
        for which in (0, 1):
            got = orc.cover(P, eps, which, noncons=True).join(pts.x, pts.y, pts.attr)
            assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
        for j in range(P.n):
            _, _, _, am = orc.join_o2(P, eps, pts, member=True, only=j, noncons=True)
            _, _, em = orc.join_exact(P, pts, member=True, only=j)
            for i in np.nonzero(am.astype(bool) != em.astype(bool))[0]:
                assert orc.near_boundary(P, j, int(pts.x[i]), int(pts.y[i]), eps)


# ----------------------------------- multi-polygons and holes (Sec. 5.2)

def test_holes_handworked(orc):
    with open(os.path.join(GOLD, "handworked_holes_b4.json")) as f:
        g = json.load(f)
    B = g["grid_bits"]
    pts = lattice(B)
    for name, rings in g["polygons"].items():
        P = multi_of([rings], B)
        assert int(orc.join_exact(P, pts)[0][0]) == g["exact"][name]
        for c in g["cases"]:
            for which in (0, 1):
                cnt, sm = orc.cover(P, c["eps"], which).join(pts.x, pts.y, pts.attr)
                assert int(cnt[0]) == c[name] and int(sm[0]) == c[name], (name, c, which)
            assert int(orc.join_o2(P, c["eps"], pts)[0][0]) == c[name]


def test_multi_classify_is_ring_combination(orc):
    """A polygon of several rings classifies a cell as: boundary when any ring
    does; otherwise interior when an odd number of its rings contain the cell
    (even-odd region), else exterior -- checked against the single-ring
    classification of each ring."""
    B = 12
    M = W.holed_stars(np.random.default_rng(21), 12, B, radius=(2 ** 7, 2 ** 8))
    rings = W.Polygons(M.ring_off, M.x, M.y, B)
    rng = np.random.default_rng(22)
    for side in (1, 8, 64, 512):
        x0 = rng.integers(0, 2 ** B - side, 3000) // side * side
        y0 = rng.integers(0, 2 ** B - side, 3000) // side * side
        for j in range(M.n):
            got = orc.classify(M, j, x0, y0, side)
            cls = [orc.classify(rings, r, x0, y0, side)
                   for r in range(M.poly_ring_off[j], M.poly_ring_off[j + 1])]
            bnd = np.any([c == 2 for c in cls], axis=0)
            odd = (np.sum([c == 1 for c in cls], axis=0) % 2) == 1
            want = np.where(bnd, 2, np.where(odd, 1, 0))
            assert np.array_equal(got, want), (side, j)


def test_multi_o1_o2_exact(orc):
    """Holed and multi-part stars: covering join = definitional test (both
    curves, conservative and non-conservative); the exact join never exceeds
    the conservative one, and its misses are within eps."""
    B = 14
    M = W.holed_stars(np.random.default_rng(31), 10, B, radius=(2 ** 8, 2 ** 9))
    rng = np.random.default_rng(32)
    pts = W.Points(rng.integers(0, 2 ** B, 40_000, dtype=np.uint32),
                   rng.integers(0, 2 ** B, 40_000, dtype=np.uint32),
                   rng.integers(-1000, 1000, 40_000).astype(np.int32), B)
    ex = orc.join_exact(M, pts)
    for eps in (3, 40, 300):
        for nc in (False, True):
            want = orc.join_o2(M, eps, pts, noncons=nc)
            for which in (0, 1):
                got = orc.cover(M, eps, which, noncons=nc).join(pts.x, pts.y, pts.attr)
                assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
            if not nc:
                assert (ex[0] <= want[0]).all()
        for j in range(M.n):
            _, _, _, am = orc.join_o2(M, eps, pts, member=True, only=j)
            _, _, em = orc.join_exact(M, pts, member=True, only=j)
            am, em = am.astype(bool), em.astype(bool)
            assert not np.any(em & ~am)
            for i in np.nonzero(am & ~em)[0][:50]:
                assert orc.near_boundary(M, j, int(pts.x[i]), int(pts.y[i]), eps)


# ------------------------------------------------------ invariants (Sec. 2.2, 6)

@pytest.fixture(scope="module")
def stars_small():
    w = W.tiny_stars(20_000)
    return w


def test_no_false_negatives_and_eps_bound(orc, stars_small):
    """I1: exact is contained in the approximation (conservative raster).
    I2: every false positive lies within eps of the polygon's boundary."""
    w = stars_small
    P, pts = w.polygons, w.points
    for eps in (64, 200, 1000):
        for j in range(P.n):
            _, _, _, am = orc.join_o2(P, eps, pts, member=True, only=j)
            _, _, em = orc.join_exact(P, pts, member=True, only=j)
            am, em = am.astype(bool), em.astype(bool)
            assert not np.any(em & ~am)
            for i in np.nonzero(am & ~em)[0]:
                assert orc.near_boundary(P, j, int(pts.x[i]), int(pts.y[i]), eps)


def test_monotone_in_eps_and_result_range(orc, stars_small):
    """I3: halving eps never adds a point (finest covered sets nest).
    I4 (Sec. 6): exact count lies in [alpha - beta, alpha], beta = points in
    boundary cells."""
    w = stars_small
    P, pts = w.polygons, w.points
    ex, exs = orc.join_exact(P, pts)
    prev = None
    for eps in (4096, 2048, 1024, 512, 256, 128, 64, 32, 16, 8, 4, 2):
        a, s, b = orc.join_o2(P, eps, pts)
        assert (a - b <= ex).all() and (ex <= a).all()
        if prev is not None:
            assert (a <= prev).all()
        prev = a


def test_hilbert_vs_z_same_counts(orc, stars_small):
    """I6: counts do not depend on the curve; the ranges do."""
    w = stars_small
    for eps in (64, 300):
        ch = orc.cover(w.polygons, eps, 0)
        cz = orc.cover(w.polygons, eps, 1)
        a = ch.join(w.points.x, w.points.y, w.points.attr)
        b = cz.join(w.points.x, w.points.y, w.points.attr)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        assert not np.array_equal(ch.start[:10], cz.start[:10])
        o2 = orc.join_o2(w.polygons, eps, w.points)
        assert np.array_equal(a[0], o2[0]) and np.array_equal(a[1], o2[1])


def test_convergence_to_exact(orc):
    """As the grid is refined around a fixed instance, the s=1 counts fall to
    the exact counts; once the cell side drops below the smallest nonzero
    lattice-point distance (vertices < 2^b: m >= b+2) they are equal."""
    b = 5
    P0 = small_stars(41, b, n=4)
    pts0 = lattice(b)
    ex = orc.join_exact(P0, pts0)[0]
    prev = None
    for m in range(0, b + 4):
        P = W.Polygons(P0.ring_off, P0.x << m, P0.y << m, b + m)
        pts = W.Points(pts0.x << m, pts0.y << m, pts0.attr, b + m)
        cnt = orc.cover(P, 2).join(pts.x, pts.y)[0]
        assert (cnt >= ex).all()
        if prev is not None:
            assert (cnt <= prev).all()
        if m >= b + 2:
            assert np.array_equal(cnt, ex)
        prev = cnt


def test_tiling_every_point_covered(orc):
    """I5: a tiling covers every lattice point exactly and approximately, and
    points strictly inside one tile's interior get exactly one polygon."""
    rng = np.random.default_rng(3)
    T = W.voronoi_tiling(rng, 12, 10, nverts=(6, 20), min_piece=4.0)
    pts = lattice(10)
    _, _, em = orc.join_exact(T, pts, member=True)
    assert em.all()
    cov = orc.cover(T, 8)
    cnt, _ = cov.join(pts.x, pts.y, pts.attr)
    ex = orc.join_exact(T, pts)[0]
    assert cnt.sum() >= pts.n and ex.sum() >= pts.n
    o2 = orc.join_o2(T, 8, pts)
    assert np.array_equal(cnt, o2[0])


def test_near_boundary_vs_float_distance(orc):
    """The exact eps-distance test agrees with a float64 point-to-segment
    distance wherever the two are not within rounding of the threshold."""
    rng = np.random.default_rng(9)
    P = small_stars(51, 10, n=3)
    checked = 0
    for j in range(P.n):
        rx, ry = P.ring(j)
        ax, ay = rx.astype(float), ry.astype(float)
        bx, by = np.roll(ax, -1), np.roll(ay, -1)
        for _ in range(300):
            px, py = rng.integers(0, 2 ** 10, 2)
            eps = int(rng.integers(1, 200))
            dx, dy = bx - ax, by - ay
            t = np.clip(((px - ax) * dx + (py - ay) * dy) / (dx * dx + dy * dy), 0, 1)
            d = np.min(np.hypot(ax + t * dx - px, ay + t * dy - py))
            if abs(d - eps) < 1e-6 * max(1.0, eps):
                continue
            assert orc.near_boundary(P, j, int(px), int(py), eps) == (d <= eps)
            checked += 1
    assert checked > 800
