"""Batched level-of-detail queries vs the CPU oracle.

Each query's slice must equal the oracle's definitional join of the query's
polygon subset at its eps over the points inside its viewport, bit for bit, in
every launch mode, alone or in the mix, with binary search or with the
per-query learned index (which must report no fallback).
"""
import numpy as np
import pytest

from paper_2010_12548_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


def run_batch(torch, sdb, b, mode, stream=None):
    n = b.info().out_len
    cnt = torch.full((max(n, 1),), 5, dtype=torch.int64, device="cuda")
    sm = torch.full((max(n, 1),), 5, dtype=torch.int64, device="cuda")
    sdb.batch_run(b, mode, cnt, sm, stream)
    torch.cuda.synchronize()
    return cnt.cpu().numpy()[:n].view(np.uint64), sm.cpu().numpy()[:n]


def oracle_slice(orc, T, pts, row, ids):
    x0, y0, x1, y1, eps, off, k = (int(v) for v in row)
    if k == 0:
        return np.zeros(0, np.uint64), np.zeros(0, np.int64)
    inside = (pts.x >= x0) & (pts.x < x1) & (pts.y >= y0) & (pts.y < y1)
    sub = T.subset(ids[off:off + k])
    c, s, _ = orc.join_o2(sub, eps, pts.take(np.nonzero(inside)[0]), threads=8)
    return c, s


def check_all(orc, T, pts, rows, ids, cnt, sm, which=None):
    out = 0
    for q, row in enumerate(rows):
        k = int(row[6])
        if which is None or q in which:
            c, s = oracle_slice(orc, T, pts, row, ids)
            assert np.array_equal(cnt[out:out + k], c), q
            assert np.array_equal(sm[out:out + k], s), q
        out += k


@pytest.fixture(scope="module")
def small(cuda, sdblib):
    torch = cuda
    rng = np.random.default_rng(11)
    T = W.voronoi_tiling(rng, 600, 20, nverts=(6, 40))
    pts = W.mobility_points(W.BASE_SEED + 77, 1_000_003, 20, 16, sigma=(2 ** 12, 2 ** 15))
    qb = W.lod_queries(5, 48, T, side=(2 ** 6, 2 ** 18), subset=(1, 300),
                       eps_levels=tuple(2 ** e for e in range(10, 0, -1)))
    rows = [tuple(r) for r in qb.queries]
    G = 2 ** 20
    off = len(qb.subset_ids)
    extra_ids = list(range(600))
    rows += [
        (0, 0, G, G, 2 ** 25, off, 50),           # whole grid, one cell (finest level 0)
        (5, 7, 6, 8, 2, off, 600),                # one lattice point, finest side 1
        (1000, 1000, 9000, 9000, 64, off, 0),     # empty subset
        (0, 0, G, G, 2 ** 12, off + 10, 1),       # whole grid, one polygon
    ]
    ids = np.concatenate([qb.subset_ids, np.asarray(extra_ids, np.uint32)])
    p = sdblib.points_create(dev(torch, pts.x), dev(torch, pts.y), dev(torch, pts.attr), 20)
    b = sdblib.batch_create(p, T, rows, ids)
    return T, pts, rows, ids, b


def test_batch_vs_oracle_all_modes(cuda, sdblib, orc, small):
    torch = cuda
    T, pts, rows, ids, b = small
    inf = b.info()
    assert inf.n_queries == len(rows) and inf.out_len == sum(r[6] for r in rows)
    cnt, sm = run_batch(torch, sdblib, b, sdblib.BATCH_PERSISTENT)
    check_all(orc, T, pts, rows, ids, cnt, sm)
    s = torch.cuda.Stream()
    for mode in (sdblib.BATCH_PER_QUERY, sdblib.BATCH_GRAPH, sdblib.BATCH_GRAPH):
        with torch.cuda.stream(s):
            c2, s2 = run_batch(torch, sdblib, b, mode, stream=s)
        assert np.array_equal(c2, cnt) and np.array_equal(s2, sm), mode


def test_batch_tuning_keeps_results(cuda, sdblib, small):
    torch = cuda
    T, pts, rows, ids, b = small
    ref = run_batch(torch, sdblib, b, sdblib.BATCH_PERSISTENT)
    for tile, ppt in ((1, 1), (37, 2), (100000, 4), (4096, 2)):
        sdblib.batch_set_tuning(b, tile, ppt)
        got = run_batch(torch, sdblib, b, sdblib.BATCH_PERSISTENT)
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), (tile, ppt)
    tile, ppt = sdblib.batch_autotune(b)
    assert tile in (1024, 4096, 16384) and ppt in (1, 2, 4)
    got = run_batch(torch, sdblib, b, sdblib.BATCH_PERSISTENT)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


def test_query_alone_equals_in_mix(cuda, sdblib, small):
    torch = cuda
    T, pts, rows, ids, b = small
    cnt, sm = run_batch(torch, sdblib, b, sdblib.BATCH_PERSISTENT)
    offs = np.concatenate([[0], np.cumsum([r[6] for r in rows])])
    for q in (0, 7, 19, len(rows) - 1):
        r = list(rows[q])
        sub = ids[r[5]:r[5] + r[6]]
        r[5] = 0
        b1 = sdblib.batch_create(b.points, T, [tuple(r)], sub)
        c1, s1 = run_batch(torch, sdblib, b1, sdblib.BATCH_PERSISTENT)
        assert np.array_equal(c1, cnt[offs[q]:offs[q + 1]])
        assert np.array_equal(s1, sm[offs[q]:offs[q + 1]])


def test_overlapping_polygons(cuda, sdblib, orc):
    """One query over nested polygons takes the general merge and is exact;
    several queries require polygons that do not overlap within a query."""
    torch = cuda
    rng = np.random.default_rng(3)
    # a square inside another square
    S = W.Polygons(np.array([0, 4, 8], np.uint32),
                   np.array([100, 5000, 5000, 100, 2000, 3000, 3000, 2000], np.uint32),
                   np.array([100, 100, 5000, 5000, 2000, 2000, 3000, 3000], np.uint32), 14)
    pts = W.uniform_points(rng, 10_000, 14)
    p = sdblib.points_create(dev(torch, pts.x), dev(torch, pts.y), dev(torch, pts.attr), 14)
    row = (50, 60, 9000, 8000, 16, 0, 2)
    b = sdblib.batch_create(p, S, [row], np.arange(2))
    cnt, sm = run_batch(torch, sdblib, b, sdblib.BATCH_PERSISTENT)
    c, s_ = oracle_slice(orc, S, pts, row, np.arange(2))
    assert np.array_equal(cnt, c) and np.array_equal(sm, s_)
    with pytest.raises(sdblib.SdbError) as e:
        sdblib.batch_create(p, S, [row, row], np.arange(2))
    assert e.value.status == sdblib.SDB_EINVAL


def test_lod_workload_full_size_sampled(cuda, sdblib, orc):
    """4,096 queries over 200M points and the 40,000-polygon tiling; sampled
    queries against the oracle."""
    torch = cuda
    T, pts, qb = W.lod_workload()
    rows = [tuple(r) for r in qb.queries]
    p = sdblib.points_create(dev(torch, pts.x), dev(torch, pts.y), dev(torch, pts.attr), 28)
    b = sdblib.batch_create(p, T, rows, qb.subset_ids)
    sdblib.batch_autotune(b)
    cnt, sm = run_batch(torch, sdblib, b, sdblib.BATCH_PERSISTENT)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        c2, s2 = run_batch(torch, sdblib, b, sdblib.BATCH_GRAPH, stream=s)
    assert np.array_equal(c2, cnt) and np.array_equal(s2, sm)
    rng = np.random.default_rng(0)
    ranges = b.query_ranges()
    # the largest coverings, the smallest, and random ones
    order = np.argsort(ranges)
    sample = set(order[:3].tolist()) | set(order[-3:].tolist()) | set(
        rng.choice(len(rows), 10, replace=False).tolist())
    check_all(orc, T, pts, rows, qb.subset_ids, cnt, sm, which=sample)


def test_learned_batch_vs_oracle(cuda, sdblib, orc, small):
    """The per-query learned index: the same results as binary search in every
    mode, after tuning changes, and equal to the oracle; no fallback; switching
    back to binary search gives the same results again."""
    torch = cuda
    T, pts, rows, ids, b = small
    ref = run_batch(torch, sdblib, b, sdblib.BATCH_PERSISTENT)
    sdblib.batch_set_lookup(b, sdblib.LOOKUP_LEARNED)
    inf = b.info()
    assert inf.lookup == sdblib.LOOKUP_LEARNED and inf.indexed_queries > 0 and inf.n_leaves > 0
    got = run_batch(torch, sdblib, b, sdblib.BATCH_PERSISTENT)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    assert sdblib.batch_fallbacks(b) == 0
    check_all(orc, T, pts, rows, ids, got[0], got[1])
    s = torch.cuda.Stream()
    for mode in (sdblib.BATCH_PER_QUERY, sdblib.BATCH_GRAPH, sdblib.BATCH_GRAPH):
        with torch.cuda.stream(s):
            c2, s2 = run_batch(torch, sdblib, b, mode, stream=s)
        assert np.array_equal(c2, ref[0]) and np.array_equal(s2, ref[1]), mode
        assert sdblib.batch_fallbacks(b, s) == 0
    for tile, ppt in ((1, 1), (37, 2), (4096, 4)):
        sdblib.batch_set_tuning(b, tile, ppt)
        got = run_batch(torch, sdblib, b, sdblib.BATCH_PERSISTENT)
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), (tile, ppt)
    sdblib.batch_set_lookup(b, sdblib.LOOKUP_BINARY)
    assert b.info().lookup == sdblib.LOOKUP_BINARY and b.info().n_leaves == 0
    got = run_batch(torch, sdblib, b, sdblib.BATCH_PERSISTENT)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    with pytest.raises(sdblib.SdbError) as e:
        sdblib.batch_set_lookup(b, sdblib.LOOKUP_TABLE)
    assert e.value.status == sdblib.SDB_EINVAL


def test_learned_lod_full_size(cuda, sdblib, orc):
    """The 4,096-query level-of-detail batch over 200M points: learned equals
    binary search for every query, no fallback, sampled queries vs the oracle."""
    torch = cuda
    T, pts, qb = W.lod_workload()
    rows = [tuple(r) for r in qb.queries]
    p = sdblib.points_create(dev(torch, pts.x), dev(torch, pts.y), dev(torch, pts.attr), 28)
    b = sdblib.batch_create(p, T, rows, qb.subset_ids)
    ref = run_batch(torch, sdblib, b, sdblib.BATCH_PERSISTENT)
    sdblib.batch_set_lookup(b, sdblib.LOOKUP_LEARNED)
    assert b.info().indexed_queries > 0
    got = run_batch(torch, sdblib, b, sdblib.BATCH_PERSISTENT)
    assert sdblib.batch_fallbacks(b) == 0
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    ranges = b.query_ranges()
    order = np.argsort(ranges)
    check_all(orc, T, pts, rows, qb.subset_ids, got[0], got[1],
              which=set(order[-4:].tolist()))
