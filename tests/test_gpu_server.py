"""Continuous-batching server: every result equals the batch API's answer for
the same query alone (and the oracle's), whatever batch it ran in, with or
without the covering cache, batched or one launch per query, with binary
search or the learned index."""
import threading
import time

import numpy as np
import pytest

from paper_2010_12548_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


@pytest.fixture(scope="module")
def env(cuda, sdblib):
    torch = cuda
    rng = np.random.default_rng(21)
    T = W.voronoi_tiling(rng, 500, 20, nverts=(6, 40))
    pts = W.mobility_points(W.BASE_SEED + 78, 1_000_003, 20, 16, sigma=(2 ** 12, 2 ** 15))
    sessions = W.zoom_sessions(9, 12, T, start_side=2 ** 19, start_eps=2 ** 10, zooms=(5, 12))
    queries = [q for s in sessions for q in s]
    p = sdblib.points_create(dev(torch, pts.x), dev(torch, pts.y), dev(torch, pts.attr), 20)
    # reference: the batch API, each query alone
    ref = []
    for row, ids in queries:
        b = sdblib.batch_create(p, T, [row], ids)
        n = b.info().out_len
        c = torch.zeros(max(n, 1), dtype=torch.int64, device="cuda")
        s = torch.zeros(max(n, 1), dtype=torch.int64, device="cuda")
        sdblib.batch_run(b, sdblib.BATCH_PERSISTENT, c, s)
        torch.cuda.synchronize()
        ref.append((c.cpu().numpy()[:n].view(np.uint64), s.cpu().numpy()[:n]))
        b.free()
    return T, pts, p, queries, ref


def serve(sdblib, T, p, queries, order, gap_s=0.0, **cfg):
    srv = sdblib.server_create(p, T, **cfg)
    tickets = [None] * len(order)

    def submitter():
        for k, i in enumerate(order):
            row, ids = queries[i]
            tickets[k] = srv.submit(row, ids)
            if gap_s:
                time.sleep(gap_s)
    th = threading.Thread(target=submitter)
    th.start()
    th.join()
    res = [srv.wait(t, len(queries[i][1])) for t, i in zip(tickets, order)]
    st = srv.stats()
    srv.destroy()
    return res, st


@pytest.mark.parametrize("cfg", [dict(workers=4, max_batch=16),
                                 dict(workers=2, max_batch=64, use_cache=False),
                                 dict(workers=1, max_batch=1, use_cache=False, per_query=True),
                                 dict(workers=3, max_batch=8, cache_bytes=1 << 20),
                                 dict(workers=4, max_batch=16, lookup=1),
                                 dict(workers=2, max_batch=64, use_cache=False, lookup=1)])
def test_server_matches_alone(cuda, sdblib, env, cfg):
    T, pts, p, queries, ref = env
    rng = np.random.default_rng(4)
    order = list(range(len(queries))) * 2  # every query twice: the second can hit the cache
    rng.shuffle(order)
    res, st = serve(sdblib, T, p, queries, order, gap_s=0.0005, **cfg)
    for (c, s, info), i in zip(res, order):
        assert np.array_equal(c, ref[i][0]) and np.array_equal(s, ref[i][1]), i
        assert info.latency_ms >= info.queue_ms >= 0
    assert st.completed == len(order)
    if cfg.get("use_cache", True) and cfg.get("cache_bytes", 1 << 40) > (1 << 30):
        assert st.cache_hits > 0


def test_server_results_vs_oracle(cuda, sdblib, orc, env):
    T, pts, p, queries, ref = env
    for i in (0, 5, len(queries) // 2, len(queries) - 1):
        (x0, y0, x1, y1, eps, _, k), ids = queries[i]
        inside = (pts.x >= x0) & (pts.x < x1) & (pts.y >= y0) & (pts.y < y1)
        c, s, _ = orc.join_o2(T.subset(ids), eps, pts.take(np.nonzero(inside)[0]), threads=8)
        assert np.array_equal(ref[i][0], c) and np.array_equal(ref[i][1], s)


def test_server_tickets_and_timeouts(cuda, sdblib, env):
    T, pts, p, queries, ref = env
    srv = sdblib.server_create(p, T, workers=1, max_batch=1, use_cache=False)
    ts = [srv.submit(*queries[i % len(queries)]) for i in range(120)]
    with pytest.raises(sdblib.SdbError) as e:
        srv.wait(ts[-1], len(queries[119 % len(queries)][1]), timeout_ms=0)
    assert e.value.status == sdblib.SDB_ETIMEOUT
    for k, t in enumerate(ts):
        c, s, _ = srv.wait(t, len(queries[k % len(queries)][1]))
        assert np.array_equal(c, ref[k % len(queries)][0])
    with pytest.raises(sdblib.SdbError) as e:
        srv.wait(ts[0], 1, timeout_ms=0)  # already retired
    assert e.value.status == sdblib.SDB_EINVAL
    with pytest.raises(sdblib.SdbError) as e:
        srv.submit((0, 0, 2 ** 21, 10, 64, 0, 1), np.array([0], np.uint32))  # outside the grid
    assert e.value.status == sdblib.SDB_EINVAL
    srv.destroy()
    with pytest.raises(sdblib.SdbError) as e:  # the table lookup has no batched form
        sdblib.server_create(p, T, lookup=sdblib.LOOKUP_TABLE)
    assert e.value.status == sdblib.SDB_EINVAL
