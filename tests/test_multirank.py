"""The N > 1 host logic of bench.py on CPU: two gloo ranks (replicas), a
barrier, the maximum of the per-rank step times, and the whole-job rate
(every rank's units over the slowest rank's time).  No GPU and no collective on
the data path: the replicas only agree on the clock."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(ws),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    import torch.distributed as dist
    got_ws, got_rank, _ = bench.dist_init(None, backend="gloo")
    bench.barrier(got_ws)
    t = 0.010 * (rank + 1)  # rank r took (r + 1) * 10 ms
    tmax = bench.max_over_ranks(got_ws, t)
    rate = bench.job_rate(got_ws, 1000, tmax)
    q.put((got_rank, got_ws, tmax, rate))
    bench.barrier(got_ws)
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_replicas_agree_on_the_slowest_clock():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=90) for _ in ps)
    for p in ps:
        p.join(timeout=30)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    for _, ws, tmax, rate in out:
        assert ws == 2
        assert tmax == pytest.approx(0.020)
        assert rate == pytest.approx(2 * 1000 / 0.020)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(1, 0.5) == 0.5
    assert bench.job_rate(1, 100, 2.0) == 50.0
