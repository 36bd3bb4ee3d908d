#!/usr/bin/env python3
"""Benchmark of the eps-bounded approximate point-in-polygon join + aggregation.

Workload: 100M mobility-shaped points (uint32 coordinates on [0,2^24)^2, 70%
from 32 Gaussian clusters with sigma in [2^16, 2^19], 30% uniform, int32 fare
attribute), the 263-zone jittered Voronoi tiling (20-400 vertices), and the
eps sweep {2^12, 2^10, 2^8, 2^6}.

One timed step = the join of all points into per-polygon COUNT and SUM at
every eps of the sweep (device-resident points), with the learned lookup: the
cell table (2^22 buckets) as its first level and the learned index (2^16 FP32
leaves) searching inside the table's mixed buckets.  The coverings, tables and
indexes are built before the timed region, as a database builds an index; the
metric counts point-joins: points x eps levels per second of join time.

Beside the timed steps the script measures, on the same coverings, the plain
binary-search join, the learned index alone (2^16 and 2^12 leaves) and the cell
table alone; the whole hot path per step (sweep covering build from the host
polygons, table and index fits, joins); an oracle check of the timed coverings;
the Bounded Raster Join; result range estimation; point-indexed aggregation;
the end-to-end rate through the host-buffer entry point (covering build from
host polygons, points copied from pinned host memory, results read back); the
CPU oracle on a bounded sample; batched level-of-detail queries and serving.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ε-bounded join points/s (learned vs plain lookup); p50/p99 query latency"
UNIT = "points/s"
LEAF_BITS_RANGE = (12, 20)
LEAF_BITS = 16   # learned index of the timed join: 2^16 FP32 leaves
# its root: one line over the id space (the plain two-level model); a root of
# 2^12 segments along the range starts' distribution measured no faster on these
# coverings (windows 1.6x narrower, same join time) and is timed beside it
LEAF_ROOT_BITS = 0
TABLE_BITS = 22  # its first level, the cell table: 2^22 buckets (16 MB), fewer when 2F < 22
# DRAM bytes (read + write) per point of one join_kernel launch at eps = 2^6 on
# the default workload, from one ncu capture of that launch on the 20M-point
# case, scaled to 100M points per point (an upper bound: the table structures'
# share is read once per launch):
# profiles/join_kernel_table_learned_eps64_zones263_mobility20M.txt
JOIN_FINEST_TRAFFIC = {"table_learned": {"eps": 64, "leaf_bits": 16, "root_bits": 0,
                                         "bytes_per_point": 13.934}}
# DRAM bytes of one launch of radix_scatter_kernel (a keys-only pass) in the
# sweep's record sort: profiles/radix_scatter_kernel_sweep_zones263.txt
SCATTER_TRAFFIC = {"records": 117_378_603, "passes": 5, "bytes": 1.8926e9}


def leaf_bits_for(n_ranges: int) -> int:
    """Leaves for about 16 ranges each, within 2^12..2^20."""
    b = max(1, int(n_ranges) // 16).bit_length()
    return min(LEAF_BITS_RANGE[1], max(LEAF_BITS_RANGE[0], b))


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--points", type=int, default=100_000_000)
    ap.add_argument("--no-extras", action="store_true",
                    help="only the timed steps (no join-only, e2e, CPU, batch or serving legs)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--legs",
                    default="oracle,raster,range,e2e,cpu,config3,batch,pointindex,serve",
                    help="extra legs: oracle (check of the timed coverings), raster (Bounded "
                         "Raster Join), range (result range estimation), e2e, cpu, config3 "
                         "(1B points, 40k tiling, learned vs plain), batch, pointindex (range "
                         "counting over sorted points), serve")
    ap.add_argument("--pi-points", type=int, default=500_000_000)
    ap.add_argument("--lod-points", type=int, default=200_000_000)
    ap.add_argument("--lod-queries", type=int, default=4096)
    ap.add_argument("--serve-points", type=int, default=500_000_000)
    ap.add_argument("--serve-rates", default="1000,10000,50000")
    ap.add_argument("--c3-points", type=int, default=1_000_000_000)
    return ap.parse_args()


def dist_init(args, backend: str | None = None):
    """One process per GPU (torchrun environment); NCCL on GPUs, gloo when the
    caller asks for it (the CPU tests of this host logic)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = backend or "nccl"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, v):
    """The maximum of v over all ranks (the job's time is its slowest rank's)."""
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(ws, units_per_rank, seconds):
    """Whole-job throughput of weak-scaled replicas: every rank's units over the
    slowest rank's time."""
    return ws * units_per_rank / seconds


class Clocks:
    """SM clock and throttle reasons sampled during the timed region: read-only
    NVML queries every 2 ms from a thread (the timed region can be shorter than
    nvidia-smi's sampling interval), else nvidia-smi sampling every 50 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # NVML clock-event reason bits (nvml.h)
    REASONS = {0x8: "hw_slowdown", 0x40: "hw_thermal_slowdown", 0x20: "sw_thermal_slowdown",
               0x4: "sw_power_cap", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, gpu_index: int, pci_bus_id: str | None = None):
        self.idx = gpu_index
        self.bus = pci_bus_id
        self.rows = []
        self.proc = None
        self.t = None
        self.nv = None
        self.stop = threading.Event()
        self.source = None

    def _nvml(self):
        import ctypes as C
        nv = C.CDLL("libnvidia-ml.so.1")
        if nv.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        h = C.c_void_p()
        if self.bus and nv.nvmlDeviceGetHandleByPciBusId_v2(self.bus.encode(), C.byref(h)) == 0:
            pass
        elif nv.nvmlDeviceGetHandleByIndex_v2(self.idx, C.byref(h)) != 0:
            raise RuntimeError("no NVML handle")
        mx = C.c_uint()
        nv.nvmlDeviceGetMaxClockInfo(h, 1, C.byref(mx))  # NVML_CLOCK_SM
        return nv, h, mx.value

    def _poll(self, nv, h, mx):
        import ctypes as C
        clk, rs = C.c_uint(), C.c_ulonglong()
        while not self.stop.is_set():
            nv.nvmlDeviceGetClockInfo(h, 1, C.byref(clk))
            nv.nvmlDeviceGetCurrentClocksEventReasons(h, C.byref(rs))
            self.rows.append((float(clk.value), float(mx), int(rs.value)))
            time.sleep(0.002)

    def __enter__(self):
        try:
            nv, h, mx = self._nvml()
            self.source = "nvml"
            self.t = threading.Thread(target=self._poll, args=(nv, h, mx), daemon=True)
            self.t.start()
            t_end = time.time() + 1.0
            while not self.rows and time.time() < t_end:
                time.sleep(0.001)
            self.rows.clear()
            return self
        except Exception:
            self.source = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.source = "nvidia-smi"
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # the sampler takes a moment to start: wait for its first sample, then
            # keep only the samples taken from here on (the timed region)
            t_end = time.time() + 3.0
            while not self.rows and time.time() < t_end and self.proc.poll() is None:
                time.sleep(0.01)
            self.rows.clear()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        self.stop.set()
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.t:
            self.t.join(timeout=2)

    def summary(self):
        rows = list(self.rows)
        if self.source == "nvml":
            sm = [r[0] for r in rows if r[0] > 0]
            reasons = sorted({n for r in rows for bit, n in self.REASONS.items() if r[2] & bit})
            return {"sm_mhz": statistics.median(sm) if sm else None,
                    "sm_max_mhz": max((r[1] for r in rows), default=None), "reasons": reasons,
                    "samples": len(rows), "source": "nvml, 2 ms"}

        def num(s):
            try:
                return float(s.split()[0])
            except Exception:
                return None
        sm = [num(r[1]) for r in rows if len(r) >= 9 and num(r[1])]
        mx = [num(r[2]) for r in rows if len(r) >= 9 and num(r[2])]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) >= 9:
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows), "source": "nvidia-smi, 50 ms"}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def workload(n_points):
    from paper_2010_12548_gb300 import workloads as W
    return W.mobility_zones(n_points)


def cpu_oracle_rate(w, seconds: float, threads: int, max_points: int | None = None):
    """Oracle O2 (definitional per-point test) on a bounded sample of the
    workload's points, all eps levels; returns (points x eps / s, sample size, secs)."""
    from oracle import oracle as O
    O.build()
    n = 20_000
    spent = 0.0
    while True:
        pts = w.points.take(np.arange(min(n, w.points.n)))
        t0 = time.perf_counter()
        for eps in w.eps:
            O.join_o2(w.polygons, eps, pts, threads=threads)
        spent = time.perf_counter() - t0
        if spent >= seconds / 4 or n >= w.points.n or (max_points and n >= max_points):
            break
        n = int(n * min(8.0, max(2.0, seconds / max(spent, 1e-3) / 2)))
        n = min(n, w.points.n)
    return pts.n * len(w.eps) / spent, pts.n, spent


def oracle_forms(w, threads: int):
    """Both oracle forms timed on the host: O1 (recursive quadtree covering,
    ordered map of ranges, per-point ordered lookup; single thread) and O2 (the
    definitional per-point test; one thread and all cores), on the 16-star
    100k-point workload at eps 64 and on the zone workload at eps 2^12."""
    from oracle import oracle as O
    from paper_2010_12548_gb300 import workloads as W
    out = {}
    t1 = W.tiny_stars(100_000)
    for name, polys, eps, pts in (("stars16_100k_eps64", t1.polygons, t1.eps[0], t1.points),
                                  ("zones263_eps4096", w.polygons, 4096,
                                   w.points.take(np.arange(min(w.points.n, 2_000_000))))):
        t = time.perf_counter()
        oc = O.cover(polys, eps)
        build_s = time.perf_counter() - t
        t = time.perf_counter()
        oc.join(pts.x, pts.y, pts.attr)
        join_s = time.perf_counter() - t
        oc.free()
        row = {"points": pts.n, "o1_build_s": build_s, "o1_points_per_s": pts.n / join_s}
        for th in (1, threads):
            m = pts.n if th > 1 else min(pts.n, 200_000)
            sp = pts.take(np.arange(m))
            t = time.perf_counter()
            O.join_o2(polys, eps, sp, threads=th)
            row[f"o2_points_per_s_{th}t"] = m / (time.perf_counter() - t)
        out[name] = row
    return out


def run_reference(args):
    ws, rank, _ = dist_init(args) if int(os.environ.get("WORLD_SIZE", "1")) > 1 else (1, 0, 0)
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    w = workload(args.points)
    rate, sample, _ = cpu_oracle_rate(w, max(2.0, args.cpu_seconds / 2), threads)
    from oracle import oracle as O
    pts = w.points.take(np.arange(sample))
    for _ in range(args.warmup):
        for eps in w.eps[:1]:
            O.join_o2(w.polygons, eps, pts.take(np.arange(min(2000, pts.n))), threads=threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for eps in w.eps:
            O.join_o2(w.polygons, eps, pts, threads=threads)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = sample * len(w.eps) / (ms / 1e3)
    sample_desc = f"first {sample} of the {w.points.n} points, all {len(w.eps)} eps levels per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": config_of(w, args.points),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample_desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_of(w, n_points):
    return {"workload": f"zones263_mobility{n_points // 1_000_000}M_g24_eps4096-64",
            "points": n_points, "polygons": w.polygons.n, "grid_bits": 24, "eps": w.eps,
            "lookup": "table_learned (cell table 2^%d buckets, learned index 2^%d leaves under "
                      "one root line)" % (TABLE_BITS, LEAF_BITS),
            "plain_lookup": "binary", "leaf_bits": LEAF_BITS, "root_bits": LEAF_ROOT_BITS,
            "table_bits": TABLE_BITS,
            "l2": "inputs larger than L2 (point arrays 12 B/pt, 1.2 GB)"}


def lookup_prep(sdb, c, lookup, stream, leaf_bits=None, table_bits=None):
    """The lookup structures a join with `lookup` reads, built on covering c."""
    if lookup in (sdb.LOOKUP_LEARNED, sdb.LOOKUP_TABLE_LEARNED):
        sdb.covering_build_index(c, leaf_bits or LEAF_BITS, stream, root_bits=LEAF_ROOT_BITS)
    if lookup in (sdb.LOOKUP_TABLE, sdb.LOOKUP_TABLE_LEARNED):
        sdb.covering_build_table(c, table_bits or TABLE_BITS, stream)


def lookup_bytes(sdb, c, lookup):
    """Bytes of the structure a lookup reads per launch besides the points:
    the covering and its index for the searches over all ranges, the cell
    table, its mixed buckets' windows and (table + learned) the index for the
    table lookups (the ranges are then read only inside mixed buckets)."""
    inf = c.info()
    leaves = (32 * (1 << inf.index_leaf_bits) + 4 * ((1 << inf.index_root_bits) + 1)
              if inf.index_leaf_bits else 0)
    if lookup in (sdb.LOOKUP_TABLE, sdb.LOOKUP_TABLE_LEARNED):
        tab = 4 * (1 << inf.table_bits) + 8 * inf.table_mixed
        if inf.table_sub_bits:
            tab += 4 * (1 << (2 * inf.table_sub_bits)) * inf.table_mixed + 8 * inf.table_sub_mixed
        return tab + (leaves if lookup == sdb.LOOKUP_TABLE_LEARNED else 0)
    return inf.device_bytes


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    ws, rank, local = dist_init(args)
    legs = set() if args.no_extras else set(args.legs.split(","))
    import torch
    torch.cuda.set_device(local)
    from paper_2010_12548_gb300 import build as B
    B.build()
    from paper_2010_12548_gb300 import sdb

    w = workload(args.points)
    N = w.points.n
    P = w.polygons.n
    E = len(w.eps)
    dev = torch.device("cuda", local)

    def to_dev(a):
        return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).to(dev)

    x, y, a = to_dev(w.points.x), to_dev(w.points.y), to_dev(w.points.attr)
    stream = torch.cuda.current_stream()
    HEAD, PLAIN = sdb.LOOKUP_TABLE_LEARNED, sdb.LOOKUP_BINARY

    # the coverings of the sweep (one pass) and the headline lookup's structures,
    # built before the timed region: they are the join's resident inputs, like
    # the points (their build is timed separately below)
    covs = sdb.build_coverings(w.polygons, 24, w.eps, stream)
    for c in covs:
        lookup_prep(sdb, c, HEAD, stream)
    cnt = torch.zeros((E, P), dtype=torch.int64, device=dev)
    sm = torch.zeros((E, P), dtype=torch.int64, device=dev)

    def step(evs=None):
        # one pass of the join over all points at every eps of the sweep
        for i, c in enumerate(covs):
            sdb.join_aggregate(x, y, a, c, HEAD, cnt[i], sm[i], stream)
            if evs is not None:
                evs[i].record(stream)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in w.eps] for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = sdb.launch_count()
    barrier(ws)
    torch.cuda.synchronize()
    try:
        p = torch.cuda.get_device_properties(local)
        bus = "%08x:%02x:%02x.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
    except Exception:
        bus = None
    with Clocks(local, bus) as clk:
        t0.record(stream)
        for k in range(args.steps):
            step(ev[k])
        t1.record(stream)
        torch.cuda.synchronize()
    barrier(ws)
    launches = sdb.launch_count() - launches0
    ms = t0.elapsed_time(t1) / args.steps
    ms = max_over_ranks(ws, ms)
    value = job_rate(ws, N * E, ms / 1e3)
    # per-eps join time: the events recorded between the back-to-back joins
    join_ms = []
    for i in range(E):
        d = [(ev[k][i - 1] if i else (ev[k - 1][E - 1] if k else t0)).elapsed_time(ev[k][i])
             for k in range(args.steps)]
        join_ms.append(statistics.mean(d))
    res = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
           "config": config_of(w, N), "clocks": clk.summary(), "gpu_launches": launches}
    res["join_ms"] = {"table_learned": dict(zip(map(str, w.eps), join_ms))}
    infos = [c.info() for c in covs]
    res["coverings"] = {str(e): {"ranges": i.n_ranges, "cells": i.n_cells,
                                 "covering_bytes": i.device_bytes, "table_mixed": i.table_mixed,
                                 "table_sub_mixed": i.table_sub_mixed}
                        for e, i in zip(w.eps, infos)}
    head_cnt, head_sm = cnt.clone(), sm.clone()
    fallbacks = [sdb.covering_fallbacks(c, stream) for c in covs]
    res["learned_fallbacks"] = sum(fallbacks)
    peak, peak_kind = peaks()

    # ---- the same joins with the plain binary search, the learned index alone
    # and the cell table alone, on the same coverings; results must agree
    reps = max(3, min(args.steps, 10))
    agree = True
    lk_rows = {}
    # (the "_knot_root" rows fit the index with a root of 2^12 segments along
    # the range starts' distribution instead of one root line)
    for name, lk, bits, root in (("binary", PLAIN, None, None),
                                 ("learned", sdb.LOOKUP_LEARNED, LEAF_BITS, LEAF_ROOT_BITS),
                                 ("learned12", sdb.LOOKUP_LEARNED, 12, LEAF_ROOT_BITS),
                                 ("learned_knot_root", sdb.LOOKUP_LEARNED, LEAF_BITS, 12),
                                 ("table_learned_knot_root", HEAD, LEAF_BITS, 12),
                                 ("table", sdb.LOOKUP_TABLE, None, None)):
        per = {}
        for i, c in enumerate(covs):
            if bits:
                sdb.covering_build_index(c, bits, stream, root_bits=root)
            per[str(w.eps[i])] = timed(torch, stream, lambda c=c, i=i: sdb.join_aggregate(
                x, y, a, c, lk, cnt[i], sm[i], stream), reps)
            agree &= bool(torch.equal(cnt[i], head_cnt[i]) and torch.equal(sm[i], head_sm[i]))
            if lk in (sdb.LOOKUP_LEARNED, sdb.LOOKUP_TABLE_LEARNED):
                per[str(w.eps[i]) + "_fallbacks"] = sdb.covering_fallbacks(c, stream)
                mw, xw = sdb.covering_index_stats(c)
                per[str(w.eps[i]) + "_window_mean"] = mw
        tot = sum(per[str(e)] for e in w.eps)
        per["points_per_s"] = N * E / (tot / 1e3)
        lk_rows[name] = per
    for c in covs:  # back to the headline index
        sdb.covering_build_index(c, LEAF_BITS, stream, root_bits=LEAF_ROOT_BITS)
    res["join_ms"].update(lk_rows)
    res["plain_value"] = lk_rows["binary"]["points_per_s"]
    res["learned_only_value"] = lk_rows["learned"]["points_per_s"]
    res["table_value"] = lk_rows["table"]["points_per_s"]
    res["lookups_agree"] = agree
    # the sweep in one pass over the points (sdb_join_aggregate_multi through the
    # tables: the points read once, a combined top level for all four coverings)
    sw_ms = timed(torch, stream, lambda: sdb.join_aggregate_multi(x, y, a, covs, HEAD, cnt, sm,
                                                                  stream), reps)
    res["sweep_fused"] = {"ms": sw_ms, "points_per_s": N * E / (sw_ms / 1e3),
                          "same_as_separate_joins": bool(torch.equal(cnt, head_cnt)
                                                         and torch.equal(sm, head_sm)),
                          "what": "one pass over the points for all four coverings "
                                  "(table + learned lookup)"}

    # ---- the timed coverings against the CPU oracle: the first 1M points
    # joined on the device with the headline lookup vs the definitional test
    # (O2) on the host, every eps
    if rank == 0 and "oracle" in legs:
        from oracle import oracle as O
        O.build()
        m = min(N, 1_000_000)
        pts = w.points.take(np.arange(m))
        ok = True
        for i, (e, c) in enumerate(zip(w.eps, covs)):
            sdb.join_aggregate(x[:m], y[:m], a[:m], c, HEAD, cnt[i], sm[i], stream)
            torch.cuda.synchronize()
            oc, os_, _ = O.join_o2(w.polygons, e, pts, threads=os.cpu_count() or 1)
            ok &= bool(np.array_equal(cnt[i].cpu().numpy().view(np.uint64), oc)
                       and np.array_equal(sm[i].cpu().numpy(), os_))
        res["matches_oracle"] = ok
        res["oracle_check"] = f"first {m} points, all {E} eps, headline lookup vs O2"

    # ---- the whole hot path per step: sweep build from host polygons, then per
    # eps the cell table, the learned index and the join
    def full_step():
        cs = sdb.build_coverings(w.polygons, 24, w.eps, stream)
        for i, c in enumerate(cs):
            lookup_prep(sdb, c, HEAD, stream)
            sdb.join_aggregate(x, y, a, c, HEAD, cnt[i], sm[i], stream)
        return cs
    for c in full_step():
        c.free()
    torch.cuda.synchronize()
    sdb.trace_enable(True)
    fs_reps = 3
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    live = []
    for _ in range(fs_reps):
        live.extend(full_step())
        while live:
            live.pop().free()
    e1.record(stream)
    torch.cuda.synchronize()
    trace = sdb.trace_read()
    sdb.trace_enable(False)
    full_ms = e0.elapsed_time(e1) / fs_reps
    res["full_step"] = {"ms": full_ms, "points_per_s": N * E / (full_ms / 1e3),
                        "what": "sweep covering build (4 eps, one pass) + per eps cell table, "
                                "learned index fit and table_learned join"}
    res["trace_per_step"] = {k: {"launches": cc / fs_reps, "ms": t / fs_reps}
                             for k, (cc, t) in trace.items()}

    # ---- rooflines.  The headline join at the finest eps: the point stream
    # (x, y, attr: 12 B/pt) plus one read of the structures the lookup uses
    fine = str(w.eps[-1])
    per_pt = 12 + lookup_bytes(sdb, covs[-1], HEAD) / N
    achieved = N * per_pt / (join_ms[-1] / 1e3) / 1e9
    T = JOIN_FINEST_TRAFFIC.get("table_learned")
    traffic = (T["bytes_per_point"] * N
               if T and w.eps[-1] == T["eps"] and T["leaf_bits"] == LEAF_BITS
               and T["root_bits"] == LEAF_ROOT_BITS else None)
    res["roofline"] = {"kernel": "join_kernel<table_learned> eps=%s" % fine, "bound": "hbm",
                       "achieved": achieved, "peak": peak, "unit": "GB/s",
                       "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
                       "avg_launch_ms": join_ms[-1], "algorithmic_bytes_per_point": per_pt,
                       "algorithmic_bytes_per_launch": per_pt * N,
                       "profile": "profiles/join_kernel_table_learned_eps64_zones263_mobility20M.txt"}
    # the record sort's scatter inside the full step (one launch per pass over
    # all records): 8 B read + 8 B written per record and pass, 8 + 12 B in the
    # last pass (keys and values apart)
    recs = sum(i.n_cells for i in infos)
    sc_n, sc_ms = trace.get("sort.scatter", (0, 0.0))
    if sc_n:
        passes = sc_n / fs_reps
        sc_bytes = recs * (16 * (passes - 1) + 20) / passes
        sc_avg = sc_ms / sc_n
        ach = sc_bytes / (sc_avg / 1e3) / 1e9
        T = SCATTER_TRAFFIC
        res["roofline_radix_scatter"] = {
            "kernel": "radix_scatter_kernel (%d records)" % recs, "bound": "hbm",
            "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "peak_kind": peak_kind, "avg_launch_ms": sc_avg, "launches_per_step": passes,
            "traffic": T["bytes"] if T and T["records"] == recs and T["passes"] == passes
            else None, "algorithmic_bytes_per_launch": sc_bytes}
    for c in covs:
        c.free()
    covs = []

    # ---- Bounded Raster Join (Sec. 5.2): canvas blend + conservative raster mask
    if "raster" in legs:
        rows = {}
        rc, rs_ = (torch.zeros(P, dtype=torch.int64, device=dev) for _ in range(2))
        for i, eps in enumerate(w.eps):
            reps = 3 if eps >= 1024 else 1
            rms = timed(torch, stream, lambda: sdb.raster_join(w.polygons, 24, eps, x, y, a, rc,
                                                               rs_, 0, stream), reps)
            F = 24 - int(np.log2(eps)) + 1
            rows[str(eps)] = {"raster_join_ms": rms, "canvas_pixels": 4 ** F,
                              "tiles": max(1, 4 ** (F - 13)),
                              "covering_join_ms": join_ms[i],
                              "matches_covering_join": bool(torch.equal(rc, head_cnt[i])
                                                            and torch.equal(rs_, head_sm[i]))}
        res["raster_join"] = rows
    # ---- result range estimation (Sec. 6): flagged coverings, the range join,
    # and the intervals computed by the library
    if "range" in legs:
        rng_rows = {}
        bc, bs_, ba = (torch.zeros(P, dtype=torch.int64, device=dev) for _ in range(3))
        rc, rs_ = (torch.zeros(P, dtype=torch.int64, device=dev) for _ in range(2))
        for i, eps in enumerate(w.eps):
            e0.record(stream)
            c = sdb.build_covering(w.polygons, 24, eps, stream, flags=sdb.COVER_BOUNDARY_FLAGS)
            inf = c.info()
            lookup_prep(sdb, c, HEAD, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            row = {"build_and_index_ms": e0.elapsed_time(e1), "ranges": inf.n_ranges,
                   "plain_ranges": infos[i].n_ranges, "lookup": "table_learned"}
            row["range_join_ms"] = timed(torch, stream, lambda: sdb.join_aggregate_range(
                x, y, a, c, HEAD, rc, bc, rs_, bs_, ba, stream), 5)
            row["plain_join_ms"] = join_ms[i]
            lo_c, hi_c, lo_s, hi_s = sdb.result_bounds(rc, bc, rs_, bs_, ba, stream)
            torch.cuda.synchronize()
            row["matches_plain_join"] = bool(torch.equal(rc, head_cnt[i])
                                             and torch.equal(rs_, head_sm[i]))
            c_np, b_np = rc.cpu().numpy(), bc.cpu().numpy()
            live_ = c_np > 0
            row["boundary_fraction"] = float(b_np.sum() / max(1, c_np.sum()))
            row["mean_relative_count_interval"] = float(
                ((hi_c - lo_c).cpu().numpy()[live_] / c_np[live_]).mean())
            c.free()
            # the non-conservative covering (Sec. 2.2): build, join, and the share
            # of the boundary count it drops
            e0.record(stream)
            c = sdb.build_covering(w.polygons, 24, eps, stream, flags=sdb.COVER_NONCONSERVATIVE)
            lookup_prep(sdb, c, HEAD, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            row["noncons_build_and_index_ms"] = e0.elapsed_time(e1)
            row["noncons_ranges"] = c.info().n_ranges
            row["noncons_join_ms"] = timed(torch, stream, lambda: sdb.join_aggregate(
                x, y, a, c, HEAD, bs_, ba, stream), 5)
            nc_np = bs_.cpu().numpy()
            row["noncons_dropped_fraction_of_boundary"] = float(
                (c_np - nc_np).sum() / max(1, b_np.sum()))
            rng_rows[str(eps)] = row
            c.free()
        res["range_estimation"] = rng_rows
    # ---- end to end through the C ABI from host buffers.  e2e: the timed
    # step's metric through the host-buffer entry point -- every step copies the
    # points from pinned host memory (chunked, copies overlapping the joins) and
    # reads the results back, against the resident coverings and lookup
    # structures.  e2e_with_build adds, every step, the sweep's covering build
    # from the host polygons and the table and index fits.
    if "e2e" in legs:
        hx = torch.from_numpy(w.points.x.view(np.int32)).pin_memory()
        hy = torch.from_numpy(w.points.y.view(np.int32)).pin_memory()
        ha = torch.from_numpy(w.points.attr).pin_memory()
        hc = torch.zeros((E, P), dtype=torch.int64).pin_memory()
        hs = torch.zeros((E, P), dtype=torch.int64).pin_memory()

        def host_join(cs):
            sdb.join_aggregate_host_ptrs(hx.data_ptr(), hy.data_ptr(), ha.data_ptr(), N, cs,
                                         HEAD, hc.data_ptr(), hs.data_ptr(), stream)

        def e2e_build_step():
            cs = sdb.build_coverings(w.polygons, 24, w.eps, stream)
            for c in cs:
                lookup_prep(sdb, c, HEAD, stream)
            host_join(cs)
            for c in cs:
                c.free()

        def wall(fn, steps, warm):
            for _ in range(warm):
                fn()
            torch.cuda.synchronize()
            tt = time.perf_counter()
            for _ in range(steps):
                fn()
            torch.cuda.synchronize()
            return max_over_ranks(ws, (time.perf_counter() - tt) / steps)

        cs = sdb.build_coverings(w.polygons, 24, w.eps, stream)
        for c in cs:
            lookup_prep(sdb, c, HEAD, stream)
        e2e_s = wall(lambda: host_join(cs), args.steps, max(3, args.warmup))
        same = bool(np.array_equal(hc.numpy(), head_cnt.cpu().numpy()) and
                    np.array_equal(hs.numpy(), head_sm.cpu().numpy()))
        for c in cs:
            c.free()
        # the host -> device link: the point arrays copied from pinned memory in
        # the host join's chunks of 2^24 points (one copy of 3 x 400 MB measured
        # half the rate on some hosts)
        dbuf = torch.empty(N * 3, dtype=torch.int32, device=dev)
        LINK_CHUNK = 1 << 24
        def link_copy():
            with torch.cuda.stream(stream):
                for j, h in enumerate((hx, hy, ha)):
                    for a0 in range(0, N, LINK_CHUNK):
                        a1 = min(N, a0 + LINK_CHUNK)
                        dbuf[j * N + a0:j * N + a1].copy_(h[a0:a1], non_blocking=True)
        link_s = wall(link_copy, 5, 2)
        del dbuf
        res["e2e"] = {"value": job_rate(ws, N * E, e2e_s), "unit": UNIT,
                      "h2d_link_GB_per_s": N * 12 / link_s / 1e9,
                      "frac_of_link": (N * 12 / e2e_s) / (N * 12 / link_s),
                      "h2d_bytes_per_step": N * 12, "d2h_bytes_per_step": E * P * 16,
                      "ms_per_step": e2e_s * 1e3, "matches_device": same,
                      "what": "sdb_join_aggregate_host: points copied from pinned host memory "
                              "every step (chunks, copies overlapping the joins), the four "
                              "joins against the resident coverings, results read back"}
        eb_s = wall(e2e_build_step, max(3, args.steps // 4), 1)
        res["e2e_with_build"] = {
            "value": job_rate(ws, N * E, eb_s), "unit": UNIT, "ms_per_step": eb_s * 1e3,
            "h2d_bytes_per_step": N * 12, "d2h_bytes_per_step": E * P * 16,
            "matches_device": bool(np.array_equal(hc.numpy(), head_cnt.cpu().numpy()) and
                                   np.array_equal(hs.numpy(), head_sm.cpu().numpy())),
            "what": "host polygons -> sweep coverings, cell tables, learned indexes -> "
                    "host-buffer join -> host results, every step"}
    # ---- CPU oracle on a bounded sample (rank 0, N = 1 only)
    if rank == 0 and ws == 1 and "cpu" in legs:
        threads = os.cpu_count() or 1
        rate, sample, secs = cpu_oracle_rate(w, args.cpu_seconds, threads)
        rate1, sample1, secs1 = cpu_oracle_rate(w, args.cpu_seconds / 3, 1)
        res["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                               "sample": f"first {sample} of the {N} points, all {E} eps "
                                         f"levels, definitional per-point test ({secs:.1f} s)",
                               "single_thread": {"value": rate1, "cores": 1,
                                                 "sample": f"first {sample1} points, all {E} "
                                                           f"eps ({secs1:.1f} s)"},
                               "cpu": cpu_model(), "oracle_forms": oracle_forms(w, threads)}
    # ---- batched level-of-detail queries and serving (resident points)
    del x, y, a
    torch.cuda.empty_cache()
    if legs & {"batch", "serve", "pointindex", "config3"}:
        res.update(resident_legs(args, legs, sdb, torch, dev, stream))
    if "serving" in res and res["serving"].get("batched_learned"):
        nominal = [r for r in res["serving"]["batched_learned"] if r["rate"] == 10000] or \
            res["serving"]["batched_learned"]
        res["p50_ms"] = nominal[0]["p50_ms"]
        res["p99_ms"] = nominal[0]["p99_ms"]
        res["latency_note"] = "learned, batched serving at %d queries/s" % nominal[0]["rate"]
    if rank == 0:
        print(json.dumps(res), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part", "hardware")):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def timed(torch, stream, fn, reps):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def poisson_serve(sdb, srv, queries, rate, n, seed):
    """Submit n queries at Poisson arrival times (rate per second) from a
    submitter thread; returns per-query latencies, batch sizes, cache hits, the
    wall time and how late each submit came against its arrival time (the
    queries are marshalled before the clock starts, so the submitter keeps
    pace with the arrivals)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=n)
    order = rng.integers(0, len(queries), size=n)
    preps = [srv.prepare(*queries[order[k]]) for k in range(n)]
    tickets = [None] * n
    sub_t = np.zeros(n)
    t0 = time.perf_counter()
    due = t0 + np.cumsum(gaps)

    def submitter():
        for k in range(n):
            while True:
                now = time.perf_counter()
                if now >= due[k]:
                    break
                if due[k] - now > 2e-4:
                    time.sleep(min(1e-3, due[k] - now - 1e-4))
            tickets[k] = srv.submit_prepared(preps[k])
            sub_t[k] = time.perf_counter()
    th = threading.Thread(target=submitter)
    th.start()
    lat, batch, hits = [], [], 0
    th.join()
    for k in range(n):
        _, _, info = srv.wait(tickets[k], len(queries[order[k]][1]), timeout_ms=600_000)
        lat.append(info.latency_ms)
        batch.append(info.batch_size)
        hits += info.cache_hit
    wall = time.perf_counter() - t0
    lat = np.asarray(lat)
    # the last completion: each query's submit time plus the latency the server
    # measured for it (the ticket collection above runs after the arrivals and
    # is not part of the service)
    span = float((sub_t + lat / 1e3).max() - t0)
    return lat, np.asarray(batch), hits, wall, span, float(gaps.sum()), (sub_t - due) * 1e3


def point_index_leg(args, sdb, torch, dev, stream, T, pts, resident):
    """Sec. 3 point indexing (the paper's Fig. 4a setting: ~40k tract polygons
    over resident points, 32..800 covering cells per polygon): range counting
    over Hilbert-sorted points with prefix sums, binary search vs RadixSpline
    (radix bits 25, spline error 32), beside the per-point join over the same
    points; results must be equal."""
    n = args.pi_points
    p = resident(n)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    sdb.points_build_index(p, 25, 32, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ns, err, _ = sdb.points_index_stats(p, stream)
    out = {"workload": f"tracts40k_pts{n // 1_000_000}M_g28", "points": n,
           "index_build_ms": e0.elapsed_time(e1), "spline_points": ns, "spline_max_error": err,
           "radix_bits": 25, "spline_error": 32, "levels": {}}
    xs = torch.from_numpy(pts.x[:n].view(np.int32)).to(dev)
    ys = torch.from_numpy(pts.y[:n].view(np.int32)).to(dev)
    at = torch.from_numpy(pts.attr[:n]).to(dev)
    P = T.n
    c1, s1, c2, s2 = (torch.zeros(P, dtype=torch.int64, device=dev) for _ in range(4))
    for eps in (2 ** 19, 2 ** 18, 2 ** 17, 2 ** 16, 2 ** 15):
        cov = sdb.build_covering(T, 28, eps, stream)
        inf = cov.info()
        sdb.covering_build_index(cov, leaf_bits_for(inf.n_ranges), stream)
        bs = timed(torch, stream, lambda: sdb.points_aggregate(p, cov, sdb.LOOKUP_BINARY, c1, s1,
                                                               stream), 5)
        rs = timed(torch, stream, lambda: sdb.points_aggregate(p, cov, sdb.LOOKUP_RADIX_SPLINE, c1,
                                                               s1, stream), 5)
        js = timed(torch, stream, lambda: sdb.join_aggregate(xs, ys, at, cov, sdb.LOOKUP_LEARNED,
                                                             c2, s2, stream), 3)
        lookups = inf.n_ranges + 1
        out["levels"][str(eps)] = {
            "cells_per_polygon": inf.n_cells / P, "ranges": inf.n_ranges,
            "binary_ms": bs, "radix_spline_ms": rs, "point_stream_join_ms": js,
            "radix_spline_lookups_per_s": lookups / (rs / 1e3),
            "binary_lookups_per_s": lookups / (bs / 1e3),
            "matches_point_stream": bool(torch.equal(c1, c2) and torch.equal(s1, s2)),
            "fallbacks": sdb.points_index_stats(p, stream)[2]}
        cov.free()
    del xs, ys, at
    p.free()
    torch.cuda.empty_cache()
    return out


C3_EPS_SWEEP = (2 ** 12, 2 ** 11, 2 ** 10, 2 ** 9)


def config3_leg(args, sdb, torch, dev, stream, T, pts):
    """The large learned index (1B points on [0,2^28)^2, 64-cluster mix, the
    40,000-cell tiling).  Range and record counts of single covering builds
    against eps (they grow as 1/eps: the finest feasible eps is the finest whose
    records, frontier edge entries and ranges stay inside the builder's 32-bit
    limits); at the finest eps of the sweep, the join of all points with binary
    search, the learned index alone (2^16 leaves), the cell table and the
    table + learned lookup on the same covering; results must agree and match
    the oracle's definitional test on a 2M-point sample."""
    from oracle import oracle as O
    n = min(args.c3_points, pts.n)
    P = T.n
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    xs = torch.from_numpy(pts.x[:n].view(np.int32)).to(dev)
    ys = torch.from_numpy(pts.y[:n].view(np.int32)).to(dev)
    at = torch.from_numpy(pts.attr[:n]).to(dev)
    out = {"workload": f"tracts40k_pts{n // 1_000_000}M_g28", "points": n, "polygons": P,
           "sweep": {}}
    cov = None
    for eps in C3_EPS_SWEEP:
        if cov is not None:
            cov.free()
        torch.cuda.synchronize()
        e0.record(stream)
        cov = sdb.build_covering(T, 28, eps, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        inf = cov.info()
        out["sweep"][str(eps)] = {"ranges": inf.n_ranges, "cells": inf.n_cells,
                                  "covering_bytes": inf.device_bytes, "finest_level": inf.finest_level,
                                  "build_ms": e0.elapsed_time(e1)}
    eps = C3_EPS_SWEEP[-1]
    cells = out["sweep"][str(eps)]["cells"]
    out["eps"] = eps
    out["eps_2^5_estimate"] = {
        "cells": cells * eps // 32, "why_not_built": "records grow as 1/eps: about %.1e records "
        "at eps = 2^5, beyond the builder's 32-bit record and edge-entry ranges and, as a "
        "covering of ~24 B per range, beyond device memory" % (cells * eps / 32)}
    e0.record(stream)
    sdb.covering_build_table(cov, TABLE_BITS, stream)
    sdb.covering_build_index(cov, LEAF_BITS, stream, root_bits=LEAF_ROOT_BITS)
    e1.record(stream)
    torch.cuda.synchronize()
    out["table_and_index_ms"] = e0.elapsed_time(e1)
    cnt = torch.zeros(P, dtype=torch.int64, device=dev)
    sm = torch.zeros(P, dtype=torch.int64, device=dev)
    ref = None
    agree = True
    rows = {}
    for name, lk in (("table_learned", sdb.LOOKUP_TABLE_LEARNED), ("binary", sdb.LOOKUP_BINARY),
                     ("learned", sdb.LOOKUP_LEARNED), ("table", sdb.LOOKUP_TABLE)):
        ms = timed(torch, stream, lambda lk=lk: sdb.join_aggregate(xs, ys, at, cov, lk, cnt, sm,
                                                                    stream), 3)
        rows[name] = {"ms": ms, "points_per_s": n / (ms / 1e3)}
        if lk in (sdb.LOOKUP_LEARNED, sdb.LOOKUP_TABLE_LEARNED):
            rows[name]["fallbacks"] = sdb.covering_fallbacks(cov, stream)
        got = (cnt.clone(), sm.clone())
        if ref is None:
            ref = got
        agree &= bool(torch.equal(got[0], ref[0]) and torch.equal(got[1], ref[1]))
    # finer cell tables on the same covering (the 2^28 grid's boundaries cross
    # far more of the 2^22 table's buckets than on the 2^24 grid)
    for tb in (24, 26):
        sdb.covering_build_table(cov, tb, stream)
        ms = timed(torch, stream, lambda: sdb.join_aggregate(
            xs, ys, at, cov, sdb.LOOKUP_TABLE_LEARNED, cnt, sm, stream), 3)
        ti = cov.info()
        rows[f"table_learned_t{tb}"] = {"ms": ms, "points_per_s": n / (ms / 1e3),
                                        "table_mixed": ti.table_mixed,
                                        "table_sub_mixed": ti.table_sub_mixed}
        agree &= bool(torch.equal(cnt, ref[0]) and torch.equal(sm, ref[1]))
    sdb.covering_build_table(cov, TABLE_BITS, stream)
    out["joins"] = rows
    out["lookups_agree"] = agree
    best = min((k for k in rows if k.startswith("table_learned")), key=lambda k: rows[k]["ms"])
    out["value"] = rows[best]["points_per_s"]
    out["value_lookup"] = best
    out["plain_value"] = rows["binary"]["points_per_s"]
    inf = cov.info()
    out["table_mixed"] = inf.table_mixed
    out["table_sub_mixed"] = inf.table_sub_mixed
    mw, xw = sdb.covering_index_stats(cov)
    out["learned_window_mean"] = mw
    peak, peak_kind = peaks()
    per_pt = 12 + lookup_bytes(sdb, cov, sdb.LOOKUP_TABLE_LEARNED) / n
    ach = n * per_pt / (rows["table_learned"]["ms"] / 1e3) / 1e9
    out["roofline"] = {"kernel": "join_kernel<table_learned> eps=%d" % eps, "bound": "hbm",
                       "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                       "peak_kind": peak_kind, "algorithmic_bytes_per_point": per_pt}
    # the oracle's definitional test on a fixed 2M-point sample
    O.build()
    idx = np.arange(0, n, max(1, n // 2_000_000))[:2_000_000]
    sp = pts.take(idx)
    ti = torch.from_numpy(idx.astype(np.int64)).to(dev)
    sdb.join_aggregate(xs[ti].contiguous(), ys[ti].contiguous(), at[ti].contiguous(), cov,
                       sdb.LOOKUP_TABLE_LEARNED, cnt, sm, stream)
    torch.cuda.synchronize()
    oc, os_, _ = O.join_o2(T, eps, sp, threads=os.cpu_count() or 1)
    out["matches_oracle"] = bool(np.array_equal(cnt.cpu().numpy().view(np.uint64), oc)
                                 and np.array_equal(sm.cpu().numpy(), os_))
    out["oracle_check"] = f"{len(idx)} points (every {max(1, n // 2_000_000)}th), O2"
    cov.free()
    del cnt, sm
    torch.cuda.empty_cache()
    # eps = 2^5 itself, tiled: the grid's 32 x 32 level-5 quadtree cells as
    # viewport queries over the resident (Hilbert-ordered) points, 32 tiles a
    # batch; per polygon the tiles' answers add up to the whole grid's
    out["tiled"] = config3_tiled(sdb, torch, dev, stream, T, xs, ys, at, pts, n, idx)
    del xs, ys, at
    torch.cuda.empty_cache()
    return out


C3_TILE_LEVEL, C3_TILED_EPS, C3_TILES_PER_BATCH = 5, 2 ** 5, 32


def tiled_join(sdb, torch, dev, stream, T, p, qb, lookups, timing=True):
    """Per polygon COUNT and SUM over all tiles for each lookup (device tensors),
    with the build and join times."""
    P = T.n
    rows = [tuple(int(v) for v in r) for r in qb.queries]
    tot = {lk: (torch.zeros(P, dtype=torch.int64, device=dev),
                torch.zeros(P, dtype=torch.int64, device=dev)) for lk in lookups}
    build_s, join_ms = 0.0, {lk: 0.0 for lk in lookups}
    cells = ranges = max_ranges = 0
    fallbacks = 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for g0 in range(0, len(rows), C3_TILES_PER_BATCH):
        grp = rows[g0:g0 + C3_TILES_PER_BATCH]
        base = grp[0][5]
        end = grp[-1][5] + grp[-1][6]
        ids = qb.subset_ids[base:end]
        grp = [r[:5] + (r[5] - base, r[6]) for r in grp]
        t = time.perf_counter()
        b = sdb.batch_create(p, T, grp, ids, stream)
        build_s += time.perf_counter() - t
        inf = b.info()
        cells += inf.n_cells
        ranges += inf.n_ranges
        max_ranges = max(max_ranges, inf.max_ranges)
        idt = torch.from_numpy(ids.astype(np.int64)).to(dev)
        cnt = torch.zeros(max(1, inf.out_len), dtype=torch.int64, device=dev)
        sm = torch.zeros(max(1, inf.out_len), dtype=torch.int64, device=dev)
        for lk in lookups:
            sdb.batch_set_lookup(b, lk, stream)
            if timing:
                sdb.batch_run(b, sdb.BATCH_PERSISTENT, cnt, sm, stream)  # warm
            e0.record(stream)
            sdb.batch_run(b, sdb.BATCH_PERSISTENT, cnt, sm, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            join_ms[lk] += e0.elapsed_time(e1)
            if lk == sdb.LOOKUP_LEARNED:
                fallbacks += sdb.batch_fallbacks(b, stream)
            tot[lk][0].index_add_(0, idt, cnt[:inf.out_len])
            tot[lk][1].index_add_(0, idt, sm[:inf.out_len])
        b.free()
        del cnt, sm, idt
    return tot, {"build_s": build_s, "join_ms": join_ms, "cells": cells, "ranges": ranges,
                 "max_ranges_per_tile": max_ranges, "fallbacks": fallbacks}


def config3_tiled(sdb, torch, dev, stream, T, xs, ys, at, pts, n, idx):
    from oracle import oracle as O
    from paper_2010_12548_gb300 import workloads as W
    qb = W.tile_queries(T, 28, C3_TILE_LEVEL, C3_TILED_EPS)
    t = time.perf_counter()
    p = sdb.points_create(xs, ys, at, 28, stream)
    torch.cuda.synchronize()
    resident_s = time.perf_counter() - t
    lks = (sdb.LOOKUP_LEARNED, sdb.LOOKUP_BINARY)
    tot, st = tiled_join(sdb, torch, dev, stream, T, p, qb, lks)
    p.free()
    out = {"eps": C3_TILED_EPS, "tiles": len(qb.queries), "tile_level": C3_TILE_LEVEL,
           "tiles_per_batch": C3_TILES_PER_BATCH, "resident_set_s": resident_s,
           "covering_build_s": st["build_s"], "cells": st["cells"], "ranges": st["ranges"],
           "max_ranges_per_tile": st["max_ranges_per_tile"], "learned_fallbacks": st["fallbacks"],
           "learned_join_ms": st["join_ms"][sdb.LOOKUP_LEARNED],
           "binary_join_ms": st["join_ms"][sdb.LOOKUP_BINARY]}
    out["learned_points_per_s"] = n / (out["learned_join_ms"] / 1e3)
    out["binary_points_per_s"] = n / (out["binary_join_ms"] / 1e3)
    a, b = tot[sdb.LOOKUP_LEARNED], tot[sdb.LOOKUP_BINARY]
    out["lookups_agree"] = bool(torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]))
    out["every_point_counted"] = bool(int(a[0].sum().item()) >= n)
    # the sample, tiled the same way, against the definitional test at eps 2^5
    ti = torch.from_numpy(idx.astype(np.int64)).to(dev)
    sp = sdb.points_create(xs[ti].contiguous(), ys[ti].contiguous(), at[ti].contiguous(), 28,
                           stream)
    stot, _ = tiled_join(sdb, torch, dev, stream, T, sp, qb, (sdb.LOOKUP_LEARNED,), timing=False)
    sp.free()
    sample = pts.take(idx)
    oc, os_, _ = O.join_o2(T, C3_TILED_EPS, sample, threads=os.cpu_count() or 1)
    c, s_ = stot[sdb.LOOKUP_LEARNED]
    out["matches_oracle"] = bool(np.array_equal(c.cpu().numpy().view(np.uint64), oc)
                                 and np.array_equal(s_.cpu().numpy(), os_))
    out["oracle_check"] = f"{len(idx)} sampled points tiled the same way vs O2 at eps 2^5"
    return out


def resident_legs(args, legs, sdb, torch, dev, stream):
    """Batched level-of-detail queries (4,096 queries over 200M resident points)
    and serving (Poisson arrivals of zoom-session queries over 500M points)."""
    from paper_2010_12548_gb300 import workloads as W
    out = {}
    T = W.tracts40k_tiling()
    n_all = max(args.lod_points if "batch" in legs else 0,
                args.serve_points if "serve" in legs else 0,
                args.pi_points if "pointindex" in legs else 0,
                args.c3_points if "config3" in legs else 0)
    pts = W.resident_points(n_all)  # a shorter set is a prefix of a longer one

    def resident(n):
        xs = torch.from_numpy(pts.x[:n].view(np.int32)).to(dev)
        ys = torch.from_numpy(pts.y[:n].view(np.int32)).to(dev)
        at = torch.from_numpy(pts.attr[:n]).to(dev)
        p = sdb.points_create(xs, ys, at, 28, stream)
        del xs, ys, at
        torch.cuda.empty_cache()
        return p

    if "batch" in legs:
        qb = W.lod_queries(W.BASE_SEED + 4, args.lod_queries, T)
        rows = [tuple(r) for r in qb.queries]
        p = resident(args.lod_points)
        t = time.perf_counter()
        b = sdb.batch_create(p, T, rows, qb.subset_ids, stream)
        build_s = time.perf_counter() - t
        tile, ppt = sdb.batch_autotune(b, stream)
        inf = b.info()
        cnt = torch.zeros(inf.out_len, dtype=torch.int64, device=dev)
        sm = torch.zeros(inf.out_len, dtype=torch.int64, device=dev)
        side = torch.cuda.Stream()
        with torch.cuda.stream(side):
            ms = {m: timed(torch, side, lambda m=m: sdb.batch_run(b, m, cnt, sm, side), 5)
                  for m in (sdb.BATCH_PERSISTENT, sdb.BATCH_GRAPH, sdb.BATCH_PER_QUERY)}
        ref_c, ref_s = cnt.clone(), sm.clone()
        t = time.perf_counter()
        sdb.batch_set_lookup(b, sdb.LOOKUP_LEARNED, stream)
        index_s = time.perf_counter() - t
        linf = b.info()
        with torch.cuda.stream(side):
            lms = {m: timed(torch, side, lambda m=m: sdb.batch_run(b, m, cnt, sm, side), 5)
                   for m in (sdb.BATCH_PERSISTENT, sdb.BATCH_GRAPH, sdb.BATCH_PER_QUERY)}
        learned_same = bool(torch.equal(cnt, ref_c) and torch.equal(sm, ref_s))
        learned_fb = sdb.batch_fallbacks(b, stream)
        out["batched"] = {
            "workload": f"lod{args.lod_queries}_tracts40k_pts{args.lod_points // 1_000_000}M_g28",
            "queries": inf.n_queries, "pairs": inf.n_pairs, "ranges": inf.n_ranges,
            "max_ranges": inf.max_ranges, "cells": inf.n_cells, "candidate_points": inf.candidates,
            "covering_build_s": build_s, "tile": tile, "points_per_thread": ppt,
            "persistent_ms": ms[sdb.BATCH_PERSISTENT], "graph_ms": ms[sdb.BATCH_GRAPH],
            "per_query_launches_ms": ms[sdb.BATCH_PER_QUERY],
            "queries_per_s_graph": inf.n_queries / (ms[sdb.BATCH_GRAPH] / 1e3),
            "candidate_points_per_s_graph": inf.candidates / (ms[sdb.BATCH_GRAPH] / 1e3),
            "learned": {"index_build_s": index_s, "indexed_queries": linf.indexed_queries,
                        "leaves": linf.n_leaves, "persistent_ms": lms[sdb.BATCH_PERSISTENT],
                        "graph_ms": lms[sdb.BATCH_GRAPH],
                        "per_query_launches_ms": lms[sdb.BATCH_PER_QUERY],
                        "queries_per_s_graph": inf.n_queries / (lms[sdb.BATCH_GRAPH] / 1e3),
                        "same_as_binary": learned_same, "fallbacks": learned_fb}}
        b.free()
        p.free()
        del cnt, sm
        torch.cuda.empty_cache()
    if "config3" in legs:
        out["config3"] = config3_leg(args, sdb, torch, dev, stream, T, pts)
    if "pointindex" in legs:
        out["point_index"] = point_index_leg(args, sdb, torch, dev, stream, T, pts, resident)
    if "serve" in legs:
        sessions = W.zoom_sessions(W.BASE_SEED + 5, 512, T)
        queries = [q for ss in sessions for q in ss]
        p = resident(args.serve_points)
        rates = [int(r) for r in args.serve_rates.split(",") if r]
        serving = {"workload": f"zoom512sessions_tracts40k_pts{args.serve_points // 1_000_000}M_g28",
                   "queries_in_pool": len(queries), "batched_learned": [], "batched": [],
                   "plain": [],
                   "plain_note": "one query per launch, binary search, no covering cache: it "
                                 "sustains under 1k queries/s, so at higher rates its queue "
                                 "grows for the whole run (600 queries) and the percentiles "
                                 "measure that backlog"}
        for kind, cfg in (("batched_learned", dict(workers=4, max_batch=256, cache_bytes=40 << 30,
                                                   lookup=sdb.LOOKUP_LEARNED)),
                          ("batched", dict(workers=4, max_batch=256, cache_bytes=40 << 30)),
                          ("plain", dict(workers=1, max_batch=1, use_cache=False,
                                         per_query=True))):
            for rate in rates:
                srv = sdb.server_create(p, T, **cfg)
                n = int(min(4000, max(400, rate * 2)))
                if kind == "plain":
                    n = min(n, 600)
                lat, bs, hits, wall, span, offered, lag = poisson_serve(sdb, srv, queries,
                                                                        rate, n, seed=rate)
                st = srv.stats()
                srv.destroy()
                serving[kind].append({
                    "rate": rate, "queries": n, "p50_ms": float(np.percentile(lat, 50)),
                    "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
                    "throughput_qps": n / span, "span_s": span,
                    "offered_qps": n / offered,
                    "wall_s_with_collection": float(wall),
                    "submit_lag_p99_ms": float(np.percentile(lag, 99)),
                    "submit_lag_max_ms": float(lag.max()), "mean_batch": float(bs.mean()),
                    "cache_hit_rate": hits / n, "batches": int(st.batches),
                    "cache_bytes": int(st.peak_bytes)})
        out["serving"] = serving
        p.free()
    return out


if __name__ == "__main__":
    main()
