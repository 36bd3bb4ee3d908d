"""Seeded synthetic inputs shaped like the paper's mobility workloads.

This module is shared by the CUDA path's tests and benchmark and by the CPU
oracle's tests.  It holds no part of the method's arithmetic (no curve, no
covering, no lookup): only the polygons and points that the method consumes.

Workloads (stand-ins for the NYC taxi points and the NYC zone / census polygon
sets used in Sec. 3 and Sec. 5 of the paper, which are not available here):

* star polygons: random star-shaped simple polygons around an integer centre
  (sorted distinct angles, per-vertex radius), overlaps allowed;
* Voronoi tilings: the bounded Voronoi diagram of random seeds over the grid
  square, every shared edge subdivided once with integer jitter, so the
  polygons tile the square exactly (no gaps, no overlaps);
* points: uniform, or a mobility-like mix of Gaussian clusters and uniform
  background, each with a log-normal int32 "fare" attribute.

All randomness comes from numpy's PCG64 seeded per workload.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 2010125480  # workload i uses BASE_SEED + i


@dataclass
class Polygons:
    """One simple ring per polygon, CSR layout, integer vertices.

    ring_off[j]..ring_off[j+1] index polygon j's vertices in x/y.  Rings are
    counter-clockwise and carry no closing duplicate vertex.
    """
    ring_off: np.ndarray  # uint32 [P+1]
    x: np.ndarray         # uint32 [V]
    y: np.ndarray         # uint32 [V]
    grid_bits: int
    centres: np.ndarray | None = None  # int64 [P,2] kernel point of star polygons

    @property
    def n(self) -> int:
        return len(self.ring_off) - 1

    def ring(self, j: int) -> tuple[np.ndarray, np.ndarray]:
        a, b = int(self.ring_off[j]), int(self.ring_off[j + 1])
        return self.x[a:b].astype(np.int64), self.y[a:b].astype(np.int64)

    def subset(self, ids) -> "Polygons":
        ids = np.asarray(ids, dtype=np.int64)
        xs, ys, off = [], [], [0]
        for j in ids:
            rx, ry = self.ring(int(j))
            xs.append(rx)
            ys.append(ry)
            off.append(off[-1] + len(rx))
        c = None if self.centres is None else self.centres[ids]
        return Polygons(np.asarray(off, np.uint32), np.concatenate(xs).astype(np.uint32),
                        np.concatenate(ys).astype(np.uint32), self.grid_bits, c)


@dataclass
class MultiPolygons:
    """Polygons of one or more rings (outer boundaries and holes), CSR layout:
    polygon j owns rings poly_ring_off[j]..poly_ring_off[j+1], ring r the
    vertices ring_off[r]..ring_off[r+1] of x/y (no closing duplicate).  A
    polygon's region is the set of points with an odd crossing number over all
    of its rings, together with the rings themselves."""
    poly_ring_off: np.ndarray  # uint32 [P+1]
    ring_off: np.ndarray       # uint32 [R+1]
    x: np.ndarray              # uint32 [V]
    y: np.ndarray              # uint32 [V]
    grid_bits: int

    @property
    def n(self) -> int:
        return len(self.poly_ring_off) - 1


@dataclass
class Points:
    x: np.ndarray     # uint32 [N]
    y: np.ndarray     # uint32 [N]
    attr: np.ndarray  # int32 [N]
    grid_bits: int

    @property
    def n(self) -> int:
        return len(self.x)

    def take(self, idx) -> "Points":
        return Points(self.x[idx], self.y[idx], self.attr[idx], self.grid_bits)


# --------------------------------------------------------------------------
# polygon simplicity (used to reject and resample jittered rings)
# --------------------------------------------------------------------------

def _orient(ax, ay, bx, by, cx, cy):
    return (bx - ax) * (cy - ay) - (by - ay) * (cx - ax)


def _shift(a, k):
    """a rotated left by k (a cheaper np.roll(a, -k) for 1-D arrays)."""
    return np.concatenate((a[k:], a[:k]))


def ring_is_simple(rx: np.ndarray, ry: np.ndarray) -> bool:
    """Exact integer check that a closed ring has no self-contact.

    Non-adjacent edges must not meet (closed-segment test); adjacent edges
    must not fold back onto each other.  O(V^2), one pairwise pass.
    """
    rx = np.asarray(rx, np.int64)
    ry = np.asarray(ry, np.int64)
    n = len(rx)
    if n < 3:
        return False
    ax, ay = rx, ry
    bx, by = _shift(rx, 1), _shift(ry, 1)
    if np.any((ax == bx) & (ay == by)):
        return False
    # adjacent edges: fold-back = collinear with opposite direction
    cx, cy = _shift(rx, 2), _shift(ry, 2)
    cr = _orient(ax, ay, bx, by, cx, cy)
    dot = (bx - ax) * (cx - bx) + (by - ay) * (cy - by)
    if np.any((cr == 0) & (dot < 0)):
        return False
    if n == 3:
        return _orient(ax[0], ay[0], bx[0], by[0], cx[0], cy[0]) != 0
    # all pairs (i, j) of non-adjacent edges, i < j
    i, j = np.triu_indices(n, 2)
    keep = ~((i == 0) & (j == n - 1))
    i, j = i[keep], j[keep]
    px, py, qx, qy = ax[i], ay[i], bx[i], by[i]
    sx, sy, tx, ty = ax[j], ay[j], bx[j], by[j]
    o1 = np.sign(_orient(px, py, qx, qy, sx, sy))
    o2 = np.sign(_orient(px, py, qx, qy, tx, ty))
    o3 = np.sign(_orient(sx, sy, tx, ty, px, py))
    o4 = np.sign(_orient(sx, sy, tx, ty, qx, qy))
    if np.any((o1 * o2 < 0) & (o3 * o4 < 0)):
        return False

    def within(ux, uy, vx, vy, wx, wy):
        return ((np.minimum(ux, vx) <= wx) & (wx <= np.maximum(ux, vx)) &
                (np.minimum(uy, vy) <= wy) & (wy <= np.maximum(uy, vy)))
    touch = (((o1 == 0) & within(px, py, qx, qy, sx, sy)) |
             ((o2 == 0) & within(px, py, qx, qy, tx, ty)) |
             ((o3 == 0) & within(sx, sy, tx, ty, px, py)) |
             ((o4 == 0) & within(sx, sy, tx, ty, qx, qy)))
    return not np.any(touch)


def _signed_area2(rx, ry):
    rx = np.asarray(rx, np.int64)
    ry = np.asarray(ry, np.int64)
    return int(np.sum(rx * _shift(ry, 1) - _shift(rx, 1) * ry))


# --------------------------------------------------------------------------
# star polygons
# --------------------------------------------------------------------------

def star_polygons(rng: np.random.Generator, n: int, grid_bits: int,
                  nverts=(8, 32), radius=(2 ** 11, 2 ** 12)) -> Polygons:
    """Random star-shaped simple polygons with integer vertices.

    Angles are sorted distinct uniform draws, each vertex has its own radius
    uniform in ``radius``.  The centre is an integer point drawn uniformly
    from the part of the grid where no vertex needs clamping, so the ring is
    star-shaped with respect to the centre (checked exactly: every
    consecutive pair turns counter-clockwise around the centre and the ring
    winds once).
    """
    G = 2 ** grid_bits
    rmax = int(math.ceil(radius[1])) + 1
    if 2 * rmax >= G:
        raise ValueError("radius too large for the grid")
    xs, ys, off, cs = [], [], [0], []
    while len(cs) < n:
        k = int(rng.integers(nverts[0], nverts[1] + 1))
        c = rng.integers(rmax, G - 1 - rmax, size=2)
        th = np.sort(rng.uniform(0.0, 2 * math.pi, size=k))
        r = rng.uniform(radius[0], radius[1], size=k)
        vx = np.rint(c[0] + r * np.cos(th)).astype(np.int64)
        vy = np.rint(c[1] + r * np.sin(th)).astype(np.int64)
        dx, dy = vx - c[0], vy - c[1]
        cr = dx * np.roll(dy, -1) - np.roll(dx, -1) * dy
        if np.any(cr <= 0):
            continue
        turn = np.sum(np.mod(np.diff(np.append(np.arctan2(dy, dx), np.arctan2(dy[0], dx[0]))),
                             2 * math.pi))
        if abs(turn - 2 * math.pi) > 1e-6:
            continue
        xs.append(vx)
        ys.append(vy)
        off.append(off[-1] + k)
        cs.append(c.astype(np.int64))
    return Polygons(np.asarray(off, np.uint32), np.concatenate(xs).astype(np.uint32),
                    np.concatenate(ys).astype(np.uint32), grid_bits, np.asarray(cs, np.int64))


def _ring_around(rng, c, k, rlo, rhi):
    """k vertices at evenly spaced angles (jitter up to a quarter of the
    spacing, so consecutive angles differ by at most 1.5 spacings) with radii
    uniform in [rlo, rhi] around integer centre c."""
    step = 2 * math.pi / k
    th = np.arange(k) * step + rng.uniform(-0.25, 0.25, size=k) * step + rng.uniform(0, step)
    r = rng.uniform(rlo, rhi, size=k)
    return (np.rint(c[0] + r * np.cos(th)).astype(np.int64),
            np.rint(c[1] + r * np.sin(th)).astype(np.int64))


def holed_stars(rng: np.random.Generator, n: int, grid_bits: int, nverts=(6, 24),
                radius=(2 ** 10, 2 ** 11), p_hole: float = 0.5,
                p_part: float = 0.35) -> MultiPolygons:
    """Star polygons with holes and second parts (multi-polygons).

    The outer ring has k >= 6 vertices at jittered even angles, so no gap
    exceeds 90 degrees and every edge stays at least cos(45 deg) * r_min - 1
    from the centre; a hole (probability p_hole) is a ring around the same
    centre with radii at most r_min / 2, strictly inside.  A second part
    (probability p_part) is a smaller ring whose centre lies more than the
    sum of both circumradii away, so the parts are disjoint.  Polygons of the
    set may overlap each other."""
    G = 2 ** grid_bits
    r_hi = radius[1]
    margin = int(3 * r_hi) + 2
    if 2 * margin >= G:
        raise ValueError("radius too large for the grid")
    xs, ys, roff, poff = [], [], [0], [0]

    def add(vx, vy):
        xs.append(vx)
        ys.append(vy)
        roff.append(roff[-1] + len(vx))

    for _ in range(n):
        k = int(rng.integers(max(6, nverts[0]), nverts[1] + 1))
        c = rng.integers(margin, G - 1 - margin, size=2)
        rlo = rng.uniform(radius[0], r_hi)
        add(*_ring_around(rng, c, k, rlo, r_hi))
        if rng.random() < p_hole:
            add(*_ring_around(rng, c, int(rng.integers(3, 9)), rlo / 8, rlo / 2))
        if rng.random() < p_part:
            ang = rng.uniform(0, 2 * math.pi)
            d = r_hi + r_hi / 2 + 4
            c2 = np.rint(c + d * np.array([math.cos(ang), math.sin(ang)])).astype(np.int64)
            add(*_ring_around(rng, c2, int(rng.integers(3, 9)), r_hi / 6, r_hi / 2))
        poff.append(len(roff) - 1)
    return MultiPolygons(np.asarray(poff, np.uint32), np.asarray(roff, np.uint32),
                         np.concatenate(xs).astype(np.uint32), np.concatenate(ys).astype(np.uint32),
                         grid_bits)


# --------------------------------------------------------------------------
# Voronoi tilings
# --------------------------------------------------------------------------

def voronoi_tiling(rng: np.random.Generator, n: int, grid_bits: int,
                   nverts=(20, 400), jitter: float = 0.125,
                   min_piece: float = 16.0) -> Polygons:
    """Exact tiling of the square [0, 2^B - 1]^2 by jittered Voronoi cells.

    The bounded diagram comes from mirroring the seeds across the four sides
    of the square.  Voronoi vertices are rounded to integers once and shared.
    Every edge is subdivided once into pieces (both neighbours reuse the same
    points); interior edges get a perpendicular integer jitter of at most
    ``jitter`` times the piece length, edges on the square's border stay on
    it.  Per-polygon vertex targets are drawn uniformly from ``nverts``;
    a shared edge takes the smaller of its two polygons' per-edge share.
    Rings that come out non-simple are re-jittered with less amplitude.
    """
    from scipy.spatial import Voronoi

    M = float(2 ** grid_bits - 1)
    for _attempt in range(16):
        seeds = rng.uniform(0.0, M, size=(n, 2))
        mir = [seeds,
               np.c_[-seeds[:, 0], seeds[:, 1]], np.c_[2 * M - seeds[:, 0], seeds[:, 1]],
               np.c_[seeds[:, 0], -seeds[:, 1]], np.c_[seeds[:, 0], 2 * M - seeds[:, 1]]]
        vor = Voronoi(np.concatenate(mir))
        vint = np.clip(np.rint(vor.vertices), 0, M).astype(np.int64)
        regions = []
        ok = True
        for i in range(n):
            reg = vor.regions[vor.point_region[i]]
            if len(reg) < 3 or -1 in reg:
                ok = False
                break
            reg = list(reg)
            # merge vertices that round to the same integer point
            out = []
            for v in reg:
                if out and (vint[v] == vint[out[-1]]).all():
                    continue
                out.append(v)
            while len(out) > 1 and (vint[out[0]] == vint[out[-1]]).all():
                out.pop()
            if len(out) < 3:
                ok = False
                break
            if _signed_area2(vint[out, 0], vint[out, 1]) < 0:
                out = out[::-1]
            regions.append(out)
        if not ok:
            continue
        polys = _subdivide_tiling(rng, regions, vint, M, nverts, jitter, min_piece)
        if polys is not None:
            xs, ys, off = [], [], [0]
            for rx, ry in polys:
                xs.append(rx)
                ys.append(ry)
                off.append(off[-1] + len(rx))
            return Polygons(np.asarray(off, np.uint32), np.concatenate(xs).astype(np.uint32),
                            np.concatenate(ys).astype(np.uint32), grid_bits)
    raise RuntimeError("could not generate a simple Voronoi tiling")


def _subdivide_tiling(rng, regions, vint, M, nverts, jitter, min_piece):
    n = len(regions)
    edges_of = []
    uses: dict[tuple[int, int], list[int]] = {}
    for i, reg in enumerate(regions):
        es = []
        for a, b in zip(reg, reg[1:] + reg[:1]):
            key = (min(a, b), max(a, b))
            es.append(key)
            uses.setdefault(key, []).append(i)
        edges_of.append(es)
    target = rng.integers(nverts[0], nverts[1] + 1, size=n)
    share = target / np.asarray([len(e) for e in edges_of], np.float64)
    length = {k: float(np.hypot(*(vint[k[1]] - vint[k[0]]))) for k in uses}
    pieces = {}
    for k, us in uses.items():
        p = max(1, int(round(min(share[u] for u in us))))
        pieces[k] = max(1, min(p, int(length[k] // min_piece)))
    # top up rings below the minimum on their longest edges
    for i in range(n):
        for _ in range(64):
            tot = sum(pieces[k] for k in edges_of[i])
            if tot >= nverts[0]:
                break
            k = max(edges_of[i], key=lambda e: length[e] / (pieces[e] + 1))
            if length[k] // min_piece <= pieces[k]:
                break
            pieces[k] += 1
    for amp in (jitter, jitter / 2, jitter / 4, 0.0):
        sub_rng = np.random.default_rng(int(rng.integers(0, 2 ** 63)))
        pts = {}
        for k in sorted(uses):
            a, b = vint[k[0]].astype(np.float64), vint[k[1]].astype(np.float64)
            m = pieces[k]
            t = np.arange(1, m, dtype=np.float64) / m
            p = a[None, :] + t[:, None] * (b - a)[None, :]
            border = (a[0] == b[0] and a[0] in (0.0, M)) or (a[1] == b[1] and a[1] in (0.0, M))
            if m > 1 and not border and amp > 0:
                d = b - a
                nrm = np.array([-d[1], d[0]]) / max(np.hypot(*d), 1e-12)
                off = sub_rng.uniform(-amp, amp, size=m - 1) * (np.hypot(*d) / m)
                p = p + off[:, None] * nrm[None, :]
            pts[k] = np.clip(np.rint(p), 0, M).astype(np.int64)
        out = []
        good = True
        for i, reg in enumerate(regions):
            rx, ry = [], []
            for a, b in zip(reg, reg[1:] + reg[:1]):
                k = (min(a, b), max(a, b))
                inner = pts[k] if a < b else pts[k][::-1]
                rx.append(vint[a, 0])
                ry.append(vint[a, 1])
                rx.extend(inner[:, 0].tolist())
                ry.extend(inner[:, 1].tolist())
            rx = np.asarray(rx, np.int64)
            ry = np.asarray(ry, np.int64)
            keep = np.ones(len(rx), bool)
            keep[1:] = (rx[1:] != rx[:-1]) | (ry[1:] != ry[:-1])
            if len(rx) > 1 and rx[0] == rx[-1] and ry[0] == ry[-1]:
                keep[-1] = False
            rx, ry = rx[keep], ry[keep]
            if not ring_is_simple(rx, ry) or _signed_area2(rx, ry) <= 0:
                good = False
                break
            out.append((rx, ry))
        if good:
            return out
    return None


# --------------------------------------------------------------------------
# points
# --------------------------------------------------------------------------

def fare_attr(rng: np.random.Generator, n: int) -> np.ndarray:
    """int32 fare in cents: round(exp(N(7, 0.8)))."""
    return np.rint(np.exp(rng.normal(7.0, 0.8, size=n))).astype(np.int32)


def uniform_points(rng: np.random.Generator, n: int, grid_bits: int) -> Points:
    G = 2 ** grid_bits
    x = rng.integers(0, G, size=n, dtype=np.uint32)
    y = rng.integers(0, G, size=n, dtype=np.uint32)
    return Points(x, y, fare_attr(rng, n), grid_bits)


def mobility_points(seed: int, n: int, grid_bits: int, n_clusters: int,
                    sigma=(2 ** 16, 2 ** 19), frac_cluster: float = 0.7,
                    chunk: int = 1 << 22, threads: int | None = None) -> Points:
    """Cluster/uniform mix: ``frac_cluster`` of the points come from
    ``n_clusters`` isotropic Gaussians (centre uniform, sigma uniform in
    ``sigma``, truncated to the grid: a sample that rounds outside the grid
    is drawn again from its cluster, so no mass piles up on the grid's
    border), the rest are uniform.  Points appear in random order.  Generated
    in fixed-size chunks, each from its own child seed (so the result does
    not depend on memory limits or on the number of threads filling the
    chunks)."""
    import concurrent.futures as cf
    G = 2 ** grid_bits
    ss = np.random.SeedSequence(seed)
    head, body = ss.spawn(2)
    hr = np.random.default_rng(head)
    centres = hr.uniform(0, G, size=(n_clusters, 2))
    sig = hr.uniform(sigma[0], sigma[1], size=n_clusters)
    x = np.empty(n, np.uint32)
    y = np.empty(n, np.uint32)
    attr = np.empty(n, np.int32)
    nchunks = (n + chunk - 1) // chunk

    def fill(c, cs):
        r = np.random.default_rng(cs)
        a, b = c * chunk, min(n, (c + 1) * chunk)
        m = b - a
        is_c = r.random(m) < frac_cluster
        which = r.integers(0, n_clusters, size=m)
        g = r.standard_normal((m, 2))
        cx = centres[which, 0] + g[:, 0] * sig[which]
        cy = centres[which, 1] + g[:, 1] * sig[which]

        def outside(u, v):  # rounds to a coordinate outside [0, G)
            return (u < -0.5) | (u >= G - 0.5) | (v < -0.5) | (v >= G - 0.5)
        out = np.nonzero(is_c & outside(cx, cy))[0]
        for _ in range(64):
            if out.size == 0:
                break
            g = r.standard_normal((out.size, 2))
            cx[out] = centres[which[out], 0] + g[:, 0] * sig[which[out]]
            cy[out] = centres[which[out], 1] + g[:, 1] * sig[which[out]]
            out = out[outside(cx[out], cy[out])]
        ux = r.integers(0, G, size=m)
        uy = r.integers(0, G, size=m)
        px = np.where(is_c, np.clip(np.rint(cx), 0, G - 1), ux)
        py = np.where(is_c, np.clip(np.rint(cy), 0, G - 1), uy)
        x[a:b] = px.astype(np.uint32)
        y[a:b] = py.astype(np.uint32)
        attr[a:b] = fare_attr(r, m)

    seeds = body.spawn(nchunks)
    workers = threads or min(16, os.cpu_count() or 1)
    if nchunks <= 1 or workers <= 1:
        for c, cs in enumerate(seeds):
            fill(c, cs)
    else:
        with cf.ThreadPoolExecutor(workers) as ex:
            list(ex.map(fill, range(nchunks), seeds))
    return Points(x, y, attr, grid_bits)


# --------------------------------------------------------------------------
# the benchmark / test workloads
# --------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    grid_bits: int
    eps: list
    polygons: Polygons
    points: Points
    extra: dict = field(default_factory=dict)


def tiny_stars(n_points: int = 100_000) -> Workload:
    """100k uniform points on [0,2^16)^2, 16 overlapping star polygons with
    8-32 vertices and radii in [2^11, 2^12], eps = 64 grid units."""
    rng = np.random.default_rng(BASE_SEED + 0)
    polys = star_polygons(rng, 16, 16)
    pts = uniform_points(rng, n_points, 16)
    return Workload("stars16_pts100k_g16_eps64", 16, [64], polys, pts)


_TILING_CACHE: dict = {}


def _cached_tiling(key: str, make) -> Polygons:
    """Memory and disk cache of a generated tiling (generation is deterministic;
    the directory comes from SDB_WORKLOAD_CACHE, default a temp folder)."""
    if key in _TILING_CACHE:
        return _TILING_CACHE[key]
    import tempfile
    d = os.environ.get("SDB_WORKLOAD_CACHE", os.path.join(tempfile.gettempdir(), "sdb_workloads"))
    path = os.path.join(d, key + ".npz")
    T = None
    try:
        with np.load(path) as z:
            T = Polygons(z["ring_off"], z["x"], z["y"], int(z["grid_bits"]))
    except Exception:
        T = make()
        try:
            os.makedirs(d, exist_ok=True)
            tmp = path + f".{os.getpid()}.npz"
            np.savez(tmp, ring_off=T.ring_off, x=T.x, y=T.y, grid_bits=T.grid_bits)
            os.replace(tmp, path)
        except OSError:
            pass
    _TILING_CACHE[key] = T
    return T


def zones263_tiling() -> Polygons:
    """263-cell jittered Voronoi tiling of [0,2^24)^2, 20-400 vertices."""
    return _cached_tiling("zones263_g24_v1", lambda: voronoi_tiling(
        np.random.default_rng(BASE_SEED + 1), 263, 24, (20, 400)))


def tracts40k_tiling() -> Polygons:
    """40,000-cell jittered Voronoi tiling of [0,2^28)^2, 6-60 vertices."""
    return _cached_tiling("tracts40k_g28_v1", lambda: voronoi_tiling(
        np.random.default_rng(BASE_SEED + 2), 40_000, 28, (6, 60)))


def mobility_zones(n_points: int = 100_000_000) -> Workload:
    """Mobility-shaped scale-up: n points on [0,2^24)^2 (70% from 32
    Gaussian clusters, sigma in [2^16, 2^19]; 30% uniform) with fare
    attributes, the 263-zone tiling, eps sweep {2^12, 2^10, 2^8, 2^6}."""
    polys = zones263_tiling()
    pts = mobility_points(BASE_SEED + 101, n_points, 24, 32)
    return Workload(f"zones263_mobility{n_points}_g24", 24, [2 ** 12, 2 ** 10, 2 ** 8, 2 ** 6],
                    polys, pts)


# --------------------------------------------------------------------------
# level-of-detail query batches
# --------------------------------------------------------------------------

@dataclass
class QueryBatch:
    """Viewport queries: rows (x0, y0, x1, y1, eps, poly_off, poly_cnt) and the
    concatenated polygon subsets."""
    queries: np.ndarray     # int64 [Q, 7]
    subset_ids: np.ndarray  # uint32


def polygon_bboxes(P: Polygons) -> np.ndarray:
    """[P, 4] (minx, miny, maxx, maxy) per polygon."""
    off = P.ring_off.astype(np.int64)
    seg = np.repeat(np.arange(P.n), np.diff(off))
    out = np.empty((P.n, 4), np.int64)
    for c, (arr, fn) in enumerate(((P.x, np.minimum), (P.y, np.minimum), (P.x, np.maximum),
                                   (P.y, np.maximum))):
        init = np.iinfo(np.int64).max if fn is np.minimum else -1
        acc = np.full(P.n, init, np.int64)
        fn.at(acc, seg, arr.astype(np.int64))
        out[:, c] = acc
    return out


def lod_queries(seed: int, n: int, polys: Polygons, side=(2 ** 14, 2 ** 24),
                subset=(1, 5000), eps_levels=tuple(2 ** e for e in range(14, 5, -1))) -> QueryBatch:
    """Level-of-detail queries: viewport side log-uniform in ``side`` (square,
    uniform position inside the grid), eps uniform over ``eps_levels``, and a
    polygon subset of size uniform in ``subset``: a random choice among the
    polygons whose bounding box meets the viewport, filled up with random other
    polygons when fewer meet it (a view's layer of regions plus unrelated
    ones)."""
    rng = np.random.default_rng(seed)
    G = 2 ** polys.grid_bits
    bb = polygon_bboxes(polys)
    rows, ids = [], []
    for _ in range(n):
        s = int(np.exp(rng.uniform(np.log(side[0]), np.log(side[1]))))
        s = max(1, min(s, G))
        x0 = int(rng.integers(0, G - s + 1))
        y0 = int(rng.integers(0, G - s + 1))
        eps = int(eps_levels[rng.integers(0, len(eps_levels))])
        k = int(rng.integers(subset[0], subset[1] + 1))
        k = min(k, polys.n)
        meet = np.nonzero((bb[:, 0] < x0 + s) & (bb[:, 2] >= x0) &
                          (bb[:, 1] < y0 + s) & (bb[:, 3] >= y0))[0]
        if len(meet) >= k:
            sub = rng.choice(meet, size=k, replace=False)
        else:
            rest = np.setdiff1d(np.arange(polys.n), meet)
            sub = np.concatenate([meet, rng.choice(rest, size=k - len(meet), replace=False)])
            rng.shuffle(sub)
        rows.append((x0, y0, x0 + s, y0 + s, eps, sum(len(i) for i in ids), k))
        ids.append(sub.astype(np.uint32))
    return QueryBatch(np.asarray(rows, np.int64),
                      np.concatenate(ids) if ids else np.zeros(0, np.uint32))


def tile_queries(polys: Polygons, grid_bits: int, tile_level: int, eps: int,
                 margin: int = 1 << 12) -> QueryBatch:
    """The grid cut into 4^tile_level square tiles (quadtree cells of level
    tile_level, row-major), one viewport query per tile at eps, its subset the
    polygons whose bounding box, grown by ``margin`` grid units, meets the tile
    (a superset of the polygons that can reach it for any finest side up to the
    margin).  The queries of all tiles together partition the grid, so the
    per-polygon sums of their answers are the whole grid's answer."""
    side = 1 << (grid_bits - tile_level)
    bb = polygon_bboxes(polys)
    rows, ids, off = [], [], 0
    n = 1 << tile_level
    for ty in range(n):
        for tx in range(n):
            x0, y0 = tx * side, ty * side
            x1, y1 = x0 + side, y0 + side
            hit = np.nonzero((bb[:, 0] - margin < x1) & (bb[:, 2] + margin >= x0) &
                             (bb[:, 1] - margin < y1) & (bb[:, 3] + margin >= y0))[0]
            rows.append((x0, y0, x1, y1, eps, off, len(hit)))
            ids.append(hit.astype(np.uint32))
            off += len(hit)
    return QueryBatch(np.asarray(rows, np.int64), np.concatenate(ids))


def resident_points(n_points: int) -> Points:
    """Points on [0,2^28)^2 for the level-of-detail and serving workloads: 70%
    from 64 Gaussian clusters (sigma in [2^20, 2^23], clipped), 30% uniform.
    A shorter set is a prefix of a longer one (same chunks)."""
    return mobility_points(BASE_SEED + 104, n_points, 28, 64, sigma=(2 ** 20, 2 ** 23))


def lod_workload(n_points: int = 200_000_000, n_queries: int = 4096) -> tuple:
    """4,096 level-of-detail queries over 200M resident points on [0,2^28)^2
    and the 40,000-polygon tiling; eps from {2^14 .. 2^6}."""
    T = tracts40k_tiling()
    qb = lod_queries(BASE_SEED + 4, n_queries, T)
    return T, resident_points(n_points), qb


def zoom_sessions(seed: int, n_sessions: int, polys: Polygons, start_side: int = 2 ** 24,
                  start_eps: int = 2 ** 14, zooms=(5, 20), max_polys: int = 5000) -> list:
    """Zoom sessions: from a square viewport of side ``start_side`` at a
    uniform position, each step halves the side (around a point uniform in the
    middle half of the current view) and halves eps, for a number of steps
    uniform in ``zooms``; eps stops at 2, the side at 1.  Each query asks for
    the polygons whose bounding box meets its viewport (at most ``max_polys``,
    in id order).  Returns a list of sessions, each a list of (query row, ids)
    with rows (x0, y0, x1, y1, eps, 0, n)."""
    rng = np.random.default_rng(seed)
    G = 2 ** polys.grid_bits
    bb = polygon_bboxes(polys)
    out = []
    for _ in range(n_sessions):
        side = min(start_side, G)
        x0 = int(rng.integers(0, G - side + 1))
        y0 = int(rng.integers(0, G - side + 1))
        eps = start_eps
        steps = int(rng.integers(zooms[0], zooms[1] + 1))
        sess = []
        for _ in range(steps):
            meet = np.nonzero((bb[:, 0] < x0 + side) & (bb[:, 2] >= x0) &
                              (bb[:, 1] < y0 + side) & (bb[:, 3] >= y0))[0][:max_polys]
            sess.append(((x0, y0, x0 + side, y0 + side, eps, 0, len(meet)),
                         meet.astype(np.uint32)))
            # zoom in around a point of the middle half of the view
            cx = x0 + side // 4 + int(rng.integers(0, max(1, side // 2)))
            cy = y0 + side // 4 + int(rng.integers(0, max(1, side // 2)))
            side = max(1, side // 2)
            x0 = min(max(0, cx - side // 2), G - side)
            y0 = min(max(0, cy - side // 2), G - side)
            eps = max(2, eps // 2)
        out.append(sess)
    return out


def serving_workload(n_points: int = 500_000_000, n_sessions: int = 512) -> tuple:
    """500M resident points on [0,2^28)^2 (cluster/uniform mix as the
    level-of-detail workload) and zoom sessions over the 40,000-polygon
    tiling."""
    T = tracts40k_tiling()
    return T, resident_points(n_points), zoom_sessions(BASE_SEED + 5, n_sessions, T)
