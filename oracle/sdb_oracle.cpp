// CPU oracle for the distance-bounded approximate point-in-polygon join.
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
// statement of what the GPU path computes.  Only the tests, the smoke check
// and the benchmark's CPU-baseline leg may load it.  It shares no code, header,
// table or helper with the CUDA library, and the CUDA library never calls it.
//
// What it follows (paper: "The Case for Distance-Bounded Spatial
// Approximations", CIDR 2021):
//   * Sec. 2.2: a geometry is eps-approximated when the Hausdorff distance is
//     at most eps; boundary cells get side eps/sqrt(2) so their diagonal is eps;
//     interior cells may be larger; a conservative raster keeps every cell that
//     touches the boundary (false positives only).
//   * Sec. 2.1 / Fig. 1c: hierarchical raster = variable-size quadtree cells.
//   * Sec. 3: cells are linearised by a space-filling curve (Hilbert or Z);
//     polygons are indexed by their cells, a query point is mapped to its cell
//     on the finest level and looked up.
//   * Sec. 5 / Sec. 5.1: SELECT AGG(a) FROM P, R WHERE P.loc INSIDE R.geometry
//     GROUP BY R.id, evaluated as an index-nested-loop join fused with the
//     aggregation and with no exact geometric test.
//
// Readings where the paper is silent (each one is listed in the design notes):
//   * cells are closed squares, polygons closed regions: a cell counts for a
//     polygon when the two intersect (a touch is enough);
//   * the finest side is the largest power of two s with 2 s^2 <= eps^2;
//   * a lattice point (x, y) belongs to the finest cell (floor(x/s), floor(y/s));
//   * the Hilbert curve is the quadrant-digit curve whose order-1 visit order is
//     (0,0), (0,1), (1,1), (1,0);
//   * the covering is the canonical list of maximal Hilbert-id ranges on which
//     the set of covering polygons is constant, lists ascending and unique.
//
// Everything is exact integer arithmetic (int64, __int128 for squared
// distances); there is no floating point.  Points outside [0, 2^B)^2 match no
// polygon.

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <thread>
#include <vector>

namespace {

typedef int64_t i64;
typedef unsigned __int128 u128;
typedef __int128 i128;

// One polygon: one or more closed rings (outer boundaries and holes); the
// region is the set of points with an odd crossing number over all rings, plus
// the rings themselves (closed).  Edge i runs from vertex i to vertex nxt[i],
// the next vertex of the same ring.
struct Ring {
  std::vector<i64> x, y;
  std::vector<size_t> nxt;
  i64 minx, miny, maxx, maxy;
};

void finish_ring(Ring& r) {
  r.minx = *std::min_element(r.x.begin(), r.x.end());
  r.maxx = *std::max_element(r.x.begin(), r.x.end());
  r.miny = *std::min_element(r.y.begin(), r.y.end());
  r.maxy = *std::max_element(r.y.begin(), r.y.end());
}

void add_ring(Ring& r, const uint32_t* vx, const uint32_t* vy, uint32_t a, uint32_t b) {
  const size_t base = r.x.size();
  for (uint32_t v = a; v < b; ++v) {
    r.x.push_back(vx[v]);
    r.y.push_back(vy[v]);
    r.nxt.push_back(v + 1 < b ? base + (v - a) + 1 : base);
  }
}

std::vector<Ring> load_rings(uint32_t P, const uint32_t* off, const uint32_t* vx, const uint32_t* vy) {
  std::vector<Ring> rs(P);
  for (uint32_t j = 0; j < P; ++j) {
    add_ring(rs[j], vx, vy, off[j], off[j + 1]);
    finish_ring(rs[j]);
  }
  return rs;
}

// polygon j = rings [poly_ring_off[j], poly_ring_off[j+1]), ring r = vertices
// [ring_off[r], ring_off[r+1])
std::vector<Ring> load_multi(uint32_t P, const uint32_t* poly_ring_off, const uint32_t* ring_off,
                             const uint32_t* vx, const uint32_t* vy) {
  std::vector<Ring> rs(P);
  for (uint32_t j = 0; j < P; ++j) {
    for (uint32_t r = poly_ring_off[j]; r < poly_ring_off[j + 1]; ++r)
      add_ring(rs[j], vx, vy, ring_off[r], ring_off[r + 1]);
    finish_ring(rs[j]);
  }
  return rs;
}

// --- Sec. 2.2: finest cell side --------------------------------------------
// side s = 2^k, the largest power of two whose diagonal s*sqrt(2) is <= eps,
// i.e. 2 s^2 <= eps^2.  k is capped at B (one cell covering the whole grid).
int finest_k(uint64_t eps, uint32_t B, uint32_t* k_out) {
  if (eps < 2) return -1;  // even s = 1 has diagonal sqrt(2) > eps
  u128 e2 = (u128)eps * eps;
  uint32_t k = 0;
  while (k < 62) {
    u128 s = (u128)1 << (k + 1);
    if (2 * s * s <= e2) ++k; else break;
  }
  if (k > B) k = B;
  *k_out = k;
  return 0;
}

// --- Sec. 3: linearisation ----------------------------------------------------
// Hilbert index of cell (x, y) on a 2^order x 2^order grid.  At each level the
// quadrant digit is read from the current coordinates' top bits: 0 for (0,0),
// 1 for (0,1), 2 for (1,1), 3 for (1,0).  The remaining lower-order part is then
// re-oriented: for quadrant (0,0) it is mirrored about the diagonal (x<->y);
// for quadrant (1,0) it is mirrored about the anti-diagonal (both coordinates
// complemented within the sub-square, then exchanged).
uint64_t hilbert(uint32_t order, uint64_t x, uint64_t y) {
  uint64_t d = 0;
  for (int lev = (int)order - 1; lev >= 0; --lev) {
    uint64_t bx = (x >> lev) & 1u, by = (y >> lev) & 1u;
    uint64_t digit;
    if (bx == 0 && by == 0) digit = 0;
    else if (bx == 0 && by == 1) digit = 1;
    else if (bx == 1 && by == 1) digit = 2;
    else digit = 3;
    d = d * 4 + digit;
    uint64_t side = (uint64_t)1 << lev;  // sub-square side
    uint64_t lx = x & (side - 1), ly = y & (side - 1);
    if (by == 0) {
      if (bx == 1) {
        lx = side - 1 - lx;
        ly = side - 1 - ly;
      }
      std::swap(lx, ly);
    }
    x = lx;
    y = ly;
  }
  return d;
}

// Z-order (Morton) index: x bit i goes to position 2i+1, y bit i to 2i.
uint64_t zorder(uint32_t order, uint64_t x, uint64_t y) {
  uint64_t d = 0;
  for (uint32_t i = 0; i < order; ++i) {
    d |= ((x >> i) & 1u) << (2 * i + 1);
    d |= ((y >> i) & 1u) << (2 * i);
  }
  return d;
}

uint64_t curve(int which, uint32_t order, uint64_t x, uint64_t y) {
  return which == 0 ? hilbert(order, x, y) : zorder(order, x, y);
}

// --- exact predicates ---------------------------------------------------------
int sgn(i64 v) { return (v > 0) - (v < 0); }

// sign of the cross product (b - a) x (c - a)
int orient(i64 ax, i64 ay, i64 bx, i64 by, i64 cx, i64 cy) {
  return sgn((bx - ax) * (cy - ay) - (by - ay) * (cx - ax));
}

// c is collinear with segment ab: does it lie on the closed segment?
bool between(i64 ax, i64 ay, i64 bx, i64 by, i64 cx, i64 cy) {
  return std::min(ax, bx) <= cx && cx <= std::max(ax, bx) &&
         std::min(ay, by) <= cy && cy <= std::max(ay, by);
}

// closed segments ab and cd share at least one point
bool segments_meet(i64 ax, i64 ay, i64 bx, i64 by, i64 cx, i64 cy, i64 dx, i64 dy) {
  int o1 = orient(ax, ay, bx, by, cx, cy);
  int o2 = orient(ax, ay, bx, by, dx, dy);
  int o3 = orient(cx, cy, dx, dy, ax, ay);
  int o4 = orient(cx, cy, dx, dy, bx, by);
  if (o1 * o2 < 0 && o3 * o4 < 0) return true;
  if (o1 == 0 && between(ax, ay, bx, by, cx, cy)) return true;
  if (o2 == 0 && between(ax, ay, bx, by, dx, dy)) return true;
  if (o3 == 0 && between(cx, cy, dx, dy, ax, ay)) return true;
  if (o4 == 0 && between(cx, cy, dx, dy, bx, by)) return true;
  return false;
}

bool in_box(i64 px, i64 py, i64 x0, i64 y0, i64 x1, i64 y1) {
  return x0 <= px && px <= x1 && y0 <= py && py <= y1;
}

// closed segment ab meets the closed square [x0,x1] x [y0,y1]: either an
// endpoint is inside, or the segment meets one of the four sides.
bool segment_meets_square(i64 ax, i64 ay, i64 bx, i64 by, i64 x0, i64 y0, i64 x1, i64 y1) {
  if (in_box(ax, ay, x0, y0, x1, y1) || in_box(bx, by, x0, y0, x1, y1)) return true;
  return segments_meet(ax, ay, bx, by, x0, y0, x1, y0) ||
         segments_meet(ax, ay, bx, by, x1, y0, x1, y1) ||
         segments_meet(ax, ay, bx, by, x1, y1, x0, y1) ||
         segments_meet(ax, ay, bx, by, x0, y1, x0, y0);
}

// point (px, py) in the closed polygon: on an edge, or odd crossing number of
// the rightward horizontal ray (an edge counts when one endpoint is strictly
// above py and the other is not, and the edge's x at height py exceeds px).
// The point is given in units of 1/m (m = 1 or 2: half-integer points such as
// cell centres); the ring is scaled by m on the fly.
bool inside_closed_scaled(const Ring& r, i64 px, i64 py, i64 m) {
  size_t n = r.x.size();
  for (size_t i = 0; i < n; ++i) {
    size_t k = r.nxt[i];
    if (orient(m * r.x[i], m * r.y[i], m * r.x[k], m * r.y[k], px, py) == 0 &&
        between(m * r.x[i], m * r.y[i], m * r.x[k], m * r.y[k], px, py))
      return true;
  }
  bool odd = false;
  for (size_t i = 0; i < n; ++i) {
    size_t k = r.nxt[i];
    i64 ax = m * r.x[i], ay = m * r.y[i], bx = m * r.x[k], by = m * r.y[k];
    if ((ay > py) != (by > py)) {
      // x_cross = ax + (py - ay) (bx - ax) / (by - ay)  >  px, multiplied out
      i64 num = (ax - px) * (by - ay) + (py - ay) * (bx - ax);
      bool right = (by > ay) ? (num > 0) : (num < 0);
      if (right) odd = !odd;
    }
  }
  return odd;
}

bool inside_closed(const Ring& r, i64 px, i64 py) { return inside_closed_scaled(r, px, py, 1); }

enum { EXTERIOR = 0, INTERIOR = 1, BOUNDARY = 2 };

// Sec. 2.2 classification of the closed square [x0, x0+side] x [y0, y0+side]
// against closed polygon r.
int classify(const Ring& r, i64 x0, i64 y0, i64 side) {
  i64 x1 = x0 + side, y1 = y0 + side;
  if (r.maxx < x0 || r.minx > x1 || r.maxy < y0 || r.miny > y1) return EXTERIOR;
  size_t n = r.x.size();
  for (size_t i = 0; i < n; ++i) {
    size_t k = r.nxt[i];
    if (segment_meets_square(r.x[i], r.y[i], r.x[k], r.y[k], x0, y0, x1, y1)) return BOUNDARY;
  }
  // no boundary point in the square: the whole square lies on one side, and its
  // corner is not on the boundary
  return inside_closed(r, x0, y0) ? INTERIOR : EXTERIOR;
}

// --- Sec. 2.1/2.2/3: hierarchical raster covering (O1) ------------------------
struct Rec {
  uint64_t lo, hi;  // finest-level ids [lo, hi)
  uint32_t poly;
  bool boundary;    // a boundary cell at the finest level (else an interior cell)
};

// noncons (Sec. 2.2, non-conservative raster): a finest boundary cell is kept
// only when its centre lies in the closed polygon (centres are half-integers
// when the side is 1, so the test runs in doubled coordinates).
void cover_rec(const Ring& r, uint32_t j, uint32_t B, uint32_t F, uint32_t L, uint64_t cx,
               uint64_t cy, int which, bool noncons, std::vector<Rec>& out) {
  i64 side = (i64)1 << (B - L);
  int c = classify(r, (i64)cx * side, (i64)cy * side, side);
  if (c == EXTERIOR) return;
  if (L == F && c == BOUNDARY && noncons &&
      !inside_closed_scaled(r, 2 * (i64)cx * side + side, 2 * (i64)cy * side + side, 2))
    return;
  if (c == INTERIOR || L == F) {
    // interior cell (any level) or boundary cell at the finest level: all of its
    // finest-level descendants, which by the curve's prefix property are the
    // contiguous ids [h * 4^(F-L), (h+1) * 4^(F-L))
    uint64_t h = curve(which, L, cx, cy);
    uint32_t shift = 2 * (F - L);
    out.push_back(Rec{h << shift, (h + 1) << shift, j, c == BOUNDARY});
    return;
  }
  for (uint64_t dy = 0; dy < 2; ++dy)
    for (uint64_t dx = 0; dx < 2; ++dx)
      cover_rec(r, j, B, F, L + 1, 2 * cx + dx, 2 * cy + dy, which, noncons, out);
}

struct Covering {
  uint32_t B, F, k, P;
  std::vector<uint64_t> start;     // R+1, start[0] = 0, start[R] = 4^F
  std::vector<uint32_t> list_off;  // R+1
  std::vector<uint32_t> list_ids;
  uint64_t nrec;                   // cells emitted before the sweep
};

// Sweep over all record endpoints in id order: each elementary interval gets
// the ascending set of polygons whose records contain it; a new range starts
// only where that set changes (maximal ranges, canonical form).
// flagged (Sec. 6, result range estimation): a list entry is poly | 1 << 31
// when the interval lies in a boundary cell of that polygon, and ranges split
// where the flags change as well.
Covering* build_covering(const std::vector<Ring>& rings, uint32_t B, uint32_t F, uint32_t k, int which,
                         bool flagged, bool noncons) {
  std::vector<Rec> recs;
  for (uint32_t j = 0; j < rings.size(); ++j)
    cover_rec(rings[j], j, B, F, 0, 0, 0, which, noncons, recs);
  uint64_t top = (uint64_t)1 << (2 * F);
  // position -> (poly | boundary << 31, +1 / -1)
  std::map<uint64_t, std::vector<std::pair<uint32_t, int>>> ev;
  ev[0];
  ev[top];
  for (const Rec& r : recs) {
    const uint32_t e = r.poly | ((flagged && r.boundary) ? 0x80000000u : 0u);
    ev[r.lo].push_back({e, +1});
    ev[r.hi].push_back({e, -1});
  }
  // (poly, flag) -> number of open records; one polygon's cells are disjoint,
  // so a polygon is open with at most one flag at any position
  std::map<uint32_t, int> active;
  Covering* cov = new Covering();
  cov->B = B; cov->F = F; cov->k = k; cov->P = (uint32_t)rings.size();
  cov->nrec = recs.size();
  std::vector<uint32_t> prev;
  bool have_prev = false;
  for (auto it = ev.begin(); it != ev.end(); ++it) {
    if (it->first == top) break;
    for (auto& e : it->second) {
      active[e.first] += e.second;
      if (active[e.first] == 0) active.erase(e.first);
    }
    std::vector<uint32_t> cur;  // ascending by polygon (the flag is bit 31)
    for (auto& a : active) cur.push_back(a.first);
    std::sort(cur.begin(), cur.end(),
              [](uint32_t a, uint32_t b) { return (a & 0x7fffffffu) < (b & 0x7fffffffu); });
    if (have_prev && cur == prev) continue;
    cov->start.push_back(it->first);
    cov->list_off.push_back((uint32_t)cov->list_ids.size());
    for (uint32_t p : cur) cov->list_ids.push_back(p);
    prev = cur;
    have_prev = true;
  }
  cov->start.push_back(top);
  cov->list_off.push_back((uint32_t)cov->list_ids.size());
  return cov;
}

// finest cell of a point, or false when the point is outside the grid
bool point_cell(uint32_t B, uint32_t k, uint32_t x, uint32_t y, uint64_t* cx, uint64_t* cy) {
  if (B < 32 && ((uint64_t)x >> B || (uint64_t)y >> B)) return false;
  *cx = (uint64_t)x >> k;
  *cy = (uint64_t)y >> k;
  return true;
}

template <class F>
void parallel_for(uint64_t n, int threads, F&& body) {
  if (threads <= 1 || n < 1024) {
    body(0, n, 0);
    return;
  }
  std::vector<std::thread> ts;
  uint64_t chunk = (n + threads - 1) / threads;
  for (int t = 0; t < threads; ++t) {
    uint64_t a = t * chunk, b = std::min<uint64_t>(n, a + chunk);
    if (a >= b) break;
    ts.emplace_back([&, a, b, t] { body(a, b, t); });
  }
  for (auto& t : ts) t.join();
}

// Coarse bucket grid over polygon bounding boxes, used only to skip polygons
// that cannot meet a cell (a plain prefilter; every candidate is fully tested).
struct BucketGrid {
  uint32_t nb;
  i64 bsz;
  std::vector<std::vector<uint32_t>> cells;
  BucketGrid(const std::vector<Ring>& rs, uint32_t B) {
    nb = 64;
    i64 G = (i64)1 << B;
    bsz = (G + nb - 1) / nb;
    if (bsz < 1) bsz = 1;
    cells.resize((size_t)nb * nb);
    for (uint32_t j = 0; j < rs.size(); ++j) {
      i64 bx0 = std::max<i64>(0, rs[j].minx / bsz), bx1 = std::min<i64>(nb - 1, rs[j].maxx / bsz);
      i64 by0 = std::max<i64>(0, rs[j].miny / bsz), by1 = std::min<i64>(nb - 1, rs[j].maxy / bsz);
      for (i64 by = by0; by <= by1; ++by)
        for (i64 bx = bx0; bx <= bx1; ++bx) cells[by * nb + bx].push_back(j);
    }
  }
  // candidate polygons whose bbox may meet the closed square
  void candidates(i64 x0, i64 y0, i64 x1, i64 y1, std::vector<uint32_t>& out) const {
    out.clear();
    i64 bx0 = std::max<i64>(0, x0 / bsz), bx1 = std::min<i64>(nb - 1, x1 / bsz);
    i64 by0 = std::max<i64>(0, y0 / bsz), by1 = std::min<i64>(nb - 1, y1 / bsz);
    for (i64 by = by0; by <= by1; ++by)
      for (i64 bx = bx0; bx <= bx1; ++bx)
        for (uint32_t j : cells[by * nb + bx]) out.push_back(j);
    std::sort(out.begin(), out.end());
    out.erase(std::unique(out.begin(), out.end()), out.end());
  }
};

}  // namespace

extern "C" {

int orc_finest_k(uint64_t eps, uint32_t B, uint32_t* k) { return finest_k(eps, B, k); }

void orc_curve_many(int which, uint32_t order, uint64_t n, const uint32_t* x, const uint32_t* y,
                    uint64_t* out) {
  for (uint64_t i = 0; i < n; ++i) out[i] = curve(which, order, x[i], y[i]);
}

// 0 = exterior, 1 = interior, 2 = boundary, for n closed squares of one side
// against polygon j
// poly_ring_off as for orc_cover (NULL: one ring per polygon)
void orc_classify_many(const uint32_t* poly_ring_off, const uint32_t* off, const uint32_t* vx,
                       const uint32_t* vy, uint32_t j, uint64_t n, const int64_t* x0,
                       const int64_t* y0, int64_t side, uint8_t* out) {
  Ring one;
  const uint32_t r0 = poly_ring_off ? poly_ring_off[j] : j;
  const uint32_t r1 = poly_ring_off ? poly_ring_off[j + 1] : j + 1;
  for (uint32_t r = r0; r < r1; ++r) add_ring(one, vx, vy, off[r], off[r + 1]);
  finish_ring(one);
  for (uint64_t i = 0; i < n; ++i) out[i] = (uint8_t)classify(one, x0[i], y0[i], side);
}

// mode: bit 0 boundary flags (Sec. 6), bit 1 non-conservative (Sec. 2.2).
// poly_ring_off == NULL: one ring per polygon (ring_off indexed by polygon).
void* orc_cover(uint32_t P, const uint32_t* poly_ring_off, const uint32_t* ring_off,
                const uint32_t* vx, const uint32_t* vy, uint32_t B, uint64_t eps, int which,
                int mode) {
  uint32_t k;
  if (B < 1 || B > 30 || finest_k(eps, B, &k) != 0) return nullptr;
  std::vector<Ring> rs = poly_ring_off ? load_multi(P, poly_ring_off, ring_off, vx, vy)
                                       : load_rings(P, ring_off, vx, vy);
  return build_covering(rs, B, B - k, k, which, (mode & 1) != 0, (mode & 2) != 0);
}

void orc_cover_sizes(void* h, uint64_t* R, uint64_t* nids, uint64_t* nrec, uint32_t* F, uint32_t* k) {
  Covering* c = (Covering*)h;
  *R = c->start.size() - 1;
  *nids = c->list_ids.size();
  *nrec = c->nrec;
  *F = c->F;
  *k = c->k;
}

void orc_cover_export(void* h, uint64_t* start, uint32_t* list_off, uint32_t* list_ids) {
  Covering* c = (Covering*)h;
  std::copy(c->start.begin(), c->start.end(), start);
  std::copy(c->list_off.begin(), c->list_off.end(), list_off);
  std::copy(c->list_ids.begin(), c->list_ids.end(), list_ids);
}

void orc_cover_free(void* h) { delete (Covering*)h; }

// O1 join: per point, its finest cell id, then the last range whose start is <= id
// (std::upper_bound on the sorted starts), then every polygon on that range's list.
// On a flagged covering (Sec. 6) the boundary partials are kept as well, all
// nullable: bcount[p] = counted points in boundary cells of p, bsum[p] = their
// attribute sum, babs[p] = the sum of their attributes' magnitudes.
void orc_join_o1(void* h, uint64_t n, const uint32_t* x, const uint32_t* y, const int32_t* attr,
                 uint64_t* count, int64_t* sum, uint64_t* bcount, int64_t* bsum, uint64_t* babs,
                 int which) {
  Covering* c = (Covering*)h;
  std::fill(count, count + c->P, 0);
  if (sum) std::fill(sum, sum + c->P, 0);
  if (bcount) std::fill(bcount, bcount + c->P, 0);
  if (bsum) std::fill(bsum, bsum + c->P, 0);
  if (babs) std::fill(babs, babs + c->P, 0);
  for (uint64_t i = 0; i < n; ++i) {
    uint64_t cx, cy;
    if (!point_cell(c->B, c->k, x[i], y[i], &cx, &cy)) continue;
    uint64_t id = curve(which, c->F, cx, cy);
    size_t r = (size_t)(std::upper_bound(c->start.begin(), c->start.end(), id) - c->start.begin()) - 1;
    const int64_t a = attr ? attr[i] : 0;
    for (uint32_t e = c->list_off[r]; e < c->list_off[r + 1]; ++e) {
      const uint32_t p = c->list_ids[e] & 0x7fffffffu;
      const bool boundary = (c->list_ids[e] >> 31) != 0;
      count[p] += 1;
      if (sum) sum[p] += a;
      if (boundary) {
        if (bcount) bcount[p] += 1;
        if (bsum) bsum[p] += a;
        if (babs) babs[p] += (uint64_t)(a < 0 ? -a : a);
      }
    }
  }
}

// O2 join, straight from the definition: point p counts for polygon j iff the
// closed finest cell of p meets closed polygon j.  No covering, no curve.
// bnd_count (nullable): per polygon, the counted points whose cell meets the
// polygon's boundary (Sec. 6, result range: exact count lies in
// [count - bnd_count, count] for a conservative raster); bnd_sum / bnd_abs
// (nullable): those points' attribute sum and sum of magnitudes.
// member (nullable, n bytes): per point, 1 if it counts for polygon `only`
// (only >= 0) or for any polygon (only < 0).
// mode bit 1: non-conservative (a boundary cell counts only when its centre
// lies in the closed polygon).  poly_ring_off as for orc_cover.
int orc_join_o2(uint32_t P, const uint32_t* poly_ring_off, const uint32_t* off, const uint32_t* vx,
                const uint32_t* vy, uint32_t B, uint64_t eps, uint64_t n, const uint32_t* x,
                const uint32_t* y, const int32_t* attr, uint64_t* count, int64_t* sum,
                uint64_t* bnd_count, int64_t* bnd_sum, uint64_t* bnd_abs, uint8_t* member,
                int64_t only, int threads, int mode) {
  uint32_t k;
  if (B < 1 || B > 30 || finest_k(eps, B, &k) != 0) return -1;
  std::vector<Ring> rs = poly_ring_off ? load_multi(P, poly_ring_off, off, vx, vy)
                                       : load_rings(P, off, vx, vy);
  const bool noncons = (mode & 2) != 0;
  BucketGrid bg(rs, B);
  i64 s = (i64)1 << k;
  if (threads < 1) threads = 1;
  std::vector<std::vector<uint64_t>> tc(threads, std::vector<uint64_t>(P, 0));
  std::vector<std::vector<int64_t>> ts(threads, std::vector<int64_t>(P, 0));
  std::vector<std::vector<uint64_t>> tb(threads, std::vector<uint64_t>(P, 0));
  std::vector<std::vector<int64_t>> tbs(threads, std::vector<int64_t>(P, 0));
  std::vector<std::vector<uint64_t>> tba(threads, std::vector<uint64_t>(P, 0));
  parallel_for(n, threads, [&](uint64_t a, uint64_t b, int t) {
    std::vector<uint32_t> cand;
    for (uint64_t i = a; i < b; ++i) {
      uint64_t cx, cy;
      bool hit = false;
      if (point_cell(B, k, x[i], y[i], &cx, &cy)) {
        i64 x0 = (i64)cx * s, y0 = (i64)cy * s;
        bg.candidates(x0, y0, x0 + s, y0 + s, cand);
        for (uint32_t j : cand) {
          int c = classify(rs[j], x0, y0, s);
          if (c == EXTERIOR) continue;
          if (c == BOUNDARY && noncons && !inside_closed_scaled(rs[j], 2 * x0 + s, 2 * y0 + s, 2))
            continue;
          const int64_t av = attr ? attr[i] : 0;
          tc[t][j] += 1;
          ts[t][j] += av;
          if (c == BOUNDARY) {
            tb[t][j] += 1;
            tbs[t][j] += av;
            tba[t][j] += (uint64_t)(av < 0 ? -av : av);
          }
          if (only < 0 || (int64_t)j == only) hit = true;
        }
      }
      if (member) member[i] = hit;
    }
  });
  for (uint32_t j = 0; j < P; ++j) {
    count[j] = 0;
    if (sum) sum[j] = 0;
    if (bnd_count) bnd_count[j] = 0;
    if (bnd_sum) bnd_sum[j] = 0;
    if (bnd_abs) bnd_abs[j] = 0;
    for (int t = 0; t < threads; ++t) {
      count[j] += tc[t][j];
      if (sum) sum[j] += ts[t][j];
      if (bnd_count) bnd_count[j] += tb[t][j];
      if (bnd_sum) bnd_sum[j] += tbs[t][j];
      if (bnd_abs) bnd_abs[j] += tba[t][j];
    }
  }
  return 0;
}

// Point-indexed aggregation (Sec. 3, "Point Indexing"): the points' cells are
// linearised by the same curve at full resolution (level B, so a finest-level
// id h at level F covers the full-resolution ids [h << 2k, (h + 1) << 2k)),
// stored as a sorted array with prefix sums of the attribute; per covering
// range [start_r, start_r+1) the qualifying points are
// [lower_bound(start_r << 2k), lower_bound(start_r+1 << 2k)), their COUNT the
// difference of the two positions and their SUM the difference of the prefix
// sums, added to every polygon on the range's list.  Plain std::sort and
// std::lower_bound.
void orc_point_index_aggregate(void* h, uint64_t n, const uint32_t* x, const uint32_t* y,
                               const int32_t* attr, uint64_t* count, int64_t* sum, int which) {
  Covering* c = (Covering*)h;
  std::vector<std::pair<uint64_t, int64_t>> kv;
  kv.reserve(n);
  for (uint64_t i = 0; i < n; ++i) {
    uint64_t cx, cy;
    if (!point_cell(c->B, 0, x[i], y[i], &cx, &cy)) continue;
    kv.push_back({curve(which, c->B, cx, cy), attr ? (int64_t)attr[i] : 0});
  }
  std::sort(kv.begin(), kv.end());
  std::vector<uint64_t> keys(kv.size());
  std::vector<int64_t> prefix(kv.size() + 1, 0);
  for (size_t i = 0; i < kv.size(); ++i) {
    keys[i] = kv[i].first;
    prefix[i + 1] = prefix[i] + kv[i].second;
  }
  std::fill(count, count + c->P, 0);
  if (sum) std::fill(sum, sum + c->P, 0);
  const uint32_t sh = 2 * c->k;
  for (size_t r = 0; r + 1 < c->start.size(); ++r) {
    if (c->list_off[r] == c->list_off[r + 1]) continue;
    const size_t a = std::lower_bound(keys.begin(), keys.end(), c->start[r] << sh) - keys.begin();
    const size_t b = std::lower_bound(keys.begin(), keys.end(), c->start[r + 1] << sh) - keys.begin();
    for (uint32_t e = c->list_off[r]; e < c->list_off[r + 1]; ++e) {
      const uint32_t p = c->list_ids[e] & 0x7fffffffu;
      count[p] += b - a;
      if (sum) sum[p] += prefix[b] - prefix[a];
    }
  }
}

// exact closed point-in-polygon join (the answer the approximation bounds)
void orc_join_exact(uint32_t P, const uint32_t* poly_ring_off, const uint32_t* off,
                    const uint32_t* vx, const uint32_t* vy, uint32_t B, uint64_t n,
                    const uint32_t* x, const uint32_t* y, const int32_t* attr, uint64_t* count,
                    int64_t* sum, uint8_t* member, int64_t only, int threads) {
  std::vector<Ring> rs = poly_ring_off ? load_multi(P, poly_ring_off, off, vx, vy)
                                       : load_rings(P, off, vx, vy);
  BucketGrid bg(rs, B);
  if (threads < 1) threads = 1;
  std::vector<std::vector<uint64_t>> tc(threads, std::vector<uint64_t>(P, 0));
  std::vector<std::vector<int64_t>> ts(threads, std::vector<int64_t>(P, 0));
  parallel_for(n, threads, [&](uint64_t a, uint64_t b, int t) {
    std::vector<uint32_t> cand;
    for (uint64_t i = a; i < b; ++i) {
      bool hit = false;
      bg.candidates(x[i], y[i], x[i], y[i], cand);
      for (uint32_t j : cand) {
        const Ring& r = rs[j];
        if (x[i] < r.minx || x[i] > r.maxx || y[i] < r.miny || y[i] > r.maxy) continue;
        if (!inside_closed(r, x[i], y[i])) continue;
        tc[t][j] += 1;
        ts[t][j] += attr ? attr[i] : 0;
        if (only < 0 || (int64_t)j == only) hit = true;
      }
      if (member) member[i] = hit;
    }
  });
  for (uint32_t j = 0; j < P; ++j) {
    count[j] = 0;
    if (sum) sum[j] = 0;
    for (int t = 0; t < threads; ++t) {
      count[j] += tc[t][j];
      if (sum) sum[j] += ts[t][j];
    }
  }
}

// Sec. 2.2 distance bound: is the point within distance eps of polygon j's
// boundary?  Exact: squared distances compared in 128-bit integers.
int orc_near_boundary(const uint32_t* poly_ring_off, const uint32_t* off, const uint32_t* vx,
                      const uint32_t* vy, uint32_t j, uint32_t px, uint32_t py, uint64_t eps) {
  i128 e2 = (i128)eps * (i128)eps;
  // rings of polygon j (one ring when poly_ring_off is NULL)
  const uint32_t r0 = poly_ring_off ? poly_ring_off[j] : j;
  const uint32_t r1 = poly_ring_off ? poly_ring_off[j + 1] : j + 1;
  for (uint32_t rr = r0; rr < r1; ++rr)
  for (uint32_t v = off[rr]; v < off[rr + 1]; ++v) {
    uint32_t w = (v + 1 < off[rr + 1]) ? v + 1 : off[rr];
    i64 ax = vx[v], ay = vy[v], bx = vx[w], by = vy[w];
    i64 dx = bx - ax, dy = by - ay;
    i64 qx = (i64)px - ax, qy = (i64)py - ay;
    i128 t = (i128)qx * dx + (i128)qy * dy;
    i128 len2 = (i128)dx * dx + (i128)dy * dy;
    i128 d2num, d2den;
    if (t <= 0 || len2 == 0) {
      d2num = (i128)qx * qx + (i128)qy * qy;
      d2den = 1;
    } else if (t >= len2) {
      i64 rx = (i64)px - bx, ry = (i64)py - by;
      d2num = (i128)rx * rx + (i128)ry * ry;
      d2den = 1;
    } else {
      i128 cr = (i128)dx * qy - (i128)dy * qx;
      d2num = cr * cr;
      d2den = len2;
    }
    if (d2num <= e2 * d2den) return 1;
  }
  return 0;
}

}  // extern "C"
