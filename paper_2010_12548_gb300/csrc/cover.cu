// Covering builder: the conservative hierarchical raster of Sec. 2.1-2.2,
// linearised by the Hilbert curve and merged into disjoint id ranges (Sec. 3,
// "Polygon Indexing").
//
// Level-synchronous quadtree refinement on the device.  A frontier item is a
// cell of some polygon that meets the polygon's boundary, together with the
// list of the polygon's edges that meet the (closed) cell, and one parity bit:
// whether the point c+ = c + (d, d^2) (c the cell's lower-left corner, d an
// infinitesimal) lies inside the polygon.  Expanding an item tests its four
// children against the item's edges only (an edge meeting a child meets its
// parent):
//   * a child that meets an edge is a boundary cell: emitted at the finest level
//     F, otherwise pushed to the next frontier with its own edge list;
//   * a child that meets no edge lies wholly inside or wholly outside; its
//     corner's parity decides, and is derived from the parent's parity by
//     counting the parent's edges that cross the segment from the parent's
//     corner to the child's corner (both shifted by (d, d^2)).
// The shift makes every test point and test segment avoid every vertex and
// edge line symbolically, so all predicates are exact integer sign tests
// (coordinates < 2^30, products < 2^61, int64).  The root parity comes from a
// rightward ray from (0,0)+.
//
// Emitted cells become (lo = h * 4^(F-L), level) records; a sweep over all
// record endpoints (sort, unique, per-interval polygon lists, merge of equal
// neighbours) gives the canonical ranges.
#include "sdb_internal.cuh"

#include <algorithm>
#include <atomic>
#include <mutex>
#include <utility>
#include <vector>

namespace sdb {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr uint32_t NONE = 0xffffffffu;
// A record's value: slot (bits 0..25), level above the finest (26..30), and
// bit 31 set for a boundary cell of a flagged covering (Sec. 6).
constexpr uint32_t VAL_SLOT = (1u << 26) - 1u;
constexpr uint32_t VAL_FLAG = 0x80000000u;
__device__ __forceinline__ uint32_t val_level(uint32_t v) { return (v >> 26) & 31u; }
// list entry / single-polygon payload of a slot with its boundary flag
__device__ __forceinline__ uint32_t list_entry(uint32_t v) { return v & (VAL_SLOT | VAL_FLAG); }
__device__ __forceinline__ uint32_t single_pay(uint32_t v) {
  return (v & VAL_SLOT) | ((v >> 31) << 30);
}

// Records are (key, value) pairs in two arrays, or, when the key and a short
// value fit one 64-bit word, packed: key << (sb + 6) | flag << (sb + 5) |
// level << sb | slot with sb slot bits (sb = 0: not packed).  The sort then
// moves 8 bytes per record instead of 12.
__device__ __forceinline__ void put_record(uint64_t* __restrict__ rk, uint32_t* __restrict__ rv,
                                           uint64_t r, uint64_t key, uint32_t val, uint32_t sb) {
  if (sb) {
    rk[r] = record_pack(key, val, sb);
  } else {
    rk[r] = key;
    rv[r] = val;
  }
}

struct Edge {
  int32_t ax, ay, bx, by;
};

// A frontier cell of one (query, polygon) pair at level L: cell (cx, cy), its
// Hilbert id at level L and the curve's orientation (sw << 1 | cm) below it,
// so a child's id is one more digit; its edge list elist[eoff, eoff + ecnt)
// and the perturbed parity of its lower-left corner.
struct __align__(16) Item {
  uint64_t hid;
  uint32_t pair, cx, cy, eoff;
  uint32_t ecnt_par;  // edge count | parity << 31
  uint32_t orient;
};
static_assert(sizeof(Item) == 32, "two 16-byte loads per item");

__device__ __forceinline__ uint64_t qof(uint64_t key, uint32_t qshift) {
  return qshift >= 64 ? 0ull : key >> qshift;
}

// Sign of cross(b - a, q+ - a) with q+ = q + (d, d^2): o - dy*d + dx*d^2.
// Never zero for a non-degenerate edge.
__device__ __forceinline__ int pert_side(const Edge& e, int64_t qx, int64_t qy) {
  int64_t dx = (int64_t)e.bx - e.ax, dy = (int64_t)e.by - e.ay;
  int64_t o = dx * (qy - e.ay) - dy * (qx - e.ax);
  if (o != 0) return o > 0 ? 1 : -1;
  if (dy != 0) return dy < 0 ? 1 : -1;
  return dx > 0 ? 1 : -1;
}

// Does edge e cross the rightward ray from q+ ?  (integer endpoints lie above
// the line y = qy + d^2 iff y > qy)
__device__ __forceinline__ uint32_t pert_ray_cross(const Edge& e, int64_t qx, int64_t qy) {
  bool ua = e.ay > qy, ub = e.by > qy;
  if (ua == ub) return 0;
  int sd = pert_side(e, qx, qy);
  return (e.by > e.ay) ? (sd > 0) : (sd < 0);
}

// Offsets for three per-thread counts, with one atomic per counter and block
// (blockDim.x == 256): warp scans, then warp prefixes in shared memory.  Every
// thread of the block must call it.
__device__ __forceinline__ void block_alloc3(const uint32_t (&n)[3],
                                             unsigned long long* __restrict__ ctr,
                                             unsigned long long (&off)[3]) {
  __shared__ uint32_t wsum[3][8];
  __shared__ unsigned long long base[3];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t inc[3] = {n[0], n[1], n[2]};
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const uint32_t t = __shfl_up_sync(FULL, inc[j], o);
      if (lane >= o) inc[j] += t;
    }
  }
  if (lane == 31) {
#pragma unroll
    for (int j = 0; j < 3; ++j) wsum[j][w] = inc[j];
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    const int j = threadIdx.x;
    uint32_t t = 0;
    for (int k = 0; k < 8; ++k) {
      const uint32_t v = wsum[j][k];
      wsum[j][k] = t;
      t += v;
    }
    base[j] = t ? atomicAdd(&ctr[j], (unsigned long long)t) : 0ull;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < 3; ++j) off[j] = base[j] + wsum[j][w] + inc[j] - n[j];
}

__global__ void build_edges_kernel(const uint32_t* __restrict__ vx, const uint32_t* __restrict__ vy,
                                   const uint32_t* __restrict__ next, uint32_t V,
                                   Edge* __restrict__ edges, uint32_t* __restrict__ elist) {
  uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  const uint32_t w = next[v];  // the following vertex of v's ring
  edges[v] = Edge{(int32_t)vx[v], (int32_t)vy[v], (int32_t)vx[w], (int32_t)vy[w]};
  elist[v] = v;
}

// Non-conservative raster (Sec. 2.2): centre tests in doubled coordinates
// (centres of unit cells are then integers; perturbation as for the corners).
// Perturbed side of (x, y)+ against edge (a, b): sign of cross(b - a, q - a),
// ties by -dy, then dx.
__device__ __forceinline__ int dbl_side(int64_t ax, int64_t ay, int64_t dx, int64_t dy, int64_t x,
                                        int64_t y) {
  const int64_t o = dx * (y - ay) - dy * (x - ax);
  if (o != 0) return o > 0 ? 1 : -1;
  if (dy != 0) return dy < 0 ? 1 : -1;
  return dx > 0 ? 1 : -1;
}
// the rightward ray from (x, y)+ crosses the edge
__device__ __forceinline__ uint32_t dbl_ray_right(int64_t ax, int64_t ay, int64_t bx, int64_t by,
                                                  int64_t x, int64_t y) {
  if ((ay > y) == (by > y)) return 0;
  const int sd = dbl_side(ax, ay, bx - ax, by - ay, x, y);
  return (by > ay) ? (sd > 0) : (sd < 0);
}
// the upward ray from (x, y)+ crosses the edge
__device__ __forceinline__ uint32_t dbl_ray_up(int64_t ax, int64_t ay, int64_t bx, int64_t by,
                                               int64_t x, int64_t y) {
  if ((ax > x) == (bx > x)) return 0;
  const int sd = dbl_side(ax, ay, bx - ax, by - ay, x, y);
  return (bx > ax) ? (sd < 0) : (sd > 0);
}
__device__ __forceinline__ uint32_t dbl_on_edge(int64_t ax, int64_t ay, int64_t bx, int64_t by,
                                                int64_t x, int64_t y) {
  const int64_t o = (bx - ax) * (y - ay) - (by - ay) * (x - ax);
  return o == 0 && min(ax, bx) <= x && x <= max(ax, bx) && min(ay, by) <= y && y <= max(ay, by);
}

// One edge against the centres of the 2x2 children of the parent with corner
// (px, py) and child side `side`: bits 0..3 the parity flip from the parent's
// corner+ to child c's centre+ along the path right to the centre's x, then up
// (segment parities as XORs of rays); bits 4..7 the centre lies on the edge.
__device__ __forceinline__ uint32_t edge_vs_centres(const Edge& e, int64_t px, int64_t py,
                                                    int64_t side) {
  const int64_t ax = 2 * (int64_t)e.ax, ay = 2 * (int64_t)e.ay;
  const int64_t bx = 2 * (int64_t)e.bx, by = 2 * (int64_t)e.by;
  const int64_t X0 = 2 * px, Y0 = 2 * py;
  const uint32_t r0 = dbl_ray_right(ax, ay, bx, by, X0, Y0);
  uint32_t out = 0;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int64_t cx = X0 + (2 * (c & 1) + 1) * side, cy = Y0 + (2 * (c >> 1) + 1) * side;
    const uint32_t f = r0 ^ dbl_ray_right(ax, ay, bx, by, cx, Y0) ^
                       dbl_ray_up(ax, ay, bx, by, cx, Y0) ^ dbl_ray_up(ax, ay, bx, by, cx, cy);
    out |= (f << c) | (dbl_on_edge(ax, ay, bx, by, cx, cy) << (4 + c));
  }
  return out;
}

// one warp per (query, polygon) pair: the level-0 item (whole grid) with all of
// the polygon's edges and the parity of (0,0)+; a query whose finest level is 0
// gets the whole grid as one boundary cell instead
__global__ void root_items_kernel(const uint32_t* __restrict__ edge_off,
                                  const Edge* __restrict__ edges,
                                  const uint32_t* __restrict__ pair_poly,
                                  const uint32_t* __restrict__ pair_query,
                                  const uint32_t* __restrict__ pair_slot,
                                  const CoverQuery* __restrict__ qs, uint32_t NP, uint32_t qshift,
                                  uint32_t bflag, bool noncons, uint32_t B, Item* __restrict__ items,
                                  uint64_t* __restrict__ rec_key, uint32_t* __restrict__ rec_val,
                                  uint32_t sb, unsigned long long* __restrict__ counters) {
  uint32_t p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (p >= NP) return;
  const uint32_t j = pair_poly[p], qi = pair_query[p];
  if (qs[qi].F == 0) {
    if (noncons) {  // the whole grid is kept only when its centre is in the polygon
      const int64_t c = (int64_t)1 << B;  // the centre, doubled
      uint32_t par = 0, on = 0;
      for (uint32_t v = edge_off[j] + lane; v < edge_off[j + 1]; v += 32) {
        const Edge e = edges[v];
        const int64_t ax = 2 * (int64_t)e.ax, ay = 2 * (int64_t)e.ay;
        const int64_t bx = 2 * (int64_t)e.bx, by = 2 * (int64_t)e.by;
        par ^= dbl_ray_right(ax, ay, bx, by, c, c);
        on |= dbl_on_edge(ax, ay, bx, by, c, c);
      }
      const bool keep = __any_sync(FULL, on) || (__popc(__ballot_sync(FULL, par)) & 1u);
      if (!keep) return;
    }
    if (lane == 0) {
      unsigned long long r = atomicAdd(&counters[2], 1ull);
      // the whole grid as one boundary cell
      put_record(rec_key, rec_val, r, qshift >= 64 ? 0ull : ((uint64_t)qi << qshift),
                 pair_slot[p] | bflag, sb);
    }
    return;
  }
  uint32_t a = edge_off[j], b = edge_off[j + 1];
  uint32_t par = 0;
  for (uint32_t v = a + lane; v < b; v += 32) par ^= pert_ray_cross(edges[v], 0, 0);
  par = __popc(__ballot_sync(FULL, par)) & 1u;
  if (lane == 0) {
    unsigned long long i = atomicAdd(&counters[0], 1ull);
    items[i] = Item{0ull, p, 0, 0, a, (b - a) | (par << 31), 0u};
  }
}

// One edge against the 2x2 children of a parent square with lower-left corner
// (px, py) and child side 2^sh (grid bits <= 30, so corners and edge ends fit
// in int32 and the line function below in int64).  The line function
// f(p) = cross(b - a, p - a) is linear, so its values on the 3x3 lattice of
// child corners follow from one evaluation and shifted steps:
// f(px + u*side, py + v*side) = f00 + u*stepx + v*stepy.  Only their strict
// signs are kept, as 9-bit masks (bit u + 3v).
// Bits 0..3 of the result: the closed edge meets closed child c
// (c = dy*2 + dx); separating axes: the bounding boxes, and the edge's line
// (f is not of one strict sign over the child's four corners).
// Bits 5..7: parity flips from the parent's corner to the corner of child 1
// (rightward ray along the bottom row), child 2 (upward ray along the left
// column) and child 3 (child 1's corner plus the upward ray along the middle
// column), all for corners shifted by (d, d^2).  A ray from q+ crosses the
// edge iff the edge straddles the ray's line and the perturbed sign of f at
// q+ has the side that faces the edge, so the crossing parity of the segment
// between two lattice points is the XOR of their perturbed signs, taken when
// the edge straddles the segment's line.
__device__ __forceinline__ uint32_t edge_vs_children(const Edge& e, int32_t px, int32_t py,
                                                     uint32_t sh) {
  const int32_t side = 1 << sh;
  const int64_t dx = (int64_t)e.bx - e.ax, dy = (int64_t)e.by - e.ay;  // (edge direction)
  const int64_t f00 = dx * ((int64_t)py - e.ay) - dy * ((int64_t)px - e.ax);
  const int64_t stepx = -(dy << sh), stepy = dx << sh;
  uint32_t pos = 0, neg = 0;
  int64_t row = f00;
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    int64_t f = row;
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      pos |= (uint32_t)(f > 0) << (u + 3 * v);
      neg |= (uint32_t)(f < 0) << (u + 3 * v);
      f += stepx;
    }
    row += stepy;
  }
  const int32_t minx = min(e.ax, e.bx), maxx = max(e.ax, e.bx);
  const int32_t miny = min(e.ay, e.by), maxy = max(e.ay, e.by);
  uint32_t out = 0;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int cu = c & 1, cv = c >> 1;
    const int32_t x0 = px + cu * side, y0 = py + cv * side;
    const bool box = !(maxx < x0 || minx - side > x0 || maxy < y0 || miny - side > y0);
    const uint32_t corners = 0x1bu << (cu + 3 * cv);  // (u,v), (u+1,v), (u,v+1), (u+1,v+1)
    out |= (uint32_t)(box && (corners & ~pos) && (corners & ~neg)) << c;
  }
  if (dx == 0 && dy == 0) return out;
  // perturbed sign at lattice point (u, v): that of f, else of -dy, else of dx
  const bool tie_pos = dy != 0 ? dy < 0 : dx > 0;
  const uint32_t ppos = pos | (tie_pos ? (~(pos | neg) & 0x1ffu) : 0u);
  const uint32_t p00 = ppos & 1u, p10 = (ppos >> 1) & 1u, p01 = (ppos >> 3) & 1u,
                 p11 = (ppos >> 4) & 1u;
  // rightward ray along y = py + d^2; upward rays along x = px + d, px + side + d
  const uint32_t flip1 = ((e.ay > py) != (e.by > py)) ? (p00 ^ p10) : 0u;
  const uint32_t flip2 = ((e.ax > px) != (e.bx > px)) ? (p00 ^ p01) : 0u;
  const uint32_t flipm = ((e.ax > px + side) != (e.bx > px + side)) ? (p10 ^ p11) : 0u;
  return out | (flip1 << 5) | (flip2 << 6) | ((flip1 ^ flipm) << 7);
}

// One level of the refinement: each frontier item (a boundary cell of one
// pair) is split into its 4 children.  G lanes share an item (G a power of two
// up to 32, chosen from the level's mean edge count): each lane tests every
// G-th edge, the group combines meet counts and parity flips with shuffles, and
// its first lane writes the records and child items.  Child edge lists keep
// the parent's edge order (a ballot per child and chunk of G edges); the meet
// masks of the first 8 chunks are kept in a register for that second pass.
template <int G, bool NC>
__global__ __launch_bounds__(256) void expand_level_kernel(
    const Item* __restrict__ items, uint32_t n_items, const uint32_t* __restrict__ elist,
    const Edge* __restrict__ edges, const uint32_t* __restrict__ pair_query,
    const uint32_t* __restrict__ pair_slot, const CoverQuery* __restrict__ qs, uint32_t qshift,
    uint32_t bflag, uint32_t B, uint32_t L, Item* __restrict__ next_items,
    uint32_t* __restrict__ next_elist,
    uint64_t* __restrict__ rec_key, uint32_t* __restrict__ rec_val, uint32_t sb,
    unsigned long long rec_base, unsigned long long* __restrict__ counters) {
  const uint64_t gt = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = gt / G < n_items;
  const uint32_t t = (uint32_t)(gt / G);  // item of this lane's group
  const uint32_t gl = (uint32_t)(gt % G); // lane within the group
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t gmask = G == 32 ? FULL : (((1u << G) - 1u) << (lane & ~(uint32_t)(G - 1)));
  Item it{0ull, 0, 0, 0, 0, 0, 0};
  if (active) it = items[t];
  const uint32_t qi = active ? pair_query[it.pair] : 0u;
  CoverQuery Q{0, 0, 0, 0, 0};
  if (active) Q = qs[qi];
  const uint32_t F = Q.F;
  const uint32_t cl = L + 1;
  const uint32_t sh = B - cl;
  const int64_t side = (int64_t)1 << sh;
  const int64_t px = (int64_t)it.cx << (B - L), py = (int64_t)it.cy << (B - L);
  const int32_t px32 = (int32_t)px, py32 = (int32_t)py;  // < 2^30
  // children holding lattice points of the query's box [x0, x1) x [y0, y1)
  uint32_t keep = 0;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int64_t x0 = px + (c & 1) * side, y0 = py + (c >> 1) * side;
    keep |= (uint32_t)(x0 < (int64_t)Q.x1 && x0 + side > (int64_t)Q.x0 && y0 < (int64_t)Q.y1 &&
                       y0 + side > (int64_t)Q.y0)
            << c;
  }
  const uint32_t ecnt = it.ecnt_par & 0x7fffffffu;
  const uint32_t par = it.ecnt_par >> 31;
  // children c = dy*2 + dx, lower-left corner (px + dx*side, py + dy*side)
  uint32_t cnt[4] = {0, 0, 0, 0};
  uint32_t flip = 0;   // bit c: parity flip from the parent's corner to child c's
  uint32_t mcache = 0; // meet bits of this lane's edges in chunks 0..7
  // non-conservative, last level: bits 0..3 parity flips to the children's
  // centres, bits 4..7 a centre lies on an edge
  const bool nc = NC && cl == F;
  uint32_t cen = 0;
  for (uint32_t i = gl, j = 0; i < ecnt; i += G, ++j) {
    const Edge e = edges[elist[it.eoff + i]];
    const uint32_t m = edge_vs_children(e, px32, py32, sh);
#pragma unroll
    for (int c = 0; c < 4; ++c) cnt[c] += (m >> c) & 1u;
    flip ^= m >> 4;
    if (j < 8) mcache |= (m & 15u) << (4 * j);
    if (nc) {
      const uint32_t b = edge_vs_centres(e, px, py, side);
      cen = (cen ^ (b & 15u)) | (b & 0xf0u);
    }
  }
  if (G > 1) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
#pragma unroll
      for (int c = 0; c < 4; ++c) cnt[c] += __shfl_xor_sync(gmask, cnt[c], o);
      flip ^= __shfl_xor_sync(gmask, flip, o);
      const uint32_t oc = __shfl_xor_sync(gmask, cen, o);
      cen = ((cen ^ oc) & 15u) | ((cen | oc) & 0xf0u);
    }
  }
  // boundary children kept at the last level: all, or (non-conservative) those
  // whose centre is on an edge or inside (the corner's parity plus the flip)
  const uint32_t bkeep = nc ? (((cen >> 4) | ((par ? 15u : 0u) ^ (cen & 15u))) & 15u) : 15u;
  uint32_t n_rec = 0, n_it = 0, n_ed = 0;
  if (active && gl == 0) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      uint32_t inside = (par ^ (flip >> c)) & 1u;
      if (!((keep >> c) & 1u)) continue;
      if (cnt[c] > 0) {
        if (cl == F) {
          n_rec += (bkeep >> c) & 1u;
        } else {
          ++n_it;
          n_ed += cnt[c];
        }
      } else if (inside) {
        ++n_rec;
      }
    }
  }
  // counters: 0 child items, 1 child edge entries, 2 records
  unsigned long long off[3];
  block_alloc3({n_it, n_ed, n_rec}, counters, off);
  unsigned long long io = off[0], eo = off[1], ro = off[2];
  if (!active) return;
  const uint32_t leader = lane & ~(uint32_t)(G - 1);
  if (G > 1) {
    n_it = __shfl_sync(gmask, n_it, leader);
    eo = __shfl_sync(gmask, eo, leader);
  }
  uint32_t ceoff[4] = {0, 0, 0, 0};
  const uint32_t shift = 2 * (F - cl);
  const uint64_t qbits = qshift >= 64 ? 0ull : ((uint64_t)qi << qshift);
  const uint32_t slot = pair_slot[it.pair];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    if (!((keep >> c) & 1u)) {
      cnt[c] = 0;  // dropped: no record, no child item, no edge list
      continue;
    }
    const uint32_t ccx = 2 * it.cx + (c & 1), ccy = 2 * it.cy + (c >> 1);
    // child's digit and orientation under the parent's orientation (sw, cm)
    const uint32_t sw = it.orient >> 1, cm = it.orient & 1u;
    const uint32_t xt = (sw ? (uint32_t)(c >> 1) : (uint32_t)(c & 1)) ^ cm;
    const uint32_t yt = (sw ? (uint32_t)(c & 1) : (uint32_t)(c >> 1)) ^ cm;
    const uint64_t chid = (it.hid << 2) | ((xt << 1) | (xt ^ yt));
    const uint32_t corient = yt ? it.orient : (it.orient ^ 2u ^ xt);
    uint32_t inside = (par ^ (flip >> c)) & 1u;
    if (cnt[c] > 0 && cl == F && !((bkeep >> c) & 1u)) {
      cnt[c] = 0;  // non-conservative: a boundary cell whose centre lies outside
      continue;
    }
    bool emit = (cnt[c] > 0) ? (cl == F) : (inside != 0);
    if (emit) {
      if (gl == 0) {
        put_record(rec_key, rec_val, rec_base + ro++, qbits | (chid << shift),
                   slot | ((F - cl) << 26) | (cnt[c] > 0 ? bflag : 0u), sb);
      }
      cnt[c] = 0;  // a finest boundary cell needs no edge list
    } else if (cnt[c] > 0) {
      ceoff[c] = (uint32_t)eo;
      if (gl == 0)
        next_items[io++] =
            Item{chid, it.pair, ccx, ccy, (uint32_t)eo, cnt[c] | (inside << 31), corient};
      eo += cnt[c];
    }
  }
  if (n_it) {
    uint32_t fill[4] = {0, 0, 0, 0};
    const uint32_t below = (1u << (lane - leader)) - 1u;
    for (uint32_t base = 0, j = 0; base < ecnt; base += G, ++j) {
      const uint32_t i = base + gl;
      uint32_t m = 0, eid = 0;
      if (i < ecnt) {
        eid = elist[it.eoff + i];
        m = j < 8 ? (mcache >> (4 * j)) & 15u : edge_vs_children(edges[eid], px32, py32, sh) & 15u;
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (cnt[c] == 0) continue;
        const bool hit = (m >> c) & 1u;
        const uint32_t bal = G > 1 ? ((__ballot_sync(gmask, hit) & gmask) >> leader) : (uint32_t)hit;
        if (hit) next_elist[ceoff[c] + fill[c] + __popc(bal & below)] = eid;
        fill[c] += __popc(bal);
      }
    }
  }
}

// ------------------------------------------------------------ range merge
__device__ __forceinline__ uint32_t lower_bound_u64(const uint64_t* __restrict__ b, uint32_t m,
                                                    uint64_t v) {
  uint32_t lo = 0, len = m;
  while (len > 0) {
    uint32_t half = len >> 1;
    if (b[lo + half] < v) {
      lo += half + 1;
      len -= half + 1;
    } else {
      len = half;
    }
  }
  return lo;
}

__global__ void breakpoints_kernel(const uint64_t* __restrict__ key, const uint32_t* __restrict__ val,
                                   uint64_t n, uint64_t top, uint64_t* __restrict__ bp) {
  uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) {
    uint32_t d = val_level(val[r]);
    bp[2 * r] = key[r];
    bp[2 * r + 1] = key[r] + (1ull << (2 * d));
  } else if (r == n) {
    bp[2 * n] = 0;
    bp[2 * n + 1] = top;
  }
}

__global__ void spans_kernel(const uint64_t* __restrict__ key, const uint32_t* __restrict__ val,
                             uint64_t n, const uint64_t* __restrict__ b, uint32_t m,
                             uint32_t* __restrict__ klo, uint32_t* __restrict__ span) {
  uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  uint32_t d = val_level(val[r]);
  uint64_t lo = key[r], hi = lo + (1ull << (2 * d));
  uint32_t a = lower_bound_u64(b, m, lo), c = lower_bound_u64(b, m, hi);
  klo[r] = a;
  span[r] = c - a;
}

// pair i belongs to the record r with poff[r] <= i < poff[r+1]
__global__ void expand_pairs_kernel(const uint64_t* __restrict__ poff, uint64_t n,
                                    const uint32_t* __restrict__ klo,
                                    const uint32_t* __restrict__ val, uint64_t T, uint32_t pbits,
                                    uint32_t fl, uint64_t* __restrict__ pairs) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= T) return;
  // last r with poff[r] <= i
  uint64_t lo = 0, len = n;
  while (len > 1) {
    uint64_t half = len >> 1;
    if (poff[lo + half] <= i) lo += half;
    len -= half;
  }
  // the pair's polygon field: slot, then its boundary flag when flagged (fl = 1)
  const uint32_t v = val[lo];
  const uint32_t poly = fl ? (((v & VAL_SLOT) << 1) | (v >> 31)) : (v & VAL_SLOT);
  uint64_t k = (uint64_t)klo[lo] + (i - poff[lo]);
  pairs[i] = (k << pbits) | poly;
}

__global__ void widen_kernel(const uint32_t* __restrict__ in, uint64_t n, uint64_t* __restrict__ out) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = in[i];
}

__global__ void count_len_kernel(const uint64_t* __restrict__ pairs, uint64_t T, uint32_t pbits,
                                 uint32_t* __restrict__ len) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < T) atomicAdd(&len[pairs[i] >> pbits], 1u);
}

__global__ void new_range_kernel(const uint64_t* __restrict__ pairs, const uint32_t* __restrict__ len,
                                 const uint32_t* __restrict__ eoff, uint32_t nint, uint64_t pmask,
                                 uint32_t* __restrict__ flag) {
  uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nint) return;
  uint32_t f = 1;
  if (k > 0 && len[k] == len[k - 1]) {
    f = 0;
    for (uint32_t t = 0; t < len[k]; ++t) {
      if ((pairs[eoff[k] + t] & pmask) != (pairs[eoff[k - 1] + t] & pmask)) {
        f = 1;
        break;
      }
    }
  }
  flag[k] = f;
}

__global__ void emit_ranges_kernel(const uint32_t* __restrict__ flag, const uint32_t* __restrict__ ridx,
                                   const uint64_t* __restrict__ b, const uint32_t* __restrict__ len,
                                   const uint32_t* __restrict__ eoff, uint32_t nint,
                                   uint64_t* __restrict__ start, uint32_t* __restrict__ rlen,
                                   uint32_t* __restrict__ rsrc) {
  uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nint || !flag[k]) return;
  uint32_t r = ridx[k];
  start[r] = b[k];
  rlen[r] = len[k];
  rsrc[r] = eoff[k];
}

__global__ void fill_lists_kernel(const uint64_t* __restrict__ pairs, uint64_t pmask, uint32_t fl,
                                  const uint32_t* __restrict__ rlen, const uint32_t* __restrict__ rsrc,
                                  const uint32_t* __restrict__ list_off, uint64_t R,
                                  uint32_t* __restrict__ list_ids, uint32_t* __restrict__ pay) {
  uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  uint32_t n = rlen[r], o = list_off[r], s = rsrc[r];
  auto entry = [&](uint64_t pr) {  // polygon field -> slot | flag << 31
    const uint32_t f = (uint32_t)(pr & pmask);
    return fl ? ((f >> 1) | ((f & 1u) << 31)) : f;
  };
  for (uint32_t t = 0; t < n; ++t) list_ids[o + t] = entry(pairs[s + t]);
  if (n == 1) {
    const uint32_t e = entry(pairs[s]);
    pay[r] = (e & VAL_SLOT) | ((e >> 31) << 30);
  } else {
    pay[r] = n == 0 ? NONE : (0x80000000u | (uint32_t)r);
  }
}

__global__ void finish_kernel(uint64_t* start, uint32_t* list_off, uint64_t R, uint64_t top,
                              uint32_t nids) {
  start[R] = top;
  list_off[R] = nids;
}

__global__ void sample_kernel(const uint64_t* __restrict__ start, uint32_t stride, uint32_t ns,
                              uint64_t* __restrict__ sample) {
  uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < ns) sample[j] = start[(uint64_t)j * stride];
}


// ---- merge without nesting: one sort of the records by (query, id)
// Quadtree cells are either nested or disjoint.  When, within every query, no
// record strictly contains another record's start (true for tilings and their
// subsets: cells of different polygons are then identical or disjoint), each
// group of records with the same key is one elementary interval, the gaps
// between groups are empty intervals, and the canonical ranges follow by merging
// equal neighbours.  Keys are (query << qshift) | start.

// Two passes over the sorted records, each thread taking MR consecutive
// records and the groups whose first record is among them (a group may reach
// into the next threads' records; its predecessor is read backwards).  Pass 1
// counts, per block, the ranges the groups open and the list entries of those
// ranges, notes each query's first record and any nesting; pass 2 writes the
// ranges at offsets from block, thread and query prefixes.
constexpr int MT = 256;  // threads per block
constexpr int MR = 8;    // records per thread

struct MergeCtx {
  const uint64_t* sk;
  const uint32_t* sv;
  uint64_t n;
  const CoverQuery* qs;
  uint32_t qshift;
  uint64_t lomask;
};

// the group starting at record a, and what it opens: an empty gap before it
// (bit 0, from gap_lo), itself unless it continues the previous group of its
// query with the same polygon list (bit 1), and after its query's last group
// the empty tail up to 4^F (bit 2)
struct GroupInfo {
  uint64_t lo, hi, gap_lo;
  uint32_t q, k, opens;
  bool first, last, nested;
};

__device__ __forceinline__ bool same_list(const uint32_t* __restrict__ sv, uint64_t a, uint64_t pa,
                                          uint32_t k) {
  // entries are distinct within a group: equal as sets = equal sorted
  for (uint32_t t = 0; t < k; ++t) {
    const uint32_t e = list_entry(sv[a + t]);
    bool found = false;
    for (uint32_t u = 0; u < k && !found; ++u) found = list_entry(sv[pa + u]) == e;
    if (!found) return false;
  }
  return true;
}

__device__ GroupInfo group_at(const MergeCtx& c, uint64_t a) {
  GroupInfo g;
  const uint64_t key = c.sk[a];
  const uint32_t lev = val_level(c.sv[a]);
  g.q = (uint32_t)qof(key, c.qshift);
  g.lo = key & c.lomask;
  g.hi = g.lo + (1ull << (2 * lev));
  g.nested = false;
  uint64_t b = a + 1;
  while (b < c.n && c.sk[b] == key) {
    g.nested |= val_level(c.sv[b]) != lev;  // a cell and its descendant share a start
    ++b;
  }
  g.k = (uint32_t)(b - a);
  g.first = a == 0 || qof(c.sk[a - 1], c.qshift) != g.q;
  uint32_t gap, fresh;
  if (g.first) {
    g.gap_lo = 0;
    gap = g.lo > 0;
    fresh = 1;
  } else {
    const uint64_t pkey = c.sk[a - 1];
    uint64_t pa = a - 1;
    while (pa > 0 && c.sk[pa - 1] == pkey) --pa;
    g.gap_lo = (pkey & c.lomask) + (1ull << (2 * val_level(c.sv[pa])));
    gap = g.lo > g.gap_lo;
    fresh = gap || (a - pa) != g.k || !same_list(c.sv, a, pa, g.k);
  }
  g.last = b == c.n || qof(c.sk[b], c.qshift) != g.q;
  // the next group of the query must start at or after this cell's end
  if (!g.last && c.sk[b] < key + (1ull << (2 * lev))) g.nested = true;
  const uint32_t tail = g.last && g.hi < (1ull << (2 * c.qs[g.q].F));
  g.opens = gap | (fresh << 1) | (tail << 2);
  return g;
}

__device__ __forceinline__ bool is_head(const MergeCtx& c, uint64_t r) {
  return r == 0 || c.sk[r - 1] != c.sk[r];
}

// block sum of a 64-bit value (MT threads)
__device__ __forceinline__ uint64_t block_sum_u64(uint64_t v, uint64_t* s_warp) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
  if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = v;
  __syncthreads();
  uint64_t t = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < MT / 32; ++w) t += s_warp[w];
  return t;
}

// block exclusive scan of a 64-bit value (MT threads)
__device__ __forceinline__ uint64_t block_exscan_u64(uint64_t v, uint64_t* s_warp) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint64_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t t = __shfl_up_sync(FULL, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) s_warp[w] = inc;
  __syncthreads();
  uint64_t pre = 0;
  for (int ww = 0; ww < w; ++ww) pre += s_warp[ww];
  return pre + inc - v;
}

// Records of a block: warp w takes the MR * 32 records from w * MR * 32, lane l
// the records l, l + 32, ... of them (coalesced loads); groups are handled by
// the lane holding their first record, in record order within the warp.
__device__ __forceinline__ uint64_t merge_rec(uint32_t i) {
  return (uint64_t)blockIdx.x * (MT * MR) + (threadIdx.x >> 5) * (32 * MR) + i * 32 +
         (threadIdx.x & 31);
}

// per record: 0 inside a group, else head flag (bit 31), opens (bits 28..30)
// and group size; per block: ranges opened (high 32 bits) and list entries
// (low 32 bits); per query: its first record; any nesting
__global__ __launch_bounds__(MT) void merge_count_kernel(MergeCtx c, uint32_t* __restrict__ code,
                                                         uint64_t* __restrict__ bsum,
                                                         uint32_t* __restrict__ qhead,
                                                         unsigned int* __restrict__ nested) {
  __shared__ uint64_t s_warp[MT / 32];
  uint64_t acc = 0;
  bool nest = false;
  for (uint32_t i = 0; i < MR; ++i) {
    const uint64_t r = merge_rec(i);
    if (r >= c.n) continue;
    uint32_t cd = 0;
    if (is_head(c, r)) {
      const GroupInfo g = group_at(c, r);
      acc += ((uint64_t)__popc(g.opens) << 32) + ((g.opens & 2u) ? g.k : 0u);
      if (g.first) qhead[g.q] = (uint32_t)r;
      nest |= g.nested;
      cd = 0x80000000u | (g.opens << 28) | g.k;
    }
    code[r] = cd;
  }
  if (nest) *nested = 1u;
  const uint64_t t = block_sum_u64(acc, s_warp);
  if (threadIdx.x == 0) bsum[blockIdx.x] = t;
}

struct MergeOut {
  uint64_t* start;
  uint32_t* list_off;
  uint32_t* list_ids;
  uint32_t* pay;
  uint64_t* qopen;   // per query: ranges before its first group, after its last
  uint32_t* qlist;   // per query: list entries before its first group, after its last
};

__global__ __launch_bounds__(MT) void merge_emit_kernel(MergeCtx c, const uint32_t* __restrict__ rcode,
                                                        const uint64_t* __restrict__ boff,
                                                        const uint64_t* __restrict__ extra,
                                                        MergeOut o) {
  __shared__ uint64_t s_warp[MT / 32];
  const uint32_t lane = threadIdx.x & 31;
  // per record of this lane: head flag (bit 31), opens (bits 28..30), group size
  uint32_t code[MR];
  uint64_t wtot = 0;
  for (uint32_t i = 0; i < MR; ++i) {
    const uint64_t r = merge_rec(i);
    code[i] = r < c.n ? rcode[r] : 0u;
    const uint32_t opens = (code[i] >> 28) & 7u, k = code[i] & 0x0fffffffu;
    wtot += ((uint64_t)__popc(opens) << 32) + ((opens & 2u) ? k : 0u);
  }
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) wtot += __shfl_xor_sync(FULL, wtot, s);
  // the warps' totals in record order -> this warp's offset in the block
  const uint64_t wpre = block_exscan_u64(lane == 0 ? wtot : 0ull, s_warp);
  uint64_t run = boff[blockIdx.x] + __shfl_sync(FULL, wpre, 0);
  for (uint32_t i = 0; i < MR; ++i) {
    const uint32_t cd = code[i];
    const uint32_t opens = (cd >> 28) & 7u, k = cd & 0x0fffffffu;
    const uint64_t mine = ((uint64_t)__popc(opens) << 32) + ((opens & 2u) ? k : 0u);
    uint64_t inc = mine;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
      const uint64_t t = __shfl_up_sync(FULL, inc, s);
      if (lane >= (uint32_t)s) inc += t;
    }
    const uint64_t pre = run + inc - mine;
    run += __shfl_sync(FULL, inc, 31);
    if (!(cd >> 31)) continue;
    // the group again, without the list comparison (its outcome is in opens)
    const uint64_t r = merge_rec(i);
    const uint64_t key = c.sk[r];
    const uint32_t q = (uint32_t)qof(key, c.qshift);
    const uint64_t lo = key & c.lomask, hi = lo + (1ull << (2 * val_level(c.sv[r])));
    const bool first = r == 0 || qof(c.sk[r - 1], c.qshift) != q;
    const bool last = r + k == c.n || qof(c.sk[r + k], c.qshift) != q;
    uint64_t ro = pre >> 32;     // ranges before (all queries, no sentinels)
    uint32_t L = (uint32_t)pre;  // list entries before
    if (first) {
      o.qopen[2 * q] = ro;
      o.qlist[2 * q] = L;
    }
    uint64_t e = ro + extra[q];  // entry index: ranges plus earlier queries' extras
    if (opens & 1u) {
      uint64_t gap_lo = 0;
      if (!first) {  // the end of the previous group's cell
        const uint64_t pkey = c.sk[r - 1];
        uint64_t pa = r - 1;
        while (pa > 0 && c.sk[pa - 1] == pkey) --pa;
        gap_lo = (pkey & c.lomask) + (1ull << (2 * val_level(c.sv[pa])));
      }
      o.start[e] = gap_lo;
      o.list_off[e] = L;
      o.pay[e] = NONE;
      ++e;
    }
    if (opens & 2u) {
      o.start[e] = lo;
      o.list_off[e] = L;
      o.pay[e] = k == 1 ? single_pay(c.sv[r]) : (0x80000000u | (uint32_t)e);
      // the list in ascending slot order (groups are small: insertion sort)
      uint32_t* out = o.list_ids + L;
      for (uint32_t t = 0; t < k; ++t) {
        const uint32_t v = list_entry(c.sv[r + t]);
        uint32_t j = t;
        while (j > 0 && (out[j - 1] & VAL_SLOT) > (v & VAL_SLOT)) {
          out[j] = out[j - 1];
          --j;
        }
        out[j] = v;
      }
      L += k;
      ++e;
    }
    if (opens & 4u) {
      o.start[e] = hi;
      o.list_off[e] = L;
      o.pay[e] = NONE;
    }
    ro += __popc(opens);
    if (last) {
      o.qopen[2 * q + 1] = ro;
      o.qlist[2 * q + 1] = L;
    }
  }
}

// per query (one thread each): its offset and record count, its sentinel
// (start 4^F), and the single empty range of a query without records
struct QueryFix {
  uint64_t extra;      // entries of earlier queries that are no ranges of groups
  uint64_t next_head;  // first record of the next query with records (or n)
  uint32_t prev;       // the last earlier query with records (or NONE)
  uint32_t head;       // the query's first record (or NONE)
};

__global__ void merge_finish_kernel(const QueryFix* __restrict__ qf,
                                    const uint64_t* __restrict__ qopen,
                                    const uint32_t* __restrict__ qlist,
                                    const CoverQuery* __restrict__ qs, uint32_t Q,
                                    uint64_t* __restrict__ start, uint32_t* __restrict__ list_off,
                                    uint32_t* __restrict__ pay, uint64_t* __restrict__ qoff,
                                    uint64_t* __restrict__ qcells) {
  const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Q) return;
  const QueryFix f = qf[q];
  uint64_t e;
  uint32_t L;
  if (f.head != NONE) {
    qoff[q] = qopen[2 * q] + f.extra;
    e = qopen[2 * q + 1] + f.extra;
    L = qlist[2 * q + 1];
    qcells[q] = f.next_head - f.head;
  } else {
    const uint64_t ro = f.prev == NONE ? 0ull : qopen[2 * f.prev + 1];
    L = f.prev == NONE ? 0u : qlist[2 * f.prev + 1];
    e = ro + f.extra;
    qoff[q] = e;
    start[e] = 0;
    list_off[e] = L;
    pay[e] = NONE;
    ++e;
    qcells[q] = 0;
  }
  start[e] = 1ull << (2 * qs[q].F);
  list_off[e] = L;
  pay[e] = NONE;
  if (q == Q - 1) qoff[Q] = e + 1;
}

__global__ void set_u32_kernel(uint32_t* p, uint64_t n, uint32_t v) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

int bits_for(uint64_t v) {  // bits needed to represent v
  int b = 0;
  while (b < 64 && (v >> b)) ++b;
  return b;
}

sdb_status read_u64(const unsigned long long* d, unsigned long long* h, int n, cudaStream_t s) {
  SDB_TRY_CUDA(cudaMemcpyAsync(h, d, n * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  SDB_TRY_CUDA(cudaStreamSynchronize(s));
  return SDB_OK;
}

}  // namespace

// records -> canonical ranges, general path (one query, nested cells allowed):
// sweep over all record endpoints (see the file comment)
static sdb_status merge_general(uint64_t* key, uint32_t* val, uint64_t n, uint32_t F, uint32_t P,
                                bool flags, cudaStream_t s, CoverSet* out) {
  const uint32_t fl = flags ? 1u : 0u;  // the pairs' polygon field carries the flag
  Scratch sc(s);
  const uint64_t top = 1ull << (2 * F);
  const uint64_t nbp = 2 * n + 2;
  uint64_t *bp, *bptmp, *bps, *b;
  SDB_TRY(sc.get(&bp, nbp));
  SDB_TRY(sc.get(&bptmp, nbp));
  breakpoints_kernel<<<grid_for(n + 1, 256), 256, 0, s>>>(key, val, n, top, bp);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  SDB_TRY(radix_sort_keys(bp, bptmp, nbp, bits_for(top), s, &bps));
  SDB_TRY(sc.get(&b, nbp));
  size_t m = 0;
  SDB_TRY(unique_sorted(bps, nbp, b, &m, s));
  sc.release(bp);
  sc.release(bptmp);
  if (m < 2 || m > 0xfffffff0ull) {
    set_error("covering: %zu breakpoints out of range", m);
    return SDB_EINVAL;
  }
  const uint32_t nint = (uint32_t)(m - 1);
  uint32_t *klo, *span;
  uint64_t *span64, *poff, *dT;
  SDB_TRY(sc.get(&klo, n));
  SDB_TRY(sc.get(&span, n));
  SDB_TRY(sc.get(&span64, n));
  SDB_TRY(sc.get(&poff, n));
  SDB_TRY(sc.get(&dT, 1));
  spans_kernel<<<grid_for(n, 256), 256, 0, s>>>(key, val, n, b, (uint32_t)m, klo, span);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  widen_kernel<<<grid_for(n, 256), 256, 0, s>>>(span, n, span64);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  SDB_TRY(exclusive_scan<uint64_t>(span64, poff, n, dT, s));
  uint64_t T = 0;
  SDB_TRY_CUDA(cudaMemcpyAsync(&T, dT, sizeof(T), cudaMemcpyDeviceToHost, s));
  SDB_TRY_CUDA(cudaStreamSynchronize(s));
  sc.release(span);
  sc.release(span64);
  if (T >= 0xffffffffull) {
    set_error("covering: %llu (interval, polygon) pairs exceed the 32-bit list range",
              (unsigned long long)T);
    return SDB_ENOMEM;
  }
  const uint32_t pbits = (uint32_t)(bits_for(P > 1 ? P - 1 : 1)) + fl;
  const uint64_t pmask = (1ull << pbits) - 1;
  uint64_t *pairs, *ptmp, *ps;
  SDB_TRY(sc.get(&pairs, T));
  SDB_TRY(sc.get(&ptmp, T));
  if (T) {
    expand_pairs_kernel<<<grid_for(T, 256), 256, 0, s>>>(poff, n, klo, val, T, pbits, fl, pairs);
    note_launch();
    SDB_TRY_CUDA(cudaGetLastError());
  }
  SDB_TRY(radix_sort_keys(pairs, ptmp, T, bits_for((uint64_t)nint) + (int)pbits, s, &ps));
  uint32_t *len, *eoff, *flag, *ridx, *dR;
  SDB_TRY(sc.get(&len, nint));
  SDB_TRY(sc.get(&eoff, nint));
  SDB_TRY(sc.get(&flag, nint));
  SDB_TRY(sc.get(&ridx, nint));
  SDB_TRY(sc.get(&dR, 1));
  SDB_TRY_CUDA(cudaMemsetAsync(len, 0, (size_t)nint * sizeof(uint32_t), s));
  if (T) {
    count_len_kernel<<<grid_for(T, 256), 256, 0, s>>>(ps, T, pbits, len);
    note_launch();
    SDB_TRY_CUDA(cudaGetLastError());
  }
  SDB_TRY(exclusive_scan<uint32_t>(len, eoff, nint, nullptr, s));
  new_range_kernel<<<grid_for(nint, 256), 256, 0, s>>>(ps, len, eoff, nint, pmask, flag);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  SDB_TRY(exclusive_scan<uint32_t>(flag, ridx, nint, dR, s));
  uint32_t R = 0;
  SDB_TRY_CUDA(cudaMemcpyAsync(&R, dR, sizeof(R), cudaMemcpyDeviceToHost, s));
  SDB_TRY_CUDA(cudaStreamSynchronize(s));

  // persistent arrays
  SDB_TRY(dalloc_n(&out->start, (size_t)R + 1, s));
  SDB_TRY(dalloc_n(&out->list_off, (size_t)R + 1, s));
  SDB_TRY(dalloc_n(&out->pay, (size_t)R + 1, s));  // + sentinel entry
  uint32_t *rlen, *rsrc, *dN;
  SDB_TRY(sc.get(&rlen, R));
  SDB_TRY(sc.get(&rsrc, R));
  SDB_TRY(sc.get(&dN, 1));
  emit_ranges_kernel<<<grid_for(nint, 256), 256, 0, s>>>(flag, ridx, b, len, eoff, nint, out->start,
                                                         rlen, rsrc);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  SDB_TRY(exclusive_scan<uint32_t>(rlen, out->list_off, R, dN, s));
  uint32_t nids = 0;
  SDB_TRY_CUDA(cudaMemcpyAsync(&nids, dN, sizeof(nids), cudaMemcpyDeviceToHost, s));
  SDB_TRY_CUDA(cudaStreamSynchronize(s));
  SDB_TRY(dalloc_n(&out->list_ids, (size_t)nids, s));
  fill_lists_kernel<<<grid_for(R, 256), 256, 0, s>>>(ps, pmask, fl, rlen, rsrc, out->list_off, R,
                                                      out->list_ids, out->pay);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  finish_kernel<<<1, 1, 0, s>>>(out->start, out->list_off, R, top, nids);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  set_u32_kernel<<<1, 1, 0, s>>>(out->pay + R, 1, NONE);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  out->E = (uint64_t)R + 1;
  out->nids = nids;
  out->qoff = {0, out->E};
  out->qcells = {n};
  SDB_TRY_CUDA(cudaStreamSynchronize(s));
  return SDB_OK;
}

// records -> canonical ranges: sort by (query, start) once; without nesting
// (see above) the groups give the ranges directly, otherwise (one query only)
// the general sweep runs
static sdb_status merge_records(uint64_t* key, uint32_t* val, uint64_t n, const CoverSpec& spec,
                                const CoverQuery* d_qs, uint32_t qshift, int key_bits,
                                uint32_t sb, cudaStream_t s, CoverSet* out) {
  TraceScope tr("cover.merge", s);
  Scratch sc(s);
  const uint32_t Q = spec.Q;
  if (n >= 0xffffffffull) {
    set_error("covering: %llu cells exceed the 32-bit index range", (unsigned long long)n);
    return SDB_ENOMEM;
  }
  uint64_t *ktmp, *sk;
  uint32_t *vtmp, *sv;
  SDB_TRY(sc.get(&ktmp, n));
  TraceScope tr_sort("cover.sort", s);
  if (sb) {
    // packed records: sort the words on their key bits, then split them
    // (the last pass writes keys and values apart)
    SDB_TRY(sc.get(&sv, n));
    SDB_TRY(radix_sort_split(key, ktmp, n, key_bits, (int)sb + 6, sb, sv, s, &sk));
  } else {
    SDB_TRY(sc.get(&vtmp, n));
    SDB_TRY(radix_sort_pairs(key, val, ktmp, vtmp, n, key_bits, s, &sk, &sv));
  }
  // pass 1: per block, the ranges and list entries its groups open; each
  // query's first record; nesting
  const uint64_t per_block = (uint64_t)MT * MR;
  const uint64_t nb = n ? (n + per_block - 1) / per_block : 0;
  uint64_t *bsum, *boff, *dtot;
  uint32_t *qhead, *rcode;
  unsigned int* nested;
  SDB_TRY(sc.get(&rcode, n ? n : 1));
  SDB_TRY(sc.get(&bsum, nb ? nb : 1));
  SDB_TRY(sc.get(&boff, nb ? nb : 1));
  SDB_TRY(sc.get(&dtot, 1));
  SDB_TRY(sc.get(&qhead, Q));
  SDB_TRY(sc.get(&nested, 1));
  SDB_TRY_CUDA(cudaMemsetAsync(nested, 0, sizeof(unsigned int), s));
  SDB_TRY_CUDA(cudaMemsetAsync(qhead, 0xff, (size_t)Q * 4, s));
  SDB_TRY_CUDA(cudaMemsetAsync(dtot, 0, 8, s));
  const MergeCtx mc{sk, sv, n, d_qs, qshift, qshift >= 64 ? ~0ull : ((1ull << qshift) - 1ull)};
  tr_sort.end();
  if (nb) {
    TraceScope tr1("cover.count", s);
    merge_count_kernel<<<(unsigned)nb, MT, 0, s>>>(mc, rcode, bsum, qhead, nested);
    note_launch();
    SDB_TRY_CUDA(cudaGetLastError());
    SDB_TRY(exclusive_scan<uint64_t>(bsum, boff, nb, dtot, s));
  }
  uint64_t tot = 0;
  unsigned int hnest = 0;
  std::vector<uint32_t> hhead(Q);
  SDB_TRY_CUDA(cudaMemcpyAsync(&tot, dtot, 8, cudaMemcpyDeviceToHost, s));
  SDB_TRY_CUDA(cudaMemcpyAsync(&hnest, nested, 4, cudaMemcpyDeviceToHost, s));
  SDB_TRY_CUDA(cudaMemcpyAsync(hhead.data(), qhead, (size_t)Q * 4, cudaMemcpyDeviceToHost, s));
  SDB_TRY_CUDA(cudaStreamSynchronize(s));
  if (hnest) {
    if (Q != 1) {
      set_error("batched coverings need polygons that do not overlap within a query");
      return SDB_EINVAL;
    }
    uint32_t P = 0;
    for (uint32_t i = 0; i < spec.NP; ++i) P = spec.pair_slot[i] + 1 > P ? spec.pair_slot[i] + 1 : P;
    return merge_general(sk, sv, n, spec.q[0].F, P, spec.flags, s, out);
  }
  // entries: the groups' ranges, plus per query its sentinel, plus the empty
  // range of a query without records
  std::vector<QueryFix> hq(Q);
  uint64_t extra = 0;
  uint32_t prev = NONE;
  for (uint32_t q = 0; q < Q; ++q) {
    hq[q].extra = extra;
    hq[q].head = hhead[q];
    hq[q].prev = prev;
    extra += hhead[q] == NONE ? 2 : 1;
    if (hhead[q] != NONE) prev = q;
  }
  uint64_t next = n;
  for (uint32_t q = Q; q-- > 0;) {
    hq[q].next_head = next;
    if (hhead[q] != NONE) next = hhead[q];
  }
  const uint64_t E = (tot >> 32) + extra;
  const uint64_t nids = tot & 0xffffffffull;
  if (E >= 0x7fffffffull) {  // entry indices travel in 31 bits of the packed payload
    set_error("covering: %llu ranges exceed the 32-bit index range", (unsigned long long)E);
    return SDB_ENOMEM;
  }
  SDB_TRY(dalloc_n(&out->start, E, s));
  SDB_TRY(dalloc_n(&out->list_off, E, s));
  SDB_TRY(dalloc_n(&out->pay, E, s));
  SDB_TRY(dalloc_n(&out->list_ids, nids ? nids : 1, s));
  QueryFix* dq;
  uint64_t *qopen, *qoff, *qcells, *dextra;
  uint32_t* qlist;
  SDB_TRY(sc.get(&dq, Q));
  SDB_TRY(sc.get(&qopen, 2 * (size_t)Q));
  SDB_TRY(sc.get(&qlist, 2 * (size_t)Q));
  SDB_TRY(sc.get(&qoff, (size_t)Q + 1));
  SDB_TRY(sc.get(&qcells, Q));
  SDB_TRY(sc.get(&dextra, Q));
  std::vector<uint64_t> hextra(Q);
  for (uint32_t q = 0; q < Q; ++q) hextra[q] = hq[q].extra;
  SDB_TRY_CUDA(cudaMemcpyAsync(dq, hq.data(), (size_t)Q * sizeof(QueryFix), cudaMemcpyHostToDevice, s));
  SDB_TRY_CUDA(cudaMemcpyAsync(dextra, hextra.data(), (size_t)Q * 8, cudaMemcpyHostToDevice, s));
  // pass 2: the ranges
  if (nb) {
    TraceScope tr2("cover.emit", s);
    const MergeOut mo{out->start, out->list_off, out->list_ids, out->pay, qopen, qlist};
    merge_emit_kernel<<<(unsigned)nb, MT, 0, s>>>(mc, rcode, boff, dextra, mo);
    note_launch();
    SDB_TRY_CUDA(cudaGetLastError());
  }
  merge_finish_kernel<<<grid_for(Q, 256), 256, 0, s>>>(dq, qopen, qlist, d_qs, Q, out->start,
                                                       out->list_off, out->pay, qoff, qcells);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  out->qoff.assign((size_t)Q + 1, 0);
  out->qcells.assign(Q, 0);
  SDB_TRY_CUDA(cudaMemcpyAsync(out->qoff.data(), qoff, ((size_t)Q + 1) * 8, cudaMemcpyDeviceToHost,
                               s));
  SDB_TRY_CUDA(cudaMemcpyAsync(out->qcells.data(), qcells, (size_t)Q * 8, cudaMemcpyDeviceToHost,
                               s));
  SDB_TRY_CUDA(cudaStreamSynchronize(s));
  out->E = E;
  out->nids = nids;
  return SDB_OK;
}

void CoverSet::release(cudaStream_t s) {
  dfree(start, s);
  dfree(list_off, s);
  dfree(list_ids, s);
  dfree(pay, s);
  start = nullptr;
  list_off = nullptr;
  list_ids = nullptr;
  pay = nullptr;
}

static sdb_status launch_expand(uint32_t G, const Item* items, uint32_t n_items, const uint32_t* elist,
                         const Edge* edges, const uint32_t* pq, const uint32_t* ps,
                         const CoverQuery* qs, uint32_t qshift, uint32_t bflag, bool noncons,
                         uint32_t B, uint32_t L,
                         Item* nitems, uint32_t* nel, uint64_t* rkey, uint32_t* rval, uint32_t sb,
                         unsigned long long rec_base, unsigned long long* ctr, cudaStream_t s) {
  const size_t threads = (size_t)n_items * G;
#define SDB_EXPAND(g)                                                                          \
  case g:                                                                                      \
    if (noncons)                                                                               \
      expand_level_kernel<g, true><<<grid_for(threads, 256), 256, 0, s>>>(                     \
          items, n_items, elist, edges, pq, ps, qs, qshift, bflag, B, L, nitems, nel, rkey,     \
          rval, sb, rec_base, ctr);                                                            \
    else                                                                                       \
      expand_level_kernel<g, false><<<grid_for(threads, 256), 256, 0, s>>>(                    \
          items, n_items, elist, edges, pq, ps, qs, qshift, bflag, B, L, nitems, nel, rkey,     \
          rval, sb, rec_base, ctr);                                                            \
    break;
  switch (G) {
    SDB_EXPAND(1)
    SDB_EXPAND(2)
    SDB_EXPAND(4)
    SDB_EXPAND(8)
    SDB_EXPAND(16)
    SDB_EXPAND(32)
    default:
      set_error("expand: bad lane count %u", G);
      return SDB_EINVAL;
  }
#undef SDB_EXPAND
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  return SDB_OK;
}

// Capacity hints from earlier builds of the same shape in this process
// (records, frontier cells, frontier edge entries), so that a repeated build
// allocates its buffers once instead of growing them level by level (a grown
// record buffer is a new allocation plus a copy).  Builds of other shapes (the
// varied small builds of a serving loop) start small and grow.  Hints only: a
// build that needs more still grows.
struct BuildShape {
  uint32_t B, Q, NP, V, Fmax;
  bool operator==(const BuildShape& o) const {
    return B == o.B && Q == o.Q && NP == o.NP && V == o.V && Fmax == o.Fmax;
  }
};
struct BuildHint {
  uint64_t rec = 1ull << 20, items = 1ull << 12, edges = 1ull << 14;
};
std::mutex g_hint_mu;
std::vector<std::pair<BuildShape, BuildHint>> g_hints;  // most recent last, at most 16

BuildHint hint_for(const BuildShape& k) {
  std::lock_guard<std::mutex> lk(g_hint_mu);
  for (const auto& e : g_hints)
    if (e.first == k) return e.second;
  return BuildHint{};
}

void keep_hint(const BuildShape& k, const BuildHint& h) {
  std::lock_guard<std::mutex> lk(g_hint_mu);
  for (auto it = g_hints.begin(); it != g_hints.end(); ++it)
    if (it->first == k) {
      g_hints.erase(it);
      break;
    }
  if (g_hints.size() >= 16) g_hints.erase(g_hints.begin());
  g_hints.emplace_back(k, h);
}

uint64_t pow2_at_least(uint64_t v) {
  uint64_t p = 1;
  while (p < v) p <<= 1;
  return p;
}

sdb_status build_coverings(const PolyEdges& pe, const CoverSpec& spec, cudaStream_t s,
                           CoverSet* out) {
  TraceScope tr("cover.build", s);
  const uint32_t P = pe.P;
  const uint32_t V = pe.V;
  const uint32_t B = spec.B, Q = spec.Q, NP = spec.NP;
  uint32_t Fmax = 0;
  for (uint32_t q = 0; q < Q; ++q) Fmax = spec.q[q].F > Fmax ? spec.q[q].F : Fmax;
  // record keys: (query << qshift) | start; one query needs no query bits
  uint32_t qshift = 64;
  int key_bits = bits_for(1ull << (2 * Fmax));
  if (Q > 1) {
    // ids are below 4^F; a range end may reach 4^F and carry into the query
    // field, which the merge never compares across queries
    qshift = 2 * Fmax;
    key_bits = (int)qshift + bits_for(Q - 1);
    if (key_bits > 64) {
      set_error("batched coverings: %u queries at finest level %u do not fit 64-bit keys", Q, Fmax);
      return SDB_EINVAL;
    }
  }
  Scratch sc(s);
  // polygons -> device edges
  TraceScope tr_up("cover.setup", s);
  uint32_t *d_off, *d_x, *d_y, *d_vp, *elist, *d_pp, *d_pq, *d_ps;
  CoverQuery* d_qs;
  Edge* edges;
  SDB_TRY(sc.get(&d_off, P + 1));
  SDB_TRY(sc.get(&d_x, V));
  SDB_TRY(sc.get(&d_y, V));
  SDB_TRY(sc.get(&d_vp, V));
  SDB_TRY(sc.get(&edges, V));
  SDB_TRY(sc.get(&elist, V));
  SDB_TRY(sc.get(&d_pp, NP));
  SDB_TRY(sc.get(&d_pq, NP));
  SDB_TRY(sc.get(&d_ps, NP));
  SDB_TRY(sc.get(&d_qs, Q));
  SDB_TRY_CUDA(cudaMemcpyAsync(d_off, pe.edge_off.data(), (P + 1) * 4ull, cudaMemcpyHostToDevice, s));
  SDB_TRY_CUDA(cudaMemcpyAsync(d_x, pe.x, V * 4ull, cudaMemcpyHostToDevice, s));
  SDB_TRY_CUDA(cudaMemcpyAsync(d_y, pe.y, V * 4ull, cudaMemcpyHostToDevice, s));
  SDB_TRY_CUDA(cudaMemcpyAsync(d_vp, pe.next.data(), V * 4ull, cudaMemcpyHostToDevice, s));
  if (NP) {
    SDB_TRY_CUDA(cudaMemcpyAsync(d_pp, spec.pair_poly, NP * 4ull, cudaMemcpyHostToDevice, s));
    SDB_TRY_CUDA(cudaMemcpyAsync(d_pq, spec.pair_query, NP * 4ull, cudaMemcpyHostToDevice, s));
    SDB_TRY_CUDA(cudaMemcpyAsync(d_ps, spec.pair_slot, NP * 4ull, cudaMemcpyHostToDevice, s));
  }
  SDB_TRY_CUDA(cudaMemcpyAsync(d_qs, spec.q, Q * sizeof(CoverQuery), cudaMemcpyHostToDevice, s));
  build_edges_kernel<<<grid_for(V, 256), 256, 0, s>>>(d_x, d_y, d_vp, V, edges, elist);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());

  // record buffer, grown on demand; packed into one word per record when the
  // key, the slot, the level and the flag fit 64 bits
  uint32_t max_slot = 0;
  for (uint32_t i = 0; i < NP; ++i) max_slot = spec.pair_slot[i] > max_slot ? spec.pair_slot[i] : max_slot;
  uint32_t sb = (uint32_t)bits_for(max_slot);
  if (sb < 1) sb = 1;
  if (key_bits + (int)sb + 6 > 64) sb = 0;
  const BuildShape shape{B, Q, NP, V, Fmax};
  const BuildHint hint = hint_for(shape);
  BuildHint seen;
  seen.rec = seen.items = seen.edges = 0;
  uint64_t rec_cap = hint.rec, n_rec = 0;
  if (rec_cap < 8ull * NP) rec_cap = 8ull * NP;
  uint64_t* rkey = nullptr;
  uint32_t* rval = nullptr;
  SDB_TRY(dalloc_n(&rkey, rec_cap, s));
  if (!sb) SDB_TRY(dalloc_n(&rval, rec_cap, s));
  struct Free {
    uint64_t** k;
    uint32_t** v;
    cudaStream_t s;
    ~Free() {
      dfree(*k, s);
      dfree(*v, s);
    }
  } free_recs{&rkey, &rval, s};

  const uint32_t bflag = spec.flags ? VAL_FLAG : 0u;  // boundary records' flag
  unsigned long long* ctr;
  SDB_TRY(sc.get(&ctr, 3));
  SDB_TRY_CUDA(cudaMemsetAsync(ctr, 0, 3 * sizeof(unsigned long long), s));
  // frontier cells and edge lists, two buffers each (this level's, the next's)
  struct Frontier {
    Item* f[2] = {nullptr, nullptr};
    uint32_t* e[2] = {nullptr, nullptr};
    bool own_e[2] = {false, true};
    cudaStream_t s;
    ~Frontier() {
      dfree(f[0], s);
      dfree(f[1], s);
      if (own_e[0]) dfree(e[0], s);
      if (own_e[1]) dfree(e[1], s);
    }
  } fr;
  fr.s = s;
  Item** fbuf = fr.f;
  uint32_t** ebuf = fr.e;
  uint64_t fcap[2], ecap[2];
  fcap[0] = hint.items;
  if (fcap[0] < NP) fcap[0] = pow2_at_least(NP);
  fcap[1] = fcap[0];
  ecap[0] = V;  // the polygons' own edge lists (scratch)
  ecap[1] = hint.edges;
  SDB_TRY(dalloc_n(&fbuf[0], fcap[0], s));
  SDB_TRY(dalloc_n(&fbuf[1], fcap[1], s));
  SDB_TRY(dalloc_n(&ebuf[1], ecap[1], s));
  ebuf[0] = elist;
  Item* items = fbuf[0];
  if (NP) {
    root_items_kernel<<<grid_for((size_t)NP * 32, 256), 256, 0, s>>>(
        d_off, edges, d_pp, d_pq, d_ps, d_qs, NP, qshift, bflag, spec.noncons, B, items, rkey, rval,
        sb, ctr);
    note_launch();
    SDB_TRY_CUDA(cudaGetLastError());
  }
  unsigned long long h0[3];
  SDB_TRY(read_u64(ctr, h0, 3, s));
  uint64_t n_items = h0[0], n_edges = 0;
  n_rec = h0[2];
  for (uint32_t i = 0; i < NP; ++i)
    if (spec.q[spec.pair_query[i]].F > 0)
      n_edges += pe.edge_off[spec.pair_poly[i] + 1] - pe.edge_off[spec.pair_poly[i]];
  uint32_t* cur_el = elist;
  tr_up.end();
  TraceScope tr_lv("cover.levels", s);
  for (uint32_t L = 0; L < Fmax && n_items > 0; ++L) {
    const bool last = (L + 1 == Fmax);
    // capacity: every record and every child item comes from one of 4
    // children; every child edge entry from one (edge, child) pair
    if (n_rec + 4 * n_items > rec_cap) {
      uint64_t nc = rec_cap;
      while (nc < n_rec + 4 * n_items) nc *= 2;
      uint64_t* k2 = nullptr;
      uint32_t* v2 = nullptr;
      SDB_TRY(dalloc_n(&k2, nc, s));
      SDB_TRY_CUDA(cudaMemcpyAsync(k2, rkey, n_rec * 8, cudaMemcpyDeviceToDevice, s));
      dfree(rkey, s);
      rkey = k2;
      if (!sb) {
        SDB_TRY(dalloc_n(&v2, nc, s));
        SDB_TRY_CUDA(cudaMemcpyAsync(v2, rval, n_rec * 4, cudaMemcpyDeviceToDevice, s));
        dfree(rval, s);
        rval = v2;
      }
      rec_cap = nc;
    }
    if (4 * n_items > 0xffffffffull || 4 * n_edges > 0xffffffffull) {
      set_error("covering: level %u frontier too large (%llu cells, %llu edge entries)", L,
                (unsigned long long)n_items, (unsigned long long)n_edges);
      return SDB_ENOMEM;
    }
    Item* nitems = nullptr;
    uint32_t* nel = nullptr;
    if (!last) {
      // the other buffer of each pair, grown (contents are dead) when short
      sdb_status st = SDB_OK;
      if (fcap[1] < 4 * n_items) {
        dfree(fbuf[1], s);
        fbuf[1] = nullptr;
        fcap[1] = pow2_at_least(4 * n_items);
        st = dalloc_n(&fbuf[1], fcap[1], s);
      }
      if (st == SDB_OK && ecap[1] < 4 * n_edges) {
        if (fr.own_e[1]) dfree(ebuf[1], s);
        ebuf[1] = nullptr;
        fr.own_e[1] = true;
        ecap[1] = pow2_at_least(4 * n_edges);
        st = dalloc_n(&ebuf[1], ecap[1], s);
      }
      if (st != SDB_OK) return st;
      nitems = fbuf[1];
      nel = ebuf[1];
    }
    SDB_TRY_CUDA(cudaMemsetAsync(ctr, 0, 3 * sizeof(unsigned long long), s));
    // lanes per item: about the level's mean edge count, a power of two <= 32
    const uint64_t mean = (n_edges + n_items - 1) / n_items;
    uint32_t G = 1;
    if (mean >= 4)
      while (G < 32 && G < mean) G <<= 1;
    {
      TraceScope tr("cover.expand", s);
      SDB_TRY(launch_expand(G, items, (uint32_t)n_items, cur_el, edges, d_pq, d_ps, d_qs, qshift,
                            bflag, spec.noncons, B, L, nitems, nel, rkey, rval, sb, n_rec, ctr,
                            s));
      SDB_TRY_CUDA(cudaGetLastError());
    }
    unsigned long long h[3];
    SDB_TRY(read_u64(ctr, h, 3, s));
    // the next level reads what this one wrote
    std::swap(fbuf[0], fbuf[1]);
    std::swap(fcap[0], fcap[1]);
    std::swap(ebuf[0], ebuf[1]);
    std::swap(ecap[0], ecap[1]);
    std::swap(fr.own_e[0], fr.own_e[1]);
    items = fbuf[0];
    cur_el = ebuf[0];
    n_items = last ? 0 : h[0];
    n_edges = h[1];
    n_rec += h[2];
    seen.items = std::max<uint64_t>(seen.items, pow2_at_least(4 * n_items));
    seen.edges = std::max<uint64_t>(seen.edges, pow2_at_least(4 * n_edges));
  }
  tr_lv.end();
  seen.rec = std::max<uint64_t>(pow2_at_least(n_rec), 1ull << 16);
  seen.items = std::max<uint64_t>(seen.items, 1ull << 12);
  seen.edges = std::max<uint64_t>(seen.edges, 1ull << 14);
  keep_hint(shape, seen);
  out->ncells = n_rec;
  return merge_records(rkey, rval, n_rec, spec, d_qs, qshift, key_bits, sb, s, out);
}

sdb_status finish_covering(sdb_covering* cov, cudaStream_t s);

sdb_status build_covering_device(const PolyEdges& pe, uint32_t B, uint32_t k, uint32_t options,
                                 cudaStream_t s, sdb_covering* cov) {
  const uint32_t P = pe.P;
  const bool flags = (options & SDB_COVER_BOUNDARY_FLAGS) != 0;
  const uint32_t F = B - k;
  cov->B = B;
  cov->k = k;
  cov->F = F;
  cov->P = P;
  std::vector<uint32_t> pp(P), pq(P, 0);
  for (uint32_t j = 0; j < P; ++j) pp[j] = j;
  CoverQuery q{F, 0, 0, 1u << B, 1u << B};
  CoverSpec spec;
  spec.B = B;
  spec.Q = 1;
  spec.q = &q;
  spec.NP = P;
  spec.pair_poly = pp.data();
  spec.pair_query = pq.data();
  spec.pair_slot = pp.data();
  spec.flags = flags;
  spec.noncons = (options & SDB_COVER_NONCONSERVATIVE) != 0;
  cov->flagged = flags;
  CoverSet cs;
  sdb_status st = build_coverings(pe, spec, s, &cs);
  if (st != SDB_OK) {
    cs.release(s);
    return st;
  }
  cov->start = cs.start;
  cov->list_off = cs.list_off;
  cov->list_ids = cs.list_ids;
  cov->pay = cs.pay;
  cov->R = cs.E - 1;
  cov->nids = cs.nids;
  cov->ncells = cs.ncells;
  return finish_covering(cov, s);
}

// the binary search's shared-memory sample of the starts, and the size
sdb_status finish_covering(sdb_covering* cov, cudaStream_t s) {
  const uint32_t SAMPLE_MAX = 2048;
  const uint64_t keys = cov->R + 1;
  uint32_t stride = (uint32_t)((keys + SAMPLE_MAX - 1) / SAMPLE_MAX);
  if (stride < 1) stride = 1;
  const uint32_t ns = (uint32_t)((keys + stride - 1) / stride);
  SDB_TRY(dalloc_n(&cov->sample, ns, s));
  sample_kernel<<<grid_for(ns, 256), 256, 0, s>>>(cov->start, stride, ns, cov->sample);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  cov->sample_n = ns;
  cov->sample_stride = stride;
  cov->bytes = (size_t)keys * 16 + (size_t)cov->nids * 4 + (size_t)ns * 8;
  SDB_TRY_CUDA(cudaStreamSynchronize(s));
  return SDB_OK;
}

namespace {
// list offsets of a slice rebased to its first entry
__global__ void rebase_u32_kernel(const uint32_t* __restrict__ in, uint64_t n,
                                  uint32_t* __restrict__ out) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = in[i] - in[0];
}
// payloads of a slice: list references rebased by the slice's first entry
__global__ void rebase_pay_kernel(const uint32_t* __restrict__ in, uint64_t n, uint32_t base,
                                  uint32_t* __restrict__ out) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t v = in[i];
  out[i] = (v != NONE && (v & 0x80000000u)) ? (0x80000000u | ((v & 0x7fffffffu) - base)) : v;
}
}  // namespace

sdb_status build_coverings_multi(const PolyEdges& pe, uint32_t B, const uint32_t* ks, uint32_t nq,
                                 uint32_t options, cudaStream_t s, sdb_covering* const* covs) {
  const uint32_t P = pe.P;
  std::vector<CoverQuery> q(nq);
  std::vector<uint32_t> pp((size_t)P * nq), pq((size_t)P * nq), ps((size_t)P * nq);
  for (uint32_t i = 0; i < nq; ++i) {
    q[i] = CoverQuery{B - ks[i], 0, 0, 1u << B, 1u << B};
    for (uint32_t j = 0; j < P; ++j) {
      pp[(size_t)i * P + j] = j;
      pq[(size_t)i * P + j] = i;
      ps[(size_t)i * P + j] = j;
    }
  }
  CoverSpec spec;
  spec.B = B;
  spec.Q = nq;
  spec.q = q.data();
  spec.NP = P * nq;
  spec.pair_poly = pp.data();
  spec.pair_query = pq.data();
  spec.pair_slot = ps.data();
  spec.flags = (options & SDB_COVER_BOUNDARY_FLAGS) != 0;
  spec.noncons = (options & SDB_COVER_NONCONSERVATIVE) != 0;
  CoverSet cs;
  sdb_status st = nq > 1 ? build_coverings(pe, spec, s, &cs) : SDB_EINVAL;
  if (st != SDB_OK) {
    // overlapping polygons (the joint merge needs disjoint cells per query),
    // a key that does not fit, or one shift: one pass per shift
    cs.release(s);
    cudaStreamSynchronize(s);
    for (uint32_t i = 0; i < nq; ++i) {
      covs[i]->B = B;
      SDB_TRY(build_covering_device(pe, B, ks[i], options, s, covs[i]));
    }
    return SDB_OK;
  }
  // each query's slice [qoff[i], qoff[i+1]) (its last entry the sentinel)
  std::vector<uint32_t> lo(nq + 1, 0);
  for (uint32_t i = 0; i < nq; ++i)
    SDB_TRY_CUDA(cudaMemcpyAsync(&lo[i], cs.list_off + cs.qoff[i], 4, cudaMemcpyDeviceToHost, s));
  lo[nq] = (uint32_t)cs.nids;
  SDB_TRY_CUDA(cudaStreamSynchronize(s));
  sdb_status rc = SDB_OK;
  auto ck = [](cudaError_t e) {
    return e == cudaSuccess ? SDB_OK : cuda_status(e, "covering slice", __FILE__, __LINE__);
  };
  for (uint32_t i = 0; i < nq && rc == SDB_OK; ++i) {
    sdb_covering* c = covs[i];
    const uint64_t a = cs.qoff[i], e = cs.qoff[i + 1] - a;
    c->B = B;
    c->k = ks[i];
    c->F = B - ks[i];
    c->P = P;
    c->flagged = spec.flags;
    c->R = e - 1;
    c->nids = lo[i + 1] - lo[i];
    c->ncells = cs.qcells[i];
    rc = dalloc_n(&c->start, e, s);
    if (rc == SDB_OK) rc = dalloc_n(&c->list_off, e, s);
    if (rc == SDB_OK) rc = dalloc_n(&c->pay, e, s);
    if (rc == SDB_OK) rc = dalloc_n(&c->list_ids, c->nids, s);
    if (rc != SDB_OK) break;
    rc = ck(cudaMemcpyAsync(c->start, cs.start + a, e * 8, cudaMemcpyDeviceToDevice, s));
    if (rc == SDB_OK && c->nids)
      rc = ck(cudaMemcpyAsync(c->list_ids, cs.list_ids + lo[i], (size_t)c->nids * 4,
                              cudaMemcpyDeviceToDevice, s));
    if (rc != SDB_OK) break;
    rebase_u32_kernel<<<grid_for(e, 256), 256, 0, s>>>(cs.list_off + a, e, c->list_off);
    note_launch();
    rebase_pay_kernel<<<grid_for(e, 256), 256, 0, s>>>(cs.pay + a, e, (uint32_t)a, c->pay);
    note_launch();
    rc = ck(cudaGetLastError());
    if (rc == SDB_OK) rc = finish_covering(c, s);
  }
  cs.release(s);
  return rc;
}

}  // namespace sdb
