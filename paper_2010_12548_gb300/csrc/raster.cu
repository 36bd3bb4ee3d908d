// Bounded Raster Join (Sec. 5.2) restated in CUDA, on device buffers (no
// graphics API).  The plan of the paper's operators:
//   blend:  every point adds (1, attr) to its pixel of a uniform canvas whose
//           pixels are the finest cells (side 2^k, so the pixel diagonal is at
//           most eps, Sec. 2.2) -- per-pixel partial aggregates;
//   mask:   every polygon is rasterised conservatively onto the same pixels
//           (a pixel belongs to the polygon when the closed pixel meets the
//           closed polygon);
//   reduce: the masked pixels' aggregates are summed per polygon.
// The canvas has 4^F pixels; it is cut into tiles of 2^t x 2^t pixels that are
// processed a group at a time (the paper divides the canvas when the
// resolution exceeds what the GPU supports).  Inside a tile, each pixel row is
// turned into inclusive prefix sums, so the mask-and-reduce of one polygon row
// costs one subtraction per covered span.
//
// Conservative rasterisation of polygon row y (closed strip Y0 = y*s .. Y0+s):
//  * every edge that meets the strip touches the pixels whose closed x-range
//    meets the x-range of the edge clipped to the strip;
//  * a pixel that no edge touches lies wholly inside or outside; it is inside
//    when its lower-left corner (m*s, Y0) is, which the crossings of the line
//    y = Y0 decide (half-open rule: an edge crosses when exactly one end is
//    above Y0), corners strictly between the 2i-th and (2i+1)-th crossing being
//    inside.
// All coordinates are integers; crossings and clipped ends are exact
// rationals (int64 numerator, positive denominator), floors and ceilings are
// exact, comparisons use 128-bit products.
#include "sdb_internal.cuh"

namespace sdb {

namespace {

constexpr int MAXI = 128;  // spans / crossings of one polygon row (compacted when full)
constexpr int THREADS = 128;
constexpr uint32_t SMEM_EDGES = 2048;

struct REdge {
  int32_t ax, ay, bx, by;
};

// exact floor / ceil of n / d for d > 0
__device__ __forceinline__ int64_t fdiv(int64_t n, int64_t d) {
  int64_t q = n / d;
  return (n % d != 0 && n < 0) ? q - 1 : q;
}
__device__ __forceinline__ int64_t cdiv(int64_t n, int64_t d) {
  int64_t q = n / d;
  return (n % d != 0 && n > 0) ? q + 1 : q;
}

__device__ __forceinline__ int64_t imax64(int64_t a, int64_t b) { return a > b ? a : b; }
__device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

struct Rat {  // n / d, d > 0
  int64_t n, d;
};
__device__ __forceinline__ bool rat_less(const Rat& a, const Rat& b) {
  return (__int128)a.n * b.d < (__int128)b.n * a.d;
}

// x of edge e at height y (the edge is not horizontal and spans y)
__device__ __forceinline__ Rat x_at(const REdge& e, int64_t y) {
  int64_t D = (int64_t)e.by - e.ay;
  int64_t N = (int64_t)e.ax * D + (y - e.ay) * ((int64_t)e.bx - e.ax);
  if (D < 0) {
    D = -D;
    N = -N;
  }
  return Rat{N, D};
}

// -------------------------------------------------------------- points
__global__ void tile_keys_kernel(const uint32_t* __restrict__ x, const uint32_t* __restrict__ y,
                                 uint64_t n, uint32_t B, uint32_t k, uint32_t F, uint32_t t,
                                 uint64_t ntiles, uint64_t* __restrict__ key,
                                 uint32_t* __restrict__ idx) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t xi = x[i], yi = y[i];
  const bool in = !((xi | yi) >> B);
  const uint64_t tx = (uint64_t)(xi >> k) >> t, ty = (uint64_t)(yi >> k) >> t;
  key[i] = in ? (ty << (F - t)) + tx : ntiles;  // outside the grid: after every tile
  idx[i] = (uint32_t)i;
}

__global__ void tile_bounds_kernel(const uint64_t* __restrict__ key, uint64_t n, uint64_t ntiles,
                                   uint64_t* __restrict__ off) {
  const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j > ntiles) return;
  uint64_t lo = 0, len = n;  // first position with key >= j
  while (len > 0) {
    const uint64_t half = len >> 1;
    if (key[lo + half] < j) {
      lo += half + 1;
      len -= half + 1;
    } else {
      len = half;
    }
  }
  off[j] = lo;
}

struct Canvas {
  unsigned long long* cnt;  // [G][T][T], row-major, then inclusive row prefixes
  unsigned long long* sum;
  uint32_t T, t, F, k, B;
  uint64_t tiles_per_side;
  uint64_t tile0;  // first tile of the group
};

// blend: the group's points into their tile canvases
__global__ void blend_kernel(Canvas C, const uint32_t* __restrict__ x, const uint32_t* __restrict__ y,
                             const int32_t* __restrict__ a, const uint32_t* __restrict__ idx,
                             const uint64_t* __restrict__ off, uint32_t G, bool identity,
                             uint64_t n) {
  const uint32_t g = blockIdx.y;
  if (g >= G) return;
  const uint64_t tile = C.tile0 + g;
  const uint64_t b = identity ? 0 : off[tile], e = identity ? n : off[tile + 1];
  const uint64_t tx0 = (tile % C.tiles_per_side) << C.t, ty0 = (tile / C.tiles_per_side) << C.t;
  const uint64_t base = (uint64_t)g * C.T * C.T;
  for (uint64_t p = b + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < e;
       p += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t i = identity ? (uint32_t)p : idx[p];
    const uint32_t xi = x[i], yi = y[i];
    if ((xi | yi) >> C.B) continue;
    const uint64_t px = (xi >> C.k) - tx0, py = (yi >> C.k) - ty0;
    const uint64_t pix = base + py * C.T + px;
    atomicAdd(C.cnt + pix, 1ull);
    if (a) atomicAdd(C.sum + pix, (unsigned long long)(long long)a[i]);
  }
}

// inclusive prefix sums along every pixel row (one block per row)
__global__ void row_prefix_kernel(Canvas C, uint32_t rows) {
  const uint32_t row = blockIdx.x;
  if (row >= rows) return;
  __shared__ unsigned long long carry_c, carry_s;
  __shared__ unsigned long long wc[THREADS / 32], ws[THREADS / 32];
  unsigned long long* rc = C.cnt + (uint64_t)row * C.T;
  unsigned long long* rs = C.sum + (uint64_t)row * C.T;
  if (threadIdx.x == 0) carry_c = carry_s = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (uint32_t c0 = 0; c0 < C.T; c0 += THREADS) {
    const uint32_t c = c0 + threadIdx.x;
    unsigned long long vc = c < C.T ? rc[c] : 0, vs = c < C.T ? rs[c] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long tc = __shfl_up_sync(0xffffffffu, vc, o);
      const unsigned long long ts = __shfl_up_sync(0xffffffffu, vs, o);
      if (lane >= o) {
        vc += tc;
        vs += ts;
      }
    }
    if (lane == 31) {
      wc[w] = vc;
      ws[w] = vs;
    }
    __syncthreads();
    unsigned long long pc = carry_c, ps = carry_s;
    for (int i = 0; i < w; ++i) {
      pc += wc[i];
      ps += ws[i];
    }
    if (c < C.T) {
      rc[c] = vc + pc;
      rs[c] = vs + ps;
    }
    __syncthreads();
    if (threadIdx.x == THREADS - 1) {
      carry_c = vc + pc;
      carry_s = vs + ps;
    }
    __syncthreads();
  }
}

struct Span {
  int32_t a, b;
};

__device__ __forceinline__ void sort_spans(Span* s, int n) {
  for (int i = 1; i < n; ++i) {
    const Span v = s[i];
    int j = i;
    while (j > 0 && s[j - 1].a > v.a) {
      s[j] = s[j - 1];
      --j;
    }
    s[j] = v;
  }
}

// sort and merge overlapping or adjacent spans in place; returns the new count
__device__ __forceinline__ int merge_spans(Span* s, int n) {
  sort_spans(s, n);
  int m = 0;
  for (int i = 0; i < n; ++i) {
    if (m > 0 && s[i].a <= s[m - 1].b + 1) {
      s[m - 1].b = max(s[m - 1].b, s[i].b);
    } else {
      s[m++] = s[i];
    }
  }
  return m;
}

// mask + reduce: block (polygon, tile of the group), threads over pixel rows
__global__ __launch_bounds__(THREADS) void polygon_rows_kernel(
    Canvas C, uint32_t G, const uint32_t* __restrict__ ring_off, const REdge* __restrict__ edges,
    const int32_t* __restrict__ bbox, unsigned long long* __restrict__ count,
    unsigned long long* __restrict__ sum, bool with_sum, unsigned int* __restrict__ overflow) {
  const uint32_t j = blockIdx.x, g = blockIdx.y;
  if (g >= G) return;
  const uint64_t tile = C.tile0 + g;
  const int64_t s = (int64_t)1 << C.k;
  const int64_t tx0 = (int64_t)((tile % C.tiles_per_side) << C.t);
  const int64_t ty0 = (int64_t)((tile / C.tiles_per_side) << C.t);
  const int64_t last = ((int64_t)1 << C.F) - 1;
  // pixel rows / columns the bounding box can touch (closed pixels)
  const int64_t bx0 = imax64(0, cdiv(bbox[4 * j + 0], s) - 1);
  const int64_t bx1 = imin64(last, fdiv(bbox[4 * j + 2], s));
  const int64_t by0 = imax64(0, cdiv(bbox[4 * j + 1], s) - 1);
  const int64_t by1 = imin64(last, fdiv(bbox[4 * j + 3], s));
  const int64_t r0 = max(by0, ty0), r1 = min(by1, ty0 + (int64_t)C.T - 1);
  if (r0 > r1 || bx1 < tx0 || bx0 > tx0 + (int64_t)C.T - 1) return;

  const uint32_t e0 = ring_off[j], ne = ring_off[j + 1] - e0;
  __shared__ REdge s_e[SMEM_EDGES];
  const bool staged = ne <= SMEM_EDGES;
  if (staged)
    for (uint32_t i = threadIdx.x; i < ne; i += THREADS) s_e[i] = edges[e0 + i];
  __syncthreads();
  const REdge* E = staged ? s_e : edges + e0;

  unsigned long long acc_c = 0, acc_s = 0;
  Span sp[MAXI];
  Rat cr[MAXI];
  const uint64_t gbase = (uint64_t)g * C.T * C.T;
  for (int64_t y = r0 + threadIdx.x; y <= r1; y += THREADS) {
    const int64_t Y0 = y * s, Y1 = Y0 + s;
    int n = 0, nc = 0;
    bool over = false;
    for (uint32_t i = 0; i < ne; ++i) {
      const REdge e = E[i];
      const int64_t lo = min(e.ay, e.by), hi = max(e.ay, e.by);
      if (hi < Y0 || lo > Y1) continue;  // misses the closed strip
      Rat xl, xr;
      if (e.ay == e.by) {
        xl = Rat{min(e.ax, e.bx), 1};
        xr = Rat{max(e.ax, e.bx), 1};
      } else {
        const Rat p = x_at(e, max(Y0, lo)), q = x_at(e, min(Y1, hi));
        const bool pq = rat_less(p, q);
        xl = pq ? p : q;
        xr = pq ? q : p;
      }
      // closed pixels m with m*s <= xr and (m+1)*s >= xl
      const int64_t m0 = imax64(0, cdiv(xl.n, xl.d * s) - 1);
      const int64_t m1 = imin64(last, fdiv(xr.n, xr.d * s));
      if (n == MAXI) {
        n = merge_spans(sp, n);
        if (n == MAXI) over = true;
      }
      if (!over && m0 <= m1) sp[n++] = Span{(int32_t)m0, (int32_t)m1};
      // crossing of the line y = Y0 (half-open)
      if ((e.ay > Y0) != (e.by > Y0)) {
        if (nc < MAXI)
          cr[nc++] = x_at(e, Y0);
        else
          over = true;
      }
    }
    // interior pixels: corners strictly between crossings 2i and 2i+1
    for (int i = 1; i < nc; ++i) {  // sort crossings
      const Rat v = cr[i];
      int q = i;
      while (q > 0 && rat_less(v, cr[q - 1])) {
        cr[q] = cr[q - 1];
        --q;
      }
      cr[q] = v;
    }
    for (int i = 0; i + 1 < nc; i += 2) {
      const int64_t m0 = imax64(0, fdiv(cr[i].n, cr[i].d * s) + 1);
      const int64_t m1 = imin64(last, cdiv(cr[i + 1].n, cr[i + 1].d * s) - 1);
      if (m0 > m1) continue;
      if (n == MAXI) {
        n = merge_spans(sp, n);
        if (n == MAXI) {
          over = true;
          break;
        }
      }
      sp[n++] = Span{(int32_t)m0, (int32_t)m1};
    }
    if (over) {
      atomicExch(overflow, 1u);
      continue;
    }
    n = merge_spans(sp, n);
    const unsigned long long* rc = C.cnt + gbase + (uint64_t)(y - ty0) * C.T;
    const unsigned long long* rs = C.sum + gbase + (uint64_t)(y - ty0) * C.T;
    for (int i = 0; i < n; ++i) {
      const int64_t a = imax64(sp[i].a, tx0), b = imin64(sp[i].b, tx0 + C.T - 1);
      if (a > b) continue;
      const int64_t la = a - tx0, lb = b - tx0;
      acc_c += rc[lb] - (la > 0 ? rc[la - 1] : 0ull);
      if (with_sum) acc_s += rs[lb] - (la > 0 ? rs[la - 1] : 0ull);
    }
  }
  // block reduction, one atomic per polygon and tile
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc_c += __shfl_xor_sync(0xffffffffu, acc_c, o);
    acc_s += __shfl_xor_sync(0xffffffffu, acc_s, o);
  }
  __shared__ unsigned long long rc_w[THREADS / 32], rs_w[THREADS / 32];
  if ((threadIdx.x & 31) == 0) {
    rc_w[threadIdx.x >> 5] = acc_c;
    rs_w[threadIdx.x >> 5] = acc_s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tc = 0, ts = 0;
    for (int i = 0; i < THREADS / 32; ++i) {
      tc += rc_w[i];
      ts += rs_w[i];
    }
    if (tc) atomicAdd(count + j, tc);
    if (with_sum && ts) atomicAdd(sum + j, ts);
  }
}

__global__ void raster_edges_kernel(const uint32_t* __restrict__ vx,
                                    const uint32_t* __restrict__ vy,
                                    const uint32_t* __restrict__ next, uint32_t V,
                                    REdge* __restrict__ edges) {
  const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  const uint32_t w = next[v];  // the following vertex of v's ring
  edges[v] = REdge{(int32_t)vx[v], (int32_t)vy[v], (int32_t)vx[w], (int32_t)vy[w]};
}

}  // namespace

sdb_status raster_join(const PolyEdges& pe, uint32_t B, uint32_t k, const uint32_t* x,
                       const uint32_t* y, const int32_t* attr, uint64_t n, uint32_t tile_bits,
                       uint64_t budget_bytes, uint64_t* count, int64_t* sum, cudaStream_t s) {
  const uint32_t P = pe.P, V = pe.V;
  const uint32_t F = B - k;
  const uint32_t t = F < tile_bits ? F : tile_bits;
  if (F - t > 8) {
    set_error("raster join: canvas of 4^%u pixels needs more than 2^16 tiles of 2^%u pixels a side",
              F, t);
    return SDB_EINVAL;
  }
  const uint64_t tps = 1ull << (F - t);  // tiles per side
  const uint64_t ntiles = tps * tps;
  const uint32_t T = 1u << t;
  const uint64_t tile_bytes = (uint64_t)T * T * 16;
  uint64_t G = budget_bytes / tile_bytes;
  if (G < 1) G = 1;
  if (G > ntiles) G = ntiles;
  if (G > 65535) G = 65535;
  Scratch sc(s);
  SDB_TRY_CUDA(cudaMemsetAsync(count, 0, (size_t)P * 8, s));
  if (sum) SDB_TRY_CUDA(cudaMemsetAsync(sum, 0, (size_t)P * 8, s));
  // polygons: edges and bounding boxes
  std::vector<int32_t> hb(4 * (size_t)P);
  for (uint32_t j = 0; j < P; ++j) {  // bounding box over all of j's rings
    int32_t x0 = INT32_MAX, y0 = INT32_MAX, x1 = 0, y1 = 0;
    for (uint32_t v = pe.edge_off[j]; v < pe.edge_off[j + 1]; ++v) {
      x0 = std::min<int32_t>(x0, (int32_t)pe.x[v]);
      y0 = std::min<int32_t>(y0, (int32_t)pe.y[v]);
      x1 = std::max<int32_t>(x1, (int32_t)pe.x[v]);
      y1 = std::max<int32_t>(y1, (int32_t)pe.y[v]);
    }
    hb[4 * j] = x0;
    hb[4 * j + 1] = y0;
    hb[4 * j + 2] = x1;
    hb[4 * j + 3] = y1;
  }
  uint32_t *d_off, *d_x, *d_y, *d_vp;
  int32_t* d_bb;
  REdge* d_e;
  unsigned int* d_over;
  SDB_TRY(sc.get(&d_off, P + 1));
  SDB_TRY(sc.get(&d_x, V));
  SDB_TRY(sc.get(&d_y, V));
  SDB_TRY(sc.get(&d_vp, V));
  SDB_TRY(sc.get(&d_bb, 4 * (size_t)P));
  SDB_TRY(sc.get(&d_e, V));
  SDB_TRY(sc.get(&d_over, 1));
  SDB_TRY_CUDA(cudaMemcpyAsync(d_off, pe.edge_off.data(), (P + 1) * 4ull, cudaMemcpyHostToDevice, s));
  SDB_TRY_CUDA(cudaMemcpyAsync(d_x, pe.x, V * 4ull, cudaMemcpyHostToDevice, s));
  SDB_TRY_CUDA(cudaMemcpyAsync(d_y, pe.y, V * 4ull, cudaMemcpyHostToDevice, s));
  SDB_TRY_CUDA(cudaMemcpyAsync(d_vp, pe.next.data(), V * 4ull, cudaMemcpyHostToDevice, s));
  SDB_TRY_CUDA(cudaMemcpyAsync(d_bb, hb.data(), hb.size() * 4, cudaMemcpyHostToDevice, s));
  SDB_TRY_CUDA(cudaMemsetAsync(d_over, 0, 4, s));
  raster_edges_kernel<<<grid_for(V, 256), 256, 0, s>>>(d_x, d_y, d_vp, V, d_e);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  // points bucketed by tile (one tile: no bucketing)
  const bool one = ntiles == 1;
  uint32_t* idx = nullptr;
  uint64_t* off = nullptr;
  if (!one && n > 0) {
    uint64_t *key, *ktmp, *ks;
    uint32_t *itmp, *is;
    SDB_TRY(sc.get(&key, n));
    SDB_TRY(sc.get(&ktmp, n));
    SDB_TRY(sc.get(&idx, n));
    SDB_TRY(sc.get(&itmp, n));
    tile_keys_kernel<<<grid_for(n, 256), 256, 0, s>>>(x, y, n, B, k, F, t, ntiles, key, idx);
    note_launch();
    SDB_TRY_CUDA(cudaGetLastError());
    SDB_TRY(radix_sort_pairs(key, idx, ktmp, itmp, n, 2 * (int)(F - t) + 1, s, &ks, &is));
    idx = is;
    SDB_TRY(sc.get(&off, ntiles + 1));
    tile_bounds_kernel<<<grid_for(ntiles + 1, 256), 256, 0, s>>>(ks, n, ntiles, off);
    note_launch();
    SDB_TRY_CUDA(cudaGetLastError());
  }
  Canvas C{};
  SDB_TRY(sc.get(&C.cnt, G * T * T));
  SDB_TRY(sc.get(&C.sum, G * T * T));
  C.T = T;
  C.t = t;
  C.F = F;
  C.k = k;
  C.B = B;
  C.tiles_per_side = tps;
  for (uint64_t t0 = 0; t0 < ntiles; t0 += G) {
    const uint32_t g = (uint32_t)std::min<uint64_t>(G, ntiles - t0);
    C.tile0 = t0;
    SDB_TRY_CUDA(cudaMemsetAsync(C.cnt, 0, (size_t)g * T * T * 8, s));
    if (sum) SDB_TRY_CUDA(cudaMemsetAsync(C.sum, 0, (size_t)g * T * T * 8, s));
    if (n > 0) {
      dim3 grid(std::max<unsigned>(1, (unsigned)std::min<uint64_t>(grid_for(n, 256), 4096 / g + 1)),
                g);
      blend_kernel<<<grid, 256, 0, s>>>(C, x, y, sum ? attr : nullptr, idx, off, g, one, n);
      note_launch();
      SDB_TRY_CUDA(cudaGetLastError());
    }
    row_prefix_kernel<<<g * T, THREADS, 0, s>>>(C, g * T);
    note_launch();
    SDB_TRY_CUDA(cudaGetLastError());
    polygon_rows_kernel<<<dim3(P, g), THREADS, 0, s>>>(
        C, g, d_off, d_e, d_bb, reinterpret_cast<unsigned long long*>(count),
        reinterpret_cast<unsigned long long*>(sum), sum != nullptr, d_over);
    note_launch();
    SDB_TRY_CUDA(cudaGetLastError());
  }
  unsigned int over = 0;
  SDB_TRY_CUDA(cudaMemcpyAsync(&over, d_over, 4, cudaMemcpyDeviceToHost, s));
  SDB_TRY_CUDA(cudaStreamSynchronize(s));
  if (over) {
    set_error("raster join: a polygon row needs more than %d spans or crossings", MAXI);
    return SDB_EINVAL;
  }
  return SDB_OK;
}

}  // namespace sdb
