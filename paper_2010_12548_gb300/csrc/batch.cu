// Batched level-of-detail queries over a resident point set.
//
// Users explore data at several levels of detail: an overview first, then
// zooms into regions of interest (Sec. 1, "Motivating Application").  A query
// here is an axis-aligned viewport, a subset of the polygons and a distance
// bound eps; it asks for COUNT and SUM per polygon of the subset over the
// points inside the viewport, answered from the eps-bounded covering (Sec. 2.2,
// Sec. 5.1).
//
//  * Points are made resident once, ordered by their full-resolution Hilbert
//    id, so a viewport is a handful of contiguous index ranges: the viewport is
//    cut into at most 9 x 9 aligned quadtree cells (side <= a quarter of the
//    viewport), each a contiguous id range, found by binary search.
//  * All queries' coverings are built in one level-synchronous pass over the
//    (query, polygon) pairs whose polygon can reach the viewport, cells clipped
//    to the viewport (cover.cu), which keeps them small at fine eps.
//  * The join is one persistent launch: blocks pull (query, point-tile) work
//    items from a device counter; per point the viewport test, the cell id at
//    the query's finest level, binary search in the query's ranges, and
//    per-slot COUNT/SUM in the query's output slice.  Alternatively one launch
//    per query, or the persistent launch replayed as a captured CUDA graph.
//  * Learned lookup (Sec. 3, learned index): each query covering with enough
//    ranges gets a two-level model, a linear root over the span of its range
//    starts (leaf = (h - lo) >> shift) and FP32 linear leaves fitted by least
//    squares with their maximum errors measured by the lookup's own arithmetic;
//    a point searches only its leaf's error window, the result is verified, and
//    binary search over the slice is the counted fallback.  The points of a
//    work item are Hilbert-ordered, so neighbouring lanes read the same leaf and
//    window lines.
//  * An autotuner picks the tile size and points per thread by timing the
//    candidates on the batch itself.
#include "hilbert.cuh"
#include "sdb_internal.cuh"

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

namespace sdb {
namespace {

constexpr uint32_t NONE = 0xffffffffu;
constexpr int THREADS = 256;
constexpr int MAXC = 81;  // candidate index ranges per query (9 x 9 cells)

using QueryDev = BatchQueryDev;
using ChunkDev = BatchChunkDev;
using TileRec = BatchTile;

// ---------------------------------------------------------------- points
__global__ void point_keys_kernel(const uint32_t* __restrict__ x, const uint32_t* __restrict__ y,
                                  uint64_t n, uint32_t B, uint32_t nsteps, uint32_t st0,
                                  uint64_t* __restrict__ key, uint32_t* __restrict__ idx,
                                  unsigned int* __restrict__ bad) {
  __shared__ uint32_t tab[HILBERT3_SMEM_WORDS];
  hilbert3_fill(tab);
  __syncthreads();
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t xi = x[i], yi = y[i];
    if (B < 32 && ((xi >> B) | (yi >> B))) *bad = 1u;
    key[i] = hilbert3_encode(xi, yi, nsteps, st0, tab);
    idx[i] = (uint32_t)i;
  }
}

__global__ void gather_points_kernel(const uint32_t* __restrict__ idx, uint64_t n,
                                     const uint32_t* __restrict__ x, const uint32_t* __restrict__ y,
                                     const int32_t* __restrict__ a, uint32_t* __restrict__ xs,
                                     uint32_t* __restrict__ ys, int32_t* __restrict__ as) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t j = idx[i];
  xs[i] = x[j];
  ys[i] = y[j];
  as[i] = a ? a[j] : 0;
}

// ---------------------------------------------------------------- candidates
// one thread per query: the viewport cut into aligned cells at most a quarter
// of its side, each cell a contiguous id range, turned into point index ranges
__global__ void candidates_kernel(const QueryDev* __restrict__ qd, uint32_t Q,
                                  const uint64_t* __restrict__ key, uint64_t n, uint32_t B,
                                  uint32_t* __restrict__ cand, uint32_t* __restrict__ ncand) {
  uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Q) return;
  const QueryDev Qd = qd[q];
  const uint32_t side = max(Qd.x1 - Qd.x0, Qd.y1 - Qd.y0);
  uint32_t lc = 0;  // log2 of the cell side
  while (lc < B && (2u << lc) <= max(1u, side / 4)) ++lc;
  const uint32_t L = B - lc;  // cell level
  uint32_t a[MAXC], b[MAXC];
  int m = 0;
  for (uint32_t cy = Qd.y0 >> lc; cy <= (Qd.y1 - 1) >> lc; ++cy)
    for (uint32_t cx = Qd.x0 >> lc; cx <= (Qd.x1 - 1) >> lc; ++cx) {
      const uint64_t h = hilbert_id(cx, cy, L);
      const uint64_t k0 = h << (2 * lc), k1 = (h + 1) << (2 * lc);
      uint64_t lo = 0, len = n;  // first index with key >= k0
      while (len > 0) {
        uint64_t half = len >> 1;
        if (key[lo + half] < k0) {
          lo += half + 1;
          len -= half + 1;
        } else {
          len = half;
        }
      }
      uint64_t hi = lo, len2 = n - lo;  // first index with key >= k1
      while (len2 > 0) {
        uint64_t half = len2 >> 1;
        if (key[hi + half] < k1) {
          hi += half + 1;
          len2 -= half + 1;
        } else {
          len2 = half;
        }
      }
      if (hi > lo && m < MAXC) {
        a[m] = (uint32_t)lo;
        b[m] = (uint32_t)hi;
        ++m;
      }
    }
  // sort by start, merge touching ranges
  for (int i = 1; i < m; ++i) {
    uint32_t va = a[i], vb = b[i];
    int j = i;
    while (j > 0 && a[j - 1] > va) {
      a[j] = a[j - 1];
      b[j] = b[j - 1];
      --j;
    }
    a[j] = va;
    b[j] = vb;
  }
  int w = 0;
  for (int i = 0; i < m; ++i) {
    if (w > 0 && a[i] <= b[w - 1]) {
      b[w - 1] = max(b[w - 1], b[i]);
    } else {
      a[w] = a[i];
      b[w] = b[i];
      ++w;
    }
  }
  for (int i = 0; i < w; ++i) {
    cand[(size_t)q * MAXC * 2 + 2 * i] = a[i];
    cand[(size_t)q * MAXC * 2 + 2 * i + 1] = b[i];
  }
  ncand[q] = (uint32_t)w;
}

__global__ void tile_count_kernel(const uint32_t* __restrict__ cand,
                                  const uint32_t* __restrict__ ncand, uint32_t Q, uint32_t T,
                                  uint64_t* __restrict__ ntile) {
  uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Q) return;
  uint64_t t = 0;
  for (uint32_t i = 0; i < ncand[q]; ++i) {
    const uint32_t a = cand[(size_t)q * MAXC * 2 + 2 * i], b = cand[(size_t)q * MAXC * 2 + 2 * i + 1];
    t += ((uint64_t)b - a + T - 1) / T;
  }
  ntile[q] = t;
}

__global__ void tile_fill_kernel(const uint32_t* __restrict__ cand,
                                 const uint32_t* __restrict__ ncand, uint32_t Q, uint32_t T,
                                 const uint64_t* __restrict__ toff, TileRec* __restrict__ tiles) {
  uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Q) return;
  uint64_t t = toff[q];
  for (uint32_t i = 0; i < ncand[q]; ++i) {
    const uint32_t a = cand[(size_t)q * MAXC * 2 + 2 * i], b = cand[(size_t)q * MAXC * 2 + 2 * i + 1];
    for (uint64_t s = a; s < b; s += T)
      tiles[t++] = TileRec{q, (uint32_t)s, (uint32_t)min((uint64_t)b, s + T), 0};
  }
}

// ---------------------------------------------------------------- join
struct BatchArgs {
  const uint32_t* x;
  const uint32_t* y;
  const int32_t* attr;
  const QueryDev* q;
  const TileRec* tiles;
  const ChunkDev* chunks;
  unsigned long long* count;
  unsigned long long* sum;
  const LeafRec* leaves;          // per-query learned leaves (queries with nleaves > 0)
  unsigned long long* fallbacks;  // learned searches that missed
};

// last r in [0, R) with st[r] <= h (st[R] is the slice's sentinel, above all ids)
__device__ __forceinline__ uint32_t slice_bs(const uint64_t* __restrict__ st, uint32_t R,
                                             uint64_t h) {
  uint32_t lo = 0;
  for (uint32_t len = R + 1; len > 1;) {
    const uint32_t half = len >> 1;
    if (__ldg(st + lo + half) <= h) lo += half;
    len -= half;
  }
  return lo;
}

// the range of id h in a query slice through its learned index: ids outside
// the leaves' span are the first or last range; else the leaf's prediction,
// a search of its error window (an end no probe has proven is read back), and
// binary search over the slice when the window does not bracket h (counted)
__device__ __forceinline__ uint32_t slice_learned(const uint64_t* __restrict__ st,
                                                  const QueryDev& Q, const LeafRec* leaves,
                                                  unsigned long long* fallbacks, uint64_t h) {
  if (h < Q.llo) return 0;
  if (h >= Q.lhi) return Q.R - 1;
  uint64_t l = (h - Q.llo) >> Q.lwshift;
  if (l >= Q.nleaves) l = Q.nleaves - 1;
  uint64_t w0, w1, w2, w3;
  asm("ld.global.nc.v4.u64 {%0, %1, %2, %3}, [%4];"
      : "=l"(w0), "=l"(w1), "=l"(w2), "=l"(w3)
      : "l"(leaves + Q.loff + l));
  LeafRec lr;
  lr.base = w0;
  lr.a = __uint_as_float((uint32_t)w1);
  lr.b = __uint_as_float((uint32_t)(w1 >> 32));
  lr.first = (uint32_t)w2;
  lr.last = (uint32_t)(w2 >> 32);
  lr.errlo = (int32_t)(uint32_t)w3;
  lr.errhi = (int32_t)(uint32_t)(w3 >> 32);
  const int64_t pr = leaf_predict(lr, h);
  int64_t a = pr - lr.errlo, b = pr + lr.errhi;
  if (a < (int64_t)lr.first) a = lr.first;
  if (b > (int64_t)lr.last) b = lr.last;
  if (b < a) b = a;
  uint32_t lo = (uint32_t)a, len = (uint32_t)(b - a + 1), known = 0;
  while (len > 1) {
    const uint32_t half = len >> 1;
    if (__ldg(st + lo + half) <= h) {
      lo += half;
      known |= 1u;
    } else {
      known |= 2u;
    }
    len -= half;
  }
  const bool ok0 = (known & 1u) || __ldg(st + lo) <= h;
  const bool ok1 = (known & 2u) || h < __ldg(st + lo + 1);
  if (ok0 && ok1) return lo;
  atomicAdd(fallbacks, 1ull);
  return slice_bs(st, Q.R, h);
}

// Per-block accumulators of a work item's query slots in shared memory (when
// the query has at most BATCH_SMEM_SLOTS slots): a count and the attribute
// split exactly into its low 16 bits and the rest; a work item holds at most
// 2^16 points, so none can wrap (2^16 * 65535 < 2^32, 2^16 * 2^15 <= 2^31), and
// the item's totals go to the outputs with one global atomic each.
constexpr uint32_t BATCH_SMEM_SLOTS = 2048;
constexpr uint32_t BATCH_MAX_TILE = 1u << 16;

__device__ __forceinline__ void add_slot(const BatchArgs& A, uint32_t out, uint32_t p, int32_t a,
                                         bool sum, uint32_t* s_acc, uint32_t ns) {
  if (s_acc) {
    atomicAdd(&s_acc[p], 1u);
    if (sum) {
      atomicAdd(&s_acc[ns + p], (uint32_t)a & 0xffffu);
      atomicAdd(reinterpret_cast<int32_t*>(&s_acc[2 * ns + p]), a >> 16);
    }
    return;
  }
  atomicAdd(&A.count[out + p], 1ull);
  if (sum) atomicAdd(&A.sum[out + p], (unsigned long long)(long long)a);
}

template <int G, bool SUM>
__global__ __launch_bounds__(THREADS) void batch_kernel(BatchArgs A, uint32_t tile_lo,
                                                        uint32_t tile_hi,
                                                        unsigned long long* head) {
  __shared__ uint32_t tab[HILBERT3_SMEM_WORDS];
  __shared__ uint32_t s_tile;
  extern __shared__ uint32_t s_slots[];  // (SUM ? 3 : 1) * BATCH_SMEM_SLOTS words
  hilbert3_fill(tab);
  __syncthreads();
  for (;;) {
    if (threadIdx.x == 0) s_tile = tile_lo + (uint32_t)atomicAdd(head, 1ull);
    __syncthreads();
    const uint32_t t = s_tile;
    __syncthreads();
    if (t >= tile_hi) break;
    const TileRec tr = A.tiles[t];
    const QueryDev Q = A.q[tr.q];
    const ChunkDev C = A.chunks[Q.chunk];
    // block-uniform: the work item's query decides where its sums gather
    const uint32_t ns = Q.npoly;
    uint32_t* s_acc = (ns <= BATCH_SMEM_SLOTS && tr.end - tr.begin <= BATCH_MAX_TILE) ? s_slots
                                                                                      : nullptr;
    if (s_acc) {
      for (uint32_t i = threadIdx.x; i < (SUM ? 3 : 1) * ns; i += THREADS) s_acc[i] = 0;
      __syncthreads();
    }
    for (uint32_t i0 = tr.begin + threadIdx.x * G; i0 < tr.end; i0 += THREADS * G) {
      uint64_t h[G];
      bool ok[G];
      int32_t av[G];
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const uint32_t i = i0 + g;
        ok[g] = i < tr.end;
        const uint32_t x = ok[g] ? A.x[i] : 0u, y = ok[g] ? A.y[i] : 0u;
        av[g] = (SUM && ok[g]) ? A.attr[i] : 0;
        ok[g] = ok[g] && x >= Q.x0 && x < Q.x1 && y >= Q.y0 && y < Q.y1;
        h[g] = ok[g] ? hilbert3_encode(x >> Q.k, y >> Q.k, Q.nsteps, Q.st0, tab) : 0ull;
      }
      // last entry r in [0, R) of the slice with start <= h (sentinel above)
      uint32_t lo[G];
#pragma unroll
      for (int g = 0; g < G; ++g) lo[g] = 0;
      if (Q.nleaves) {  // block-uniform: every point of the work item is in query Q
#pragma unroll
        for (int g = 0; g < G; ++g)
          if (ok[g]) lo[g] = slice_learned(C.start + Q.sbase, Q, A.leaves, A.fallbacks, h[g]);
      } else {
        for (uint32_t len = Q.R + 1; len > 1;) {
          const uint32_t half = len >> 1;
          uint64_t v[G];
#pragma unroll
          for (int g = 0; g < G; ++g) v[g] = __ldg(C.start + Q.sbase + lo[g] + half);
#pragma unroll
          for (int g = 0; g < G; ++g)
            if (v[g] <= h[g]) lo[g] += half;
          len -= half;
        }
      }
#pragma unroll
      for (int g = 0; g < G; ++g) {
        if (!ok[g]) continue;
        const uint64_t e = Q.sbase + lo[g];
        const uint32_t p = __ldg(C.pay + e);
        if (p < 0x80000000u) {
          add_slot(A, Q.out_off, p, av[g], SUM, s_acc, ns);
        } else if (p != NONE) {
          const uint32_t rr = p & 0x7fffffffu;
          const uint32_t b = __ldg(C.list_off + rr), en = __ldg(C.list_off + rr + 1);
          for (uint32_t j = b; j < en; ++j)
            add_slot(A, Q.out_off, __ldg(C.list_ids + j), av[g], SUM, s_acc, ns);
        }
      }
    }
    if (s_acc) {  // the work item's totals into the query's output slots
      __syncthreads();
      for (uint32_t i = threadIdx.x; i < ns; i += THREADS) {
        const uint32_t c = s_acc[i];
        if (!c) continue;
        atomicAdd(&A.count[Q.out_off + i], (unsigned long long)c);
        if (SUM) {
          const long long tot =
              (long long)reinterpret_cast<const int32_t*>(s_acc)[2 * ns + i] * 65536 +
              (long long)s_acc[ns + i];
          atomicAdd(&A.sum[Q.out_off + i], (unsigned long long)tot);
        }
      }
    }
  }
}

// ---------------------------------------------------------------- learned index
// per query with leaves: the span [llo, lhi) of ids between its second range
// start and one past its last range start
__global__ void slice_span_kernel(const QueryDev* __restrict__ qd, uint32_t Q,
                                  const ChunkDev* __restrict__ chunks, uint32_t min_ranges,
                                  uint64_t* __restrict__ span) {
  const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Q) return;
  const QueryDev d = qd[q];
  if (d.R < 2 || d.R < min_ranges) {
    span[2 * q] = span[2 * q + 1] = 0;
    return;
  }
  const uint64_t* st = chunks[d.chunk].start + d.sbase;
  span[2 * q] = st[1];
  span[2 * q + 1] = st[d.R - 1] + 1;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ long long warp_max_ll(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long t = __shfl_xor_sync(0xffffffffu, v, o);
    v = t > v ? t : v;
  }
  return v;
}

// one warp per leaf: leaf l of query q receives the ids [base, end), base =
// llo + (l << shift), end = base + 2^shift (the last leaf ends at lhi); its
// ranges are first .. last (local indices: the ranges holding base and end - 1).
// Least squares of the local index on the leaf-relative start (FP32, centred),
// then the largest prediction errors below and above over every id the leaf
// receives, from the lookup's own arithmetic at the two ends of each range's
// part of the leaf (the prediction is monotone in h).
__global__ void batch_leaf_fit_kernel(const QueryDev* __restrict__ qd,
                                      const ChunkDev* __restrict__ chunks,
                                      const uint32_t* __restrict__ leaf_q, uint64_t total,
                                      LeafRec* __restrict__ leaves) {
  const uint64_t g = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= total) return;
  const QueryDev Q = qd[leaf_q[g]];
  const uint64_t l = g - Q.loff;
  const uint64_t* st = chunks[Q.chunk].start + Q.sbase;
  const uint64_t b0 = Q.llo + (l << Q.lwshift);
  uint64_t b1 = l + 1 == Q.nleaves ? Q.lhi : b0 + (1ull << Q.lwshift);
  if (b1 > Q.lhi) b1 = Q.lhi;
  const uint32_t first = slice_bs(st, Q.R, b0), last = slice_bs(st, Q.R, b1 - 1);
  LeafRec lr;
  lr.base = b0;
  lr.first = first;
  lr.last = last;
  const uint32_t n = last - first + 1;
  float sx = 0.f, sy = 0.f;
  for (uint32_t i = first + lane; i <= last; i += 32) {
    const uint64_t v = st[i] > b0 ? st[i] : b0;
    sx += __ull2float_rn(v - b0);
    sy += (float)(i - first);
  }
  const float inv_n = 1.0f / (float)n;
  const float mx = warp_sum_f(sx) * inv_n, my = warp_sum_f(sy) * inv_n;
  float sxx = 0.f, sxy = 0.f;
  for (uint32_t i = first + lane; i <= last; i += 32) {
    const uint64_t v = st[i] > b0 ? st[i] : b0;
    const float dx = __ull2float_rn(v - b0) - mx, dy = (float)(i - first) - my;
    sxx = fmaf(dx, dx, sxx);
    sxy = fmaf(dx, dy, sxy);
  }
  sxx = warp_sum_f(sxx);
  sxy = warp_sum_f(sxy);
  const float slope = (sxx > 0.f && sxy > 0.f) ? sxy / sxx : 0.f;
  lr.a = slope;
  lr.b = my - slope * mx;
  lr.errlo = 0;
  lr.errhi = 0;
  long long ehi = 0, elo = 0;
  for (uint32_t i = first + lane; i <= last; i += 32) {
    const uint64_t lo_h = st[i] > b0 ? st[i] : b0;
    const uint64_t hi_h = (st[i + 1] < b1 ? st[i + 1] : b1) - 1;
    const long long plo = (long long)leaf_predict(lr, lo_h);
    const long long phi = (long long)leaf_predict(lr, hi_h);
    const long long up = (long long)i - plo, dn = phi - (long long)i;
    ehi = up > ehi ? up : ehi;
    elo = dn > elo ? dn : elo;
  }
  ehi = warp_max_ll(ehi);
  elo = warp_max_ll(elo);
  const long long CAP = 1ll << 30;
  lr.errhi = (int32_t)(ehi > CAP ? CAP : ehi);
  lr.errlo = (int32_t)(elo > CAP ? CAP : elo);
  if (lane == 0) leaves[g] = lr;
}

}  // namespace
}  // namespace sdb

struct sdb_batch {
  int device = 0;
  uint32_t NP = 0;
  sdb::BatchCore core;
  std::vector<sdb::CoverSet> cs;  // one per chunk of queries
  uint64_t n_ranges = 0, n_cells = 0, max_ranges = 0;
  cudaGraphExec_t graph = nullptr;
  void* g_count = nullptr;
  void* g_sum = nullptr;
};

namespace sdb {
namespace {

template <int G, bool SUM>
sdb_status launch_batch_t(const BatchArgs& A, uint32_t lo, uint32_t hi,
                          unsigned long long* head, cudaStream_t s) {
  auto kern = batch_kernel<G, SUM>;
  const size_t smem = (size_t)(SUM ? 3 : 1) * BATCH_SMEM_SLOTS * 4;
  int per_sm = 0;
  SDB_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, smem));
  uint64_t blocks = (uint64_t)num_sms() * (per_sm > 0 ? per_sm : 1);
  if (blocks > hi - lo) blocks = hi - lo;
  if (blocks == 0) return SDB_OK;
  kern<<<(unsigned)blocks, THREADS, smem, s>>>(A, lo, hi, head);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  return SDB_OK;
}

sdb_status launch_batch(const BatchArgs& A, uint32_t ppt, bool sum, uint32_t lo, uint32_t hi,
                        unsigned long long* head, cudaStream_t s) {
  if (ppt == 1) return sum ? launch_batch_t<1, true>(A, lo, hi, head, s)
                           : launch_batch_t<1, false>(A, lo, hi, head, s);
  if (ppt == 2) return sum ? launch_batch_t<2, true>(A, lo, hi, head, s)
                           : launch_batch_t<2, false>(A, lo, hi, head, s);
  return sum ? launch_batch_t<4, true>(A, lo, hi, head, s)
             : launch_batch_t<4, false>(A, lo, hi, head, s);
}

bool valid_device(int dev) {
  int cur = -1;
  return cudaGetDevice(&cur) == cudaSuccess && cur == dev;
}

sdb_status status_of(cudaError_t e, const char* what) {
  return e == cudaSuccess ? SDB_OK : cuda_status(e, what, __FILE__, __LINE__);
}

}  // namespace

void BatchCore::release(cudaStream_t s) {
  dfree(leaves, s);
  dfree(fallbacks, s);
  leaves = nullptr;
  fallbacks = nullptr;
  dfree(dq, s);
  dfree(dchunks, s);
  dfree(cand, s);
  dfree(ncand, s);
  dfree(tiles, s);
  dfree(heads, s);
  dq = nullptr;
  dchunks = nullptr;
  cand = nullptr;
  ncand = nullptr;
  tiles = nullptr;
  heads = nullptr;
}

sdb_status batch_query_dev(uint32_t B, const sdb_query& Qu, uint64_t out_off, BatchQueryDev* d,
                           uint32_t* F_out) {
  uint32_t k = 0, F = 0;
  SDB_TRY(sdb_finest_level(B, Qu.eps, &k, &F));
  const uint32_t G = 1u << B;
  if (!(Qu.x0 < Qu.x1 && Qu.y0 < Qu.y1 && Qu.x1 <= G && Qu.y1 <= G)) {
    set_error("viewport must be non-empty and inside the grid");
    return SDB_EINVAL;
  }
  memset(d, 0, sizeof(*d));
  d->k = k;
  hilbert3_params(F, &d->nsteps, &d->st0);
  d->x0 = Qu.x0;
  d->y0 = Qu.y0;
  d->x1 = Qu.x1;
  d->y1 = Qu.y1;
  d->out_off = (uint32_t)out_off;
  d->npoly = Qu.poly_cnt;
  *F_out = F;
  return SDB_OK;
}

sdb_status batch_core_tiles(BatchCore* c, uint32_t T, cudaStream_t s) {
  Scratch sc(s);
  uint64_t *nt, *toff, *dtot;
  SDB_TRY(sc.get(&nt, c->Q));
  SDB_TRY(sc.get(&toff, (size_t)c->Q + 1));
  SDB_TRY(sc.get(&dtot, 1));
  tile_count_kernel<<<grid_for(c->Q, 128), 128, 0, s>>>(c->cand, c->ncand, c->Q, T, nt);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  SDB_TRY(exclusive_scan<uint64_t>(nt, toff, c->Q, dtot, s));
  SDB_TRY_CUDA(cudaMemcpyAsync(toff + c->Q, dtot, 8, cudaMemcpyDeviceToDevice, s));
  c->qtile.assign((size_t)c->Q + 1, 0);
  SDB_TRY_CUDA(cudaMemcpyAsync(c->qtile.data(), toff, ((size_t)c->Q + 1) * 8,
                               cudaMemcpyDeviceToHost, s));
  SDB_TRY_CUDA(cudaStreamSynchronize(s));
  const uint64_t total = c->qtile[c->Q];
  if (total >= 0xffffffffull) {
    set_error("batch: %llu tiles exceed the 32-bit range", (unsigned long long)total);
    return SDB_EINVAL;
  }
  if (c->tiles) dfree(c->tiles, s);
  c->tiles = nullptr;
  SDB_TRY(dalloc_n(&c->tiles, total, s));
  tile_fill_kernel<<<grid_for(c->Q, 128), 128, 0, s>>>(c->cand, c->ncand, c->Q, T, toff, c->tiles);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  SDB_TRY_CUDA(cudaStreamSynchronize(s));
  c->ntiles = total;
  c->tile = T;
  return SDB_OK;
}

sdb_status batch_core_prepare(BatchCore* c, cudaStream_t s) {
  const uint32_t Q = c->Q;
  SDB_TRY(dalloc_n(&c->dq, Q, s));
  SDB_TRY(dalloc_n(&c->dchunks, c->hchunks.size(), s));
  SDB_TRY(dalloc_n(&c->cand, (size_t)Q * MAXC * 2, s));
  SDB_TRY(dalloc_n(&c->ncand, Q, s));
  SDB_TRY(dalloc_n(&c->heads, (size_t)Q + 1, s));
  SDB_TRY_CUDA(cudaMemcpyAsync(c->dq, c->hq.data(), Q * sizeof(BatchQueryDev),
                               cudaMemcpyHostToDevice, s));
  if (!c->hchunks.empty())
    SDB_TRY_CUDA(cudaMemcpyAsync(c->dchunks, c->hchunks.data(),
                                 c->hchunks.size() * sizeof(BatchChunkDev), cudaMemcpyHostToDevice,
                                 s));
  candidates_kernel<<<grid_for(Q, 64), 64, 0, s>>>(c->dq, Q, c->pts->key, c->pts->n, c->pts->B,
                                                   c->cand, c->ncand);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  SDB_TRY(batch_core_tiles(c, c->tile, s));
  // candidate points (for reporting)
  std::vector<uint32_t> hc((size_t)Q * MAXC * 2), hn(Q);
  SDB_TRY_CUDA(cudaMemcpyAsync(hc.data(), c->cand, hc.size() * 4, cudaMemcpyDeviceToHost, s));
  SDB_TRY_CUDA(cudaMemcpyAsync(hn.data(), c->ncand, hn.size() * 4, cudaMemcpyDeviceToHost, s));
  SDB_TRY_CUDA(cudaStreamSynchronize(s));
  c->candidates = 0;
  for (uint32_t q = 0; q < Q; ++q)
    for (uint32_t i = 0; i < hn[q]; ++i)
      c->candidates += hc[(size_t)q * MAXC * 2 + 2 * i + 1] - hc[(size_t)q * MAXC * 2 + 2 * i];
  return SDB_OK;
}

sdb_status batch_core_index(BatchCore* c, uint32_t min_ranges, uint32_t ranges_per_leaf,
                            cudaStream_t s) {
  const uint32_t Q = c->Q;
  dfree(c->leaves, s);
  c->leaves = nullptr;
  c->nleaves = 0;
  c->indexed = 0;
  c->learned = min_ranges > 0;
  for (auto& d : c->hq) d.nleaves = d.loff = d.lwshift = 0, d.llo = d.lhi = 0;
  if (c->learned) {
    if (ranges_per_leaf == 0) ranges_per_leaf = 1;
    Scratch sc(s);
    uint64_t* dspan;
    SDB_TRY(sc.get(&dspan, (size_t)Q * 2));
    slice_span_kernel<<<grid_for(Q, 128), 128, 0, s>>>(c->dq, Q, c->dchunks, min_ranges, dspan);
    note_launch();
    SDB_TRY_CUDA(cudaGetLastError());
    std::vector<uint64_t> span((size_t)Q * 2);
    SDB_TRY_CUDA(cudaMemcpyAsync(span.data(), dspan, span.size() * 8, cudaMemcpyDeviceToHost, s));
    SDB_TRY_CUDA(cudaStreamSynchronize(s));
    std::vector<uint32_t> leaf_q;
    uint64_t total = 0;
    for (uint32_t q = 0; q < Q; ++q) {
      BatchQueryDev& d = c->hq[q];
      const uint64_t lo = span[2 * q], hi = span[2 * q + 1];
      if (hi <= lo) continue;  // too few ranges: binary search
      // leaves for about ranges_per_leaf ranges each, a power of two in 16 .. 2^16
      uint64_t want = 16;
      while (want < 65536 && want * ranges_per_leaf < d.R) want *= 2;
      const uint64_t sp = hi - lo;
      uint32_t ws = 0;
      while (((sp + (1ull << ws) - 1) >> ws) > want) ++ws;
      const uint64_t L = (sp + (1ull << ws) - 1) >> ws;
      d.nleaves = (uint32_t)L;
      d.lwshift = ws;
      d.loff = (uint32_t)total;
      d.llo = lo;
      d.lhi = hi;
      total += L;
      if (total >= 0xffffffffull) {
        set_error("batch learned index: %llu leaves exceed the 32-bit range",
                  (unsigned long long)total);
        return SDB_EINVAL;
      }
      leaf_q.insert(leaf_q.end(), (size_t)L, q);
      ++c->indexed;
    }
    if (total) {
      uint32_t* dlq;
      SDB_TRY(sc.get(&dlq, total));
      SDB_TRY(dalloc_n(&c->leaves, total, s));
      if (reinterpret_cast<uintptr_t>(c->leaves) & 31u) {  // leaves are read 32 bytes at once
        set_error("batch learned index: leaf records not 32-byte aligned");
        return SDB_ECUDA;
      }
      SDB_TRY_CUDA(cudaMemcpyAsync(dlq, leaf_q.data(), total * 4, cudaMemcpyHostToDevice, s));
      SDB_TRY_CUDA(cudaMemcpyAsync(c->dq, c->hq.data(), Q * sizeof(BatchQueryDev),
                                   cudaMemcpyHostToDevice, s));
      batch_leaf_fit_kernel<<<grid_for(total * 32, 256), 256, 0, s>>>(c->dq, c->dchunks, dlq,
                                                                      total, c->leaves);
      note_launch();
      SDB_TRY_CUDA(cudaGetLastError());
      SDB_TRY_CUDA(cudaStreamSynchronize(s));
    }
    c->nleaves = total;
    if (!c->fallbacks) {
      SDB_TRY(dalloc_n(&c->fallbacks, 1, s));
      SDB_TRY_CUDA(cudaMemsetAsync(c->fallbacks, 0, sizeof(unsigned long long), s));
    }
  }
  SDB_TRY_CUDA(cudaMemcpyAsync(c->dq, c->hq.data(), Q * sizeof(BatchQueryDev),
                               cudaMemcpyHostToDevice, s));
  SDB_TRY_CUDA(cudaStreamSynchronize(s));
  return SDB_OK;
}

sdb_status batch_core_run(BatchCore* c, int mode, uint64_t* count, int64_t* sum, cudaStream_t s) {
  BatchArgs A;
  A.leaves = c->leaves;
  A.fallbacks = c->fallbacks;
  if (c->fallbacks)
    SDB_TRY_CUDA(cudaMemsetAsync(c->fallbacks, 0, sizeof(unsigned long long), s));
  A.x = c->pts->x;
  A.y = c->pts->y;
  A.attr = c->pts->attr;
  A.q = c->dq;
  A.tiles = c->tiles;
  A.chunks = c->dchunks;
  A.count = reinterpret_cast<unsigned long long*>(count);
  A.sum = reinterpret_cast<unsigned long long*>(sum);
  if (c->out_len) {
    SDB_TRY_CUDA(cudaMemsetAsync(count, 0, c->out_len * 8, s));
    if (sum) SDB_TRY_CUDA(cudaMemsetAsync(sum, 0, c->out_len * 8, s));
  }
  if (mode == SDB_BATCH_PER_QUERY) {
    SDB_TRY_CUDA(cudaMemsetAsync(c->heads, 0, (size_t)c->Q * sizeof(unsigned long long), s));
    for (uint32_t q = 0; q < c->Q; ++q)
      if (c->qtile[q + 1] > c->qtile[q])
        SDB_TRY(launch_batch(A, c->ppt, sum != nullptr, (uint32_t)c->qtile[q],
                             (uint32_t)c->qtile[q + 1], c->heads + q, s));
    return SDB_OK;
  }
  SDB_TRY_CUDA(cudaMemsetAsync(c->heads + c->Q, 0, sizeof(unsigned long long), s));
  return launch_batch(A, c->ppt, sum != nullptr, 0, (uint32_t)c->ntiles, c->heads + c->Q, s);
}

// Coverings of queries [q0, q0 + nq) of a pair list, built in chunks that are
// halved and retried when they overflow the builder's 32-bit ranges or memory.
// Appends CoverSets to *sets and fills sbase/R/chunk of hq.
sdb_status build_query_coverings(const PolyEdges& pe, uint32_t B,
                                 const std::vector<CoverQuery>& cq,
                                 const std::vector<uint32_t>& pp, const std::vector<uint32_t>& pq,
                                 const std::vector<uint32_t>& ps, std::vector<BatchQueryDev>& hq,
                                 std::vector<CoverSet>* sets, uint32_t chunk_base,
                                 cudaStream_t s, uint64_t* n_ranges, uint64_t* n_cells,
                                 uint64_t* max_ranges) {
  const uint32_t Q = (uint32_t)cq.size();
  std::vector<uint64_t> pfirst((size_t)Q + 1, 0);  // pairs are in query order
  for (uint64_t i = 0, q = 0; q <= Q; ++q) {
    while (i < pq.size() && pq[i] < q) ++i;
    pfirst[q] = i;
  }
  uint32_t chunk_q = 512;
  std::vector<uint32_t> pq_local;
  for (uint32_t q0 = 0; q0 < Q;) {
    // queries of a chunk share 64-bit keys: query bits above 2 * (finest level)
    uint32_t nq = std::min(chunk_q, Q - q0);
    for (;;) {
      uint32_t Fm = 0;
      for (uint32_t q = q0; q < q0 + nq; ++q) Fm = std::max(Fm, cq[q].F);
      const uint32_t room = 64 - 2 * Fm;  // F <= 30
      if (nq == 1 || room >= 32 || nq <= (1u << room)) break;
      nq = 1u << room;
    }
    const uint64_t pa = pfirst[q0], pb = pfirst[q0 + nq];
    pq_local.assign(pq.begin() + pa, pq.begin() + pb);
    for (auto& v : pq_local) v -= q0;
    CoverSpec spec;
    spec.B = B;
    spec.Q = nq;
    spec.q = cq.data() + q0;
    spec.NP = (uint32_t)(pb - pa);
    spec.pair_poly = pp.data() + pa;
    spec.pair_query = pq_local.data();
    spec.pair_slot = ps.data() + pa;
    CoverSet set;
    sdb_status st = build_coverings(pe, spec, s, &set);
    if (st == SDB_ENOMEM && nq > 1) {
      set.release(s);
      cudaStreamSynchronize(s);
      cudaGetLastError();
      chunk_q = nq / 2;
      continue;
    }
    if (st != SDB_OK) {
      set.release(s);
      return st;
    }
    for (uint32_t q = 0; q < nq; ++q) {
      BatchQueryDev& d = hq[q0 + q];
      d.sbase = set.qoff[q];
      d.R = (uint32_t)(set.qoff[q + 1] - set.qoff[q] - 1);
      d.chunk = chunk_base + (uint32_t)sets->size();
      *max_ranges = std::max<uint64_t>(*max_ranges, d.R);
    }
    *n_ranges += set.E - nq;
    *n_cells += set.ncells;
    sets->push_back(set);
    q0 += nq;
  }
  return SDB_OK;
}

// (query, polygon) pairs whose polygon's cells can hold viewport points: the
// polygon's bounding box grown by one finest cell meets the viewport
void viewport_pairs(const std::vector<uint32_t>& bb, uint32_t q, const sdb_query& Qu, uint32_t k,
                    const uint32_t* ids, std::vector<uint32_t>& pp, std::vector<uint32_t>& pq,
                    std::vector<uint32_t>& ps) {
  const int64_t g = (int64_t)1 << k;
  for (uint32_t t = 0; t < Qu.poly_cnt; ++t) {
    const uint32_t j = ids[t];
    if ((int64_t)bb[4 * j] - g < (int64_t)Qu.x1 && (int64_t)bb[4 * j + 2] + g >= Qu.x0 &&
        (int64_t)bb[4 * j + 1] - g < (int64_t)Qu.y1 && (int64_t)bb[4 * j + 3] + g >= Qu.y0) {
      pp.push_back(j);
      pq.push_back(q);
      ps.push_back(t);
    }
  }
}

sdb_status polygon_bboxes(const sdb_polygons* polys, uint32_t B, std::vector<uint32_t>* bb) {
  const uint32_t P = polys->n_polygons, G = 1u << B;
  if (P == 0 || P >= (1u << 26) || polys->ring_off[0] != 0) {
    set_error("bad polygon set");
    return SDB_EINVAL;
  }
  bb->assign(4ull * P, 0);
  for (uint32_t j = 0; j < P; ++j) {
    if (polys->ring_off[j + 1] < polys->ring_off[j] + 3) {
      set_error("polygon %u has fewer than 3 vertices", j);
      return SDB_EINVAL;
    }
    uint32_t mnx = ~0u, mny = ~0u, mxx = 0, mxy = 0;
    for (uint32_t v = polys->ring_off[j]; v < polys->ring_off[j + 1]; ++v) {
      if (polys->x[v] >= G || polys->y[v] >= G) {
        set_error("vertex %u outside the grid", v);
        return SDB_EINVAL;
      }
      mnx = std::min(mnx, polys->x[v]);
      mxx = std::max(mxx, polys->x[v]);
      mny = std::min(mny, polys->y[v]);
      mxy = std::max(mxy, polys->y[v]);
    }
    (*bb)[4 * j] = mnx;
    (*bb)[4 * j + 1] = mny;
    (*bb)[4 * j + 2] = mxx;
    (*bb)[4 * j + 3] = mxy;
  }
  return SDB_OK;
}

}  // namespace sdb

using namespace sdb;

extern "C" {

sdb_status sdb_points_create(const uint32_t* d_x, const uint32_t* d_y, const int32_t* d_attr,
                             uint64_t n, uint32_t grid_bits, void* cuda_stream, sdb_points** out) {
  if (!out) {
    set_error("out is NULL");
    return SDB_EINVAL;
  }
  *out = nullptr;
  if (grid_bits < 1 || grid_bits > 30) {
    set_error("grid_bits %u outside 1..30", grid_bits);
    return SDB_EINVAL;
  }
  if (n == 0 || n >= 0xffffffffull || !d_x || !d_y) {
    set_error("need 1 <= n < 2^32 points with coordinates");
    return SDB_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  sdb_points* p = new (std::nothrow) sdb_points();
  if (!p) {
    set_error("host allocation failed");
    return SDB_ENOMEM;
  }
  cudaGetDevice(&p->device);
  p->B = grid_bits;
  p->n = n;
  sdb_status st = SDB_OK;
  {
    Scratch sc(s);
    uint64_t* ktmp = nullptr;
    uint32_t *idx = nullptr, *itmp = nullptr;
    unsigned int* bad = nullptr;
    uint64_t* ks = nullptr;
    uint32_t* is = nullptr;
    st = dalloc_n(&p->key, n, s);
    if (st == SDB_OK) st = dalloc_n(&p->x, n, s);
    if (st == SDB_OK) st = dalloc_n(&p->y, n, s);
    if (st == SDB_OK) st = dalloc_n(&p->attr, n, s);
    if (st == SDB_OK) st = sc.get(&ktmp, n);
    if (st == SDB_OK) st = sc.get(&idx, n);
    if (st == SDB_OK) st = sc.get(&itmp, n);
    if (st == SDB_OK) st = sc.get(&bad, 1);
    if (st == SDB_OK) st = status_of(cudaMemsetAsync(bad, 0, 4, s), "memset");
    if (st == SDB_OK) {
      uint32_t nsteps, st0;
      hilbert3_params(grid_bits, &nsteps, &st0);
      point_keys_kernel<<<num_sms() * 8, 256, 0, s>>>(d_x, d_y, n, grid_bits, nsteps, st0, p->key,
                                                      idx, bad);
      note_launch();
      st = status_of(cudaGetLastError(), "point keys");
    }
    if (st == SDB_OK) st = radix_sort_pairs(p->key, idx, ktmp, itmp, n, 2 * grid_bits, s, &ks, &is);
    if (st == SDB_OK && ks != p->key)
      st = status_of(cudaMemcpyAsync(p->key, ks, n * 8, cudaMemcpyDeviceToDevice, s), "key copy");
    if (st == SDB_OK) {
      gather_points_kernel<<<grid_for(n, 256), 256, 0, s>>>(is, n, d_x, d_y, d_attr, p->x, p->y,
                                                            p->attr);
      note_launch();
      unsigned int hb = 0;
      st = status_of(cudaMemcpyAsync(&hb, bad, 4, cudaMemcpyDeviceToHost, s), "flag copy");
      if (st == SDB_OK) st = status_of(cudaStreamSynchronize(s), "points create");
      if (st == SDB_OK && hb) {
        set_error("a point lies outside the grid [0, 2^%u)", grid_bits);
        st = SDB_EINVAL;
      }
    }
  }
  if (st != SDB_OK) {
    sdb_points_free(p);
    return st;
  }
  *out = p;
  return SDB_OK;
}

void sdb_points_free(sdb_points* p) {
  if (!p) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(p->device);
  cudaDeviceSynchronize();
  sdb::release_point_index(p, 0);
  void* ps[] = {p->key, p->x, p->y, p->attr};
  for (void* q : ps)
    if (q) cudaFreeAsync(q, 0);
  cudaStreamSynchronize(0);
  cudaSetDevice(prev);
  delete p;
}

sdb_status sdb_batch_create(const sdb_points* pts, const sdb_polygons* polys,
                            const sdb_query* queries, uint32_t n_queries,
                            const uint32_t* subset_ids, uint64_t n_subset_ids, void* cuda_stream,
                            sdb_batch** out) {
  if (!out || !pts || !polys || !queries || n_queries == 0 || !polys->ring_off || !polys->x ||
      !polys->y) {
    set_error("points, polygons, queries and out are required");
    return SDB_EINVAL;
  }
  *out = nullptr;
  if (!valid_device(pts->device)) {
    set_error("points live on another device");
    return SDB_EINVAL;
  }
  const uint32_t B = pts->B, P = polys->n_polygons;
  std::vector<uint32_t> bb;
  SDB_TRY(polygon_bboxes(polys, B, &bb));
  std::vector<CoverQuery> cq(n_queries);
  std::vector<BatchQueryDev> hq(n_queries);
  std::vector<uint32_t> pp, pq, ps;
  uint64_t out_off = 0;
  for (uint32_t q = 0; q < n_queries; ++q) {
    const sdb_query& Qu = queries[q];
    uint32_t F = 0;
    sdb_status st = batch_query_dev(B, Qu, out_off, &hq[q], &F);
    if (st != SDB_OK) {
      set_error("query %u: %s", q, std::string(sdb_last_error()).c_str());
      return st;
    }
    if ((uint64_t)Qu.poly_off + Qu.poly_cnt > n_subset_ids || (Qu.poly_cnt && !subset_ids)) {
      set_error("query %u: polygon subset outside the id array", q);
      return SDB_EINVAL;
    }
    for (uint32_t t = 0; t < Qu.poly_cnt; ++t)
      if (subset_ids[Qu.poly_off + t] >= P) {
        set_error("query %u: polygon id %u out of range", q, subset_ids[Qu.poly_off + t]);
        return SDB_EINVAL;
      }
    if (out_off + Qu.poly_cnt >= 0xffffffffull) {
      set_error("batch output exceeds 2^32 entries");
      return SDB_EINVAL;
    }
    cq[q] = CoverQuery{F, Qu.x0, Qu.y0, Qu.x1, Qu.y1};
    viewport_pairs(bb, q, Qu, hq[q].k, subset_ids ? subset_ids + Qu.poly_off : nullptr, pp, pq,
                   ps);
    out_off += Qu.poly_cnt;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  sdb_batch* b = new (std::nothrow) sdb_batch();
  if (!b) {
    set_error("host allocation failed");
    return SDB_ENOMEM;
  }
  b->device = pts->device;
  b->NP = (uint32_t)pp.size();
  b->core.pts = pts;
  b->core.Q = n_queries;
  b->core.out_len = out_off;
  sdb_status st = build_query_coverings(poly_edges(polys), B, cq, pp, pq, ps, hq, &b->cs, 0, s,
                                        &b->n_ranges, &b->n_cells, &b->max_ranges);
  if (st == SDB_OK) {
    b->core.hq = hq;
    for (auto& c : b->cs)
      b->core.hchunks.push_back(BatchChunkDev{c.start, c.pay, c.list_off, c.list_ids});
    st = batch_core_prepare(&b->core, s);
  }
  if (st != SDB_OK) {
    std::string msg = sdb_last_error();
    sdb_batch_free(b);
    set_error("%s", msg.c_str());
    return st;
  }
  *out = b;
  return SDB_OK;
}

sdb_status sdb_batch_get_info(const sdb_batch* b, sdb_batch_info* info) {
  if (!b || !info) {
    set_error("batch or info is NULL");
    return SDB_EINVAL;
  }
  memset(info, 0, sizeof(*info));
  info->n_queries = b->core.Q;
  info->n_pairs = b->NP;
  info->out_len = b->core.out_len;
  info->n_ranges = b->n_ranges;
  info->max_ranges = b->max_ranges;
  info->n_cells = b->n_cells;
  info->candidates = b->core.candidates;
  info->n_tiles = b->core.ntiles;
  info->tile = b->core.tile;
  info->points_per_thread = b->core.ppt;
  info->lookup = b->core.learned ? SDB_LOOKUP_LEARNED : SDB_LOOKUP_BINARY;
  info->indexed_queries = b->core.indexed;
  info->n_leaves = b->core.nleaves;
  return SDB_OK;
}

sdb_status sdb_batch_set_lookup(sdb_batch* b, int lookup, void* cuda_stream) {
  if (!b || (lookup != SDB_LOOKUP_BINARY && lookup != SDB_LOOKUP_LEARNED)) {
    set_error("batch NULL, or a lookup other than binary search and the learned index");
    return SDB_EINVAL;
  }
  if (!valid_device(b->device)) {
    set_error("batch lives on another device");
    return SDB_EINVAL;
  }
  if (b->graph) {  // the captured launch refers to the old lookup structures
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return batch_core_index(&b->core, lookup == SDB_LOOKUP_LEARNED ? SDB_BATCH_LEARNED_MIN_RANGES : 0,
                          SDB_BATCH_RANGES_PER_LEAF, (cudaStream_t)cuda_stream);
}

sdb_status sdb_batch_fallbacks(const sdb_batch* b, void* cuda_stream, uint64_t* out) {
  if (!b || !out) {
    set_error("batch or output is NULL");
    return SDB_EINVAL;
  }
  *out = 0;
  if (!b->core.fallbacks) return SDB_OK;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  SDB_TRY_CUDA(cudaMemcpyAsync(out, b->core.fallbacks, 8, cudaMemcpyDeviceToHost, s));
  SDB_TRY_CUDA(cudaStreamSynchronize(s));
  return SDB_OK;
}

sdb_status sdb_batch_run(sdb_batch* b, int mode, uint64_t* d_count, int64_t* d_sum,
                         void* cuda_stream) {
  if (!b || !d_count) {
    set_error("batch or d_count is NULL");
    return SDB_EINVAL;
  }
  if (!valid_device(b->device)) {
    set_error("batch lives on another device");
    return SDB_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (mode == SDB_BATCH_PERSISTENT || mode == SDB_BATCH_PER_QUERY)
    return batch_core_run(&b->core, mode, d_count, d_sum, s);
  if (mode == SDB_BATCH_GRAPH) {
    if (s == nullptr) {
      set_error("graph mode needs a created stream (the legacy stream cannot be captured)");
      return SDB_EINVAL;
    }
    if (!b->graph || b->g_count != d_count || b->g_sum != d_sum) {
      if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
      }
      cudaGraph_t g = nullptr;
      SDB_TRY_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      sdb_status st = batch_core_run(&b->core, SDB_BATCH_PERSISTENT, d_count, d_sum, s);
      cudaError_t e = cudaStreamEndCapture(s, &g);
      if (st != SDB_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
      }
      if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture", __FILE__, __LINE__);
      e = cudaGraphInstantiate(&b->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        b->graph = nullptr;
        return cuda_status(e, "cudaGraphInstantiate", __FILE__, __LINE__);
      }
      b->g_count = d_count;
      b->g_sum = d_sum;
    }
    SDB_TRY_CUDA(cudaGraphLaunch(b->graph, s));
    return SDB_OK;
  }
  set_error("unknown batch mode %d", mode);
  return SDB_EINVAL;
}

static sdb_status set_tiles(sdb_batch* b, uint32_t T, cudaStream_t s) {
  SDB_TRY(batch_core_tiles(&b->core, T, s));
  if (b->graph) {  // the captured launch refers to the old work list
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return SDB_OK;
}

sdb_status sdb_batch_autotune(sdb_batch* b, void* cuda_stream, uint32_t* tile_out,
                              uint32_t* ppt_out) {
  if (!b) {
    set_error("batch is NULL");
    return SDB_EINVAL;
  }
  if (!valid_device(b->device)) {
    set_error("batch lives on another device");
    return SDB_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  Scratch sc(s);
  uint64_t* cnt;
  int64_t* sm;
  SDB_TRY(sc.get(&cnt, b->core.out_len));
  SDB_TRY(sc.get(&sm, b->core.out_len));
  cudaEvent_t e0, e1;
  SDB_TRY_CUDA(cudaEventCreate(&e0));
  SDB_TRY_CUDA(cudaEventCreate(&e1));
  const uint32_t tiles[] = {1024, 4096, 16384};
  const uint32_t ppts[] = {1, 2, 4};
  float best = 1e30f;
  uint32_t bt = b->core.tile, bp = b->core.ppt;
  sdb_status st = SDB_OK;
  for (uint32_t T : tiles) {
    if ((st = set_tiles(b, T, s)) != SDB_OK) break;
    for (uint32_t G : ppts) {
      b->core.ppt = G;
      float ms = 0;
      for (int rep = 0; rep < 2 && st == SDB_OK; ++rep) {  // the first run warms up
        cudaEventRecord(e0, s);
        st = batch_core_run(&b->core, SDB_BATCH_PERSISTENT, cnt, sm, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) st = SDB_ECUDA;
        cudaEventElapsedTime(&ms, e0, e1);
      }
      if (st != SDB_OK) break;
      if (ms < best) {
        best = ms;
        bt = T;
        bp = G;
      }
    }
    if (st != SDB_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->core.ppt = bp;
  if (st == SDB_OK) st = set_tiles(b, bt, s);
  if (st == SDB_OK) {
    if (tile_out) *tile_out = bt;
    if (ppt_out) *ppt_out = bp;
  }
  return st;
}

sdb_status sdb_batch_set_tuning(sdb_batch* b, uint32_t tile, uint32_t points_per_thread,
                                void* cuda_stream) {
  if (!b || tile == 0 || !(points_per_thread == 1 || points_per_thread == 2 ||
                           points_per_thread == 4)) {
    set_error("batch NULL, tile 0, or points per thread not 1, 2 or 4");
    return SDB_EINVAL;
  }
  b->core.ppt = points_per_thread;
  return set_tiles(b, tile, (cudaStream_t)cuda_stream);
}

sdb_status sdb_batch_query_ranges(const sdb_batch* b, uint32_t* h_ranges) {
  if (!b || !h_ranges) {
    set_error("batch or output is NULL");
    return SDB_EINVAL;
  }
  for (uint32_t q = 0; q < b->core.Q; ++q) h_ranges[q] = b->core.hq[q].R;
  return SDB_OK;
}

void sdb_batch_free(sdb_batch* b) {
  if (!b) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (auto& c : b->cs) c.release(0);
  b->core.release(0);
  cudaStreamSynchronize(0);
  cudaSetDevice(prev);
  delete b;
}

}  // extern "C"
