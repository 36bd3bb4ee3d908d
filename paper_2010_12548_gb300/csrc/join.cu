// Join fused with aggregation (Sec. 5.1): per point, its finest-level cell id
// (Sec. 3, "a query point is mapped to a cell on the most fine-grained grid
// level"), the covering range holding that id, and COUNT/SUM for every polygon
// on the range's list.  No exact geometric test.
//
// Layout and mapping:
//  * points are SoA uint32 x[], y[], int32 attr[]; each lane takes 4 consecutive
//    points per step (one 16-byte load per array, streaming cache hint), a warp
//    covers 128 consecutive points, all warps stride over the array;
//  * the cell id is computed 3 levels at a time from a 256-entry table that
//    each block stores in shared memory once per bank (conflict-free lookups);
//  * binary search: the top ~11 levels come from a sample of the range starts
//    staged in shared memory, the rest from global memory with a fixed number
//    of steps, the 4 points of a lane searched in lockstep so their loads
//    overlap;
//  * learned search: root model -> 32-byte leaf record (one load) -> FP32
//    prediction -> search inside the leaf's error window -> bracket verified
//    (only the ends no probe has proven are read), binary search as the
//    fallback (counted);
//  * cell table: one read of the entry of the point's cell at the table's
//    level (row-major, from the coordinates alone) gives the payload of most
//    points directly; points in cells that meet several ranges are held back
//    in a per-warp shared-memory queue and, 32 at a time (all lanes busy),
//    compute their finest cell id and binary search the cell's window of
//    range starts;
//  * cell table + learned index: as the cell table, but a held-back point's
//    search runs over the learned model's error window cut to the cell's
//    window (root knots in shared memory, one 32-byte leaf load), verified,
//    with the cell's whole window as the counted fallback;
//  * aggregation: per point, its count and (split 16/16-bit, exact) attribute
//    sum are added with shared-memory atomics to per-block accumulators
//    (P <= SMEM_POLYS, flushed into the 64-bit outputs every few tiles), or
//    with global atomics straight into the outputs.
#include "hilbert.cuh"
#include "sdb_internal.cuh"

namespace sdb {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr uint32_t NONE = 0xffffffffu;
constexpr int THREADS = 256;
constexpr uint32_t SMEM_POLYS = 2048;
// windows of the table's mixed cells longer than this are searched through the
// learned model (table + learned lookup), shorter ones directly
constexpr uint32_t LEARNED_MIN_WINDOW = 64;

constexpr uint32_t SMEM_POLYS_RANGE = 1024;  // 32 bytes of accumulators per polygon

struct JoinArgs {
  const uint32_t* x;
  const uint32_t* y;
  const int32_t* attr;
  uint64_t n;
  unsigned long long* count;
  unsigned long long* sum;
  // result-range partials (Sec. 6): boundary count, boundary attribute sum
  // and sum of magnitudes
  unsigned long long* bcount;
  unsigned long long* bsum;
  unsigned long long* babs;
  int vec;
  // covering
  const uint64_t* start;
  const uint32_t* pay;
  const uint32_t* list_off;
  const uint32_t* list_ids;
  const uint64_t* sample;
  uint64_t R;
  uint32_t sample_n, stride;
  uint32_t B, k, nsteps, st0, P;
  // learned index, and its fences (start[j << FENCE_SHIFT])
  const LeafRec* leaves;
  const uint64_t* fence;
  const float* knots;
  uint32_t nknots, wshift;
  float inv_w;
  uint32_t nleaves;
  unsigned long long* fallbacks;
  // cell table: the entry of a point is at (y >> txy) << tlev | (x >> txy)
  // (row-major cells of level tlev)
  const uint32_t* tab;
  const uint2* win;  // windows of the mixed cells of the last table level
  uint32_t txy, tlev;
  // second table level (sub == nullptr: none): sub-cell of a point in mixed
  // bucket m at sub[m << 2 s2 | ((y >> txy2) & S-1) << s2 | ((x >> txy2) & S-1)]
  const uint32_t* sub;
  uint32_t s2, txy2;
  // the tree's top level, staged in shared memory (top == nullptr: none): the
  // byte of a point is at (y >> top_xy) << top_lev | (x >> top_xy), an index
  // into the palette of payloads top_pal, TOP_NONE or TOP_ASK
  const uint8_t* top;
  const uint32_t* top_pal;
  uint32_t top_xy, top_lev;
};

// last r in [0, R) with start[r] <= h, global memory only (fallback path)
__device__ __noinline__ uint32_t bs_global(const uint64_t* __restrict__ start, uint64_t R,
                                           uint64_t h) {
  uint64_t lo = 0, len = R + 1;
  while (len > 1) {
    uint64_t half = len >> 1;
    if (__ldg(start + lo + half) <= h) lo += half;
    len -= half;
  }
  return (uint32_t)lo;
}

template <int G>
__device__ __forceinline__ void find_bs(const uint64_t (&h)[G], uint32_t (&r)[G],
                                        const uint64_t* s_sample, const JoinArgs& A) {
  uint32_t j[G];
#pragma unroll
  for (int q = 0; q < G; ++q) j[q] = 0;
  for (uint32_t len = A.sample_n; len > 1;) {
    uint32_t half = len >> 1;
#pragma unroll
    for (int q = 0; q < G; ++q)
      if (s_sample[j[q] + half] <= h[q]) j[q] += half;
    len -= half;
  }
  uint64_t lo[G];
#pragma unroll
  for (int q = 0; q < G; ++q) lo[q] = (uint64_t)j[q] * A.stride;
  for (uint32_t len = A.stride; len > 1;) {
    uint32_t half = len >> 1;
    uint64_t v[G];
#pragma unroll
    for (int q = 0; q < G; ++q) {
      uint64_t idx = lo[q] + half;
      v[q] = __ldg(A.start + (idx < A.R ? idx : A.R));
    }
#pragma unroll
    for (int q = 0; q < G; ++q)
      if (v[q] <= h[q]) lo[q] += half;
    len -= half;
  }
#pragma unroll
  for (int q = 0; q < G; ++q) r[q] = (uint32_t)lo[q];
}

template <int G>
__device__ __forceinline__ void find_learned(const uint64_t (&h)[G], uint32_t (&r)[G],
                                             const float* s_knots, const JoinArgs& A) {
  // the model's window [a, b] of each point, then the last fence in it at or
  // below h (fences stay cache-resident), then the window cut to that fence's
  // block of 2^FENCE_SHIFT starts (one 128-byte line) searched to the end
  uint32_t lo[G], b[G], jlo[G], jlen[G];  // range indices are below 2^32
  uint32_t maxlen = 1;
#pragma unroll
  for (int q = 0; q < G; ++q) {
    const uint32_t l = root_leaf(s_knots, A.wshift, A.inv_w, A.nleaves, h[q]);
    // the 32-byte record in one load (records are 32-byte aligned)
    uint64_t w0, w1, w2, w3;
    asm("ld.global.nc.v4.u64 {%0, %1, %2, %3}, [%4];"
        : "=l"(w0), "=l"(w1), "=l"(w2), "=l"(w3)
        : "l"(A.leaves + l));
    LeafRec lr;
    lr.base = w0;
    lr.a = __uint_as_float((uint32_t)w1);
    lr.b = __uint_as_float((uint32_t)(w1 >> 32));
    lr.first = (uint32_t)w2;
    lr.last = (uint32_t)(w2 >> 32);
    lr.errlo = (int32_t)(uint32_t)w3;
    lr.errhi = (int32_t)(uint32_t)(w3 >> 32);
    const int64_t pr = leaf_predict(lr, h[q]);
    int64_t wa = pr - lr.errlo, wb = pr + lr.errhi;
    if (wa < (int64_t)lr.first) wa = lr.first;
    if (wb > (int64_t)lr.last) wb = lr.last;
    if (wb < wa) wb = wa;
    lo[q] = (uint32_t)wa;
    b[q] = (uint32_t)wb;
    jlo[q] = lo[q] >> FENCE_SHIFT;
    jlen[q] = ((uint32_t)wb >> FENCE_SHIFT) - jlo[q] + 1;
    maxlen = max(maxlen, jlen[q]);
  }
  // the same number of halving steps for the whole warp; finished lanes idle
  maxlen = __reduce_max_sync(FULL, maxlen);
  for (int st = 32 - __clz(maxlen - 1); st > 0; --st) {
    uint64_t v[G];
#pragma unroll
    for (int q = 0; q < G; ++q)
      if (jlen[q] > 1) v[q] = __ldg(A.fence + jlo[q] + (jlen[q] >> 1));
#pragma unroll
    for (int q = 0; q < G; ++q) {
      if (jlen[q] > 1) {
        const uint32_t half = jlen[q] >> 1;
        if (v[q] <= h[q]) jlo[q] += half;
        jlen[q] -= half;
      }
    }
  }
  uint32_t len[G];
  maxlen = 1;
#pragma unroll
  for (int q = 0; q < G; ++q) {
    const uint32_t blk = jlo[q] << FENCE_SHIFT;
    const uint32_t s0 = lo[q] > blk ? lo[q] : blk;
    const uint32_t e0 = blk + ((1u << FENCE_SHIFT) - 1) < b[q] ? blk + ((1u << FENCE_SHIFT) - 1) : b[q];
    lo[q] = s0;
    len[q] = e0 - s0 + 1;
    maxlen = max(maxlen, len[q]);
  }
  maxlen = __reduce_max_sync(FULL, maxlen);
  for (int st = 32 - __clz(maxlen - 1); st > 0; --st) {
    uint64_t v[G];
#pragma unroll
    for (int q = 0; q < G; ++q)
      if (len[q] > 1) v[q] = __ldg(A.start + lo[q] + (len[q] >> 1));
#pragma unroll
    for (int q = 0; q < G; ++q) {
      if (len[q] > 1) {
        const uint32_t half = len[q] >> 1;
        if (v[q] <= h[q]) lo[q] += half;
        len[q] -= half;
      }
    }
  }
  // verification: the result must bracket h (start[lo] from the line just
  // searched, start[lo + 1] from it or, at the line's end, from the next fence);
  // otherwise plain binary search decides
#pragma unroll
  for (int q = 0; q < G; ++q) {
    const uint32_t nx = lo[q] + 1;
    const uint64_t s0 = __ldg(A.start + lo[q]);
    const uint64_t s1 = (nx & ((1u << FENCE_SHIFT) - 1)) ? __ldg(A.start + nx)
                                                         : __ldg(A.fence + (nx >> FENCE_SHIFT));
    if (s0 <= h[q] && h[q] < s1) {
      r[q] = lo[q];
    } else {
      atomicAdd(A.fallbacks, 1ull);
      r[q] = bs_global(A.start, A.R, h[q]);
    }
  }
}

// Per-block accumulators in shared memory (P <= SMEM_POLYS): a 32-bit count
// and the attribute sum split exactly into its low 16 bits (unsigned) and the
// rest (signed), each in a 32-bit counter.  A block flushes them into the global
// 64-bit outputs at least every FLUSH_POINTS points, so none can wrap:
// FLUSH_POINTS * 65535 < 2^32 and FLUSH_POINTS * 32768 < 2^31.  Points a warp
// holds back in its queue (the cell-table lookup's mixed buckets, at most
// QCAP - 1 per warp across a flush) count against the same bound.  (One 64-bit
// word per polygon holding count and biased sum would need one atomic instead
// of three, but 64-bit shared-memory atomics measured slower on GB300.)
constexpr uint32_t FLUSH_TILES = 31;
constexpr int QCAP = 64;  // per-warp queue of points in mixed cell-table buckets
constexpr uint32_t FLUSH_POINTS = FLUSH_TILES * THREADS * 4 + (THREADS / 32) * (QCAP - 1);
static_assert((uint64_t)FLUSH_POINTS * 65535u < (1ull << 32), "low-half counter could wrap");
static_assert((uint64_t)FLUSH_POINTS * 32768u < (1ull << 31), "high-half counter could wrap");

// With result-range partials, boundary points add to a second set of the same
// counters and to a magnitude sum, split the same way (|a| <= 2^31, so its high
// half is at most 2^15 per point).
struct Acc {
  uint32_t* cnt;
  uint32_t* lo;
  int32_t* hi;
  uint32_t* bcnt;
  uint32_t* blo;
  int32_t* bhi;
  uint32_t* alo;
  uint32_t* ahi;
};

// shared-memory bytes of the accumulators of P polygons
__host__ __device__ constexpr size_t acc_bytes(size_t P, bool SUM, bool RANGE) {
  return P * ((SUM ? 12 : 4) + (RANGE ? (SUM ? 20 : 4) : 0));
}

// carve the accumulators out of shared memory at p: P words each of
// cnt [, lo, hi] [, bcnt [, blo, bhi, alo, ahi]]
template <bool SUM, bool RANGE>
__device__ __forceinline__ Acc acc_at(unsigned char* p, size_t P) {
  Acc s{};
  uint32_t* w = reinterpret_cast<uint32_t*>(p);
  s.cnt = w;
  w += P;
  if (SUM) {
    s.lo = w;
    s.hi = reinterpret_cast<int32_t*>(w + P);
    w += 2 * P;
  }
  if (RANGE) {
    s.bcnt = w;
    w += P;
    if (SUM) {
      s.blo = w;
      s.bhi = reinterpret_cast<int32_t*>(w + P);
      s.alo = w + 2 * P;
      s.ahi = w + 3 * P;
    }
  }
  return s;
}

template <bool SUM, bool RANGE>
__device__ __forceinline__ void acc_zero(const Acc& s, uint32_t P) {
  for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
    s.cnt[i] = 0;
    if (SUM) {
      s.lo[i] = 0;
      s.hi[i] = 0;
    }
    if (RANGE) {
      s.bcnt[i] = 0;
      if (SUM) {
        s.blo[i] = 0;
        s.bhi[i] = 0;
        s.alo[i] = 0;
        s.ahi[i] = 0;
      }
    }
  }
}

template <bool SMEM, bool SUM, bool RANGE>
__device__ __forceinline__ void add_one(uint32_t p, int32_t a, uint32_t bnd, const Acc& s,
                                        const JoinArgs& A) {
  const uint32_t m = a < 0 ? 0u - (uint32_t)a : (uint32_t)a;  // |a|
  if (SMEM) {
    atomicAdd(&s.cnt[p], 1u);
    if (SUM) {
      atomicAdd(&s.lo[p], (uint32_t)a & 0xffffu);
      if (a >> 16) atomicAdd(&s.hi[p], a >> 16);  // zero for attributes in [0, 2^16)
    }
    if (RANGE && bnd) {
      atomicAdd(&s.bcnt[p], 1u);
      if (SUM) {
        atomicAdd(&s.blo[p], (uint32_t)a & 0xffffu);
        atomicAdd(&s.bhi[p], a >> 16);
        atomicAdd(&s.alo[p], m & 0xffffu);
        atomicAdd(&s.ahi[p], m >> 16);
      }
    }
  } else {
    atomicAdd(&A.count[p], 1ull);
    if (SUM) atomicAdd(&A.sum[p], (unsigned long long)(long long)a);
    if (RANGE && bnd) {
      atomicAdd(&A.bcount[p], 1ull);
      if (SUM) {
        atomicAdd(&A.bsum[p], (unsigned long long)(long long)a);
        atomicAdd(&A.babs[p], (unsigned long long)m);
      }
    }
  }
}

template <bool SUM, bool RANGE>
__device__ void flush_acc(const Acc& s, const JoinArgs& A) {
  for (uint32_t i = threadIdx.x; i < A.P; i += blockDim.x) {
    const uint32_t c = s.cnt[i];
    if (c) {
      atomicAdd(&A.count[i], (unsigned long long)c);
      s.cnt[i] = 0;
      if (SUM) {
        const long long tot = (long long)s.hi[i] * 65536 + (long long)s.lo[i];
        atomicAdd(&A.sum[i], (unsigned long long)tot);
        s.lo[i] = 0;
        s.hi[i] = 0;
      }
    }
    if (RANGE) {
      const uint32_t bc = s.bcnt[i];
      if (bc) {
        atomicAdd(&A.bcount[i], (unsigned long long)bc);
        s.bcnt[i] = 0;
        if (SUM) {
          const long long bt = (long long)s.bhi[i] * 65536 + (long long)s.blo[i];
          const unsigned long long at =
              (unsigned long long)s.ahi[i] * 65536ull + (unsigned long long)s.alo[i];
          atomicAdd(&A.bsum[i], (unsigned long long)bt);
          atomicAdd(&A.babs[i], at);
          s.blo[i] = 0;
          s.bhi[i] = 0;
          s.alo[i] = 0;
          s.ahi[i] = 0;
        }
      }
    }
  }
}

// a range payload: one polygon (slot | boundary << 30), a list (2^31 | r; list
// entries slot | boundary << 31), or none
template <bool SMEM, bool SUM, bool RANGE>
__device__ __forceinline__ void add_pay(uint32_t pay, int32_t a, const Acc& acc,
                                        const JoinArgs& A) {
  if (pay < 0x80000000u) {
    add_one<SMEM, SUM, RANGE>(pay & 0x3fffffffu, a, (pay >> 30) & 1u, acc, A);
  } else if (pay != NONE) {  // several polygons share the range
    const uint32_t rr = pay & 0x7fffffffu;
    const uint32_t b = __ldg(A.list_off + rr), e = __ldg(A.list_off + rr + 1);
    for (uint32_t i = b; i < e; ++i) {
      const uint32_t id = __ldg(A.list_ids + i);
      add_one<SMEM, SUM, RANGE>(id & 0x7fffffffu, a, id >> 31, acc, A);
    }
  }
}

// a point held back in a warp's queue: its coordinates, mixed bucket and
// attribute (16 bytes)
struct QEnt {
  uint32_t x, y, m;
  int32_t a;
};

// the range of a point in mixed cell m of the table's last level (a bucket, or
// a sub-cell of the second level): its finest cell id, then a binary search of
// the cell's window of range starts (w.x = the range holding the cell's first
// id, w.y = the range holding its last, so start[w.x] <= h < start[w.y + 1]).  With the learned index (LOOKUP == SDB_LOOKUP_TABLE_LEARNED)
// the search runs over the model's error window cut to the bucket's window;
// an end of the result no probe has proven is read, and a result that does not
// bracket h falls back to the bucket's whole window (counted).
template <int LOOKUP, bool SMEM, bool SUM, bool RANGE>
__device__ __forceinline__ void resolve_mixed(const QEnt& E, const uint32_t* s_tab,
                                              const Acc& acc, const JoinArgs& A) {
  const uint64_t h = hilbert3_encode_compact(E.x >> A.k, E.y >> A.k, A.nsteps, A.st0, s_tab);
  const uint2 w = __ldg(A.win + E.m);
  uint32_t lo = w.x, len = w.y - w.x + 1;
  // the model replaces the search where the window is long; a short window
  // costs fewer probes than the model's root, leaf and verification reads
  if (LOOKUP == SDB_LOOKUP_TABLE_LEARNED && len > LEARNED_MIN_WINDOW) {
    // the root knots through the L1 cache: only points in mixed buckets read them
    const uint32_t l = root_leaf(A.knots, A.wshift, A.inv_w, A.nleaves, h);
    uint64_t w0, w1, w2, w3;
    asm("ld.global.nc.v4.u64 {%0, %1, %2, %3}, [%4];"
        : "=l"(w0), "=l"(w1), "=l"(w2), "=l"(w3)
        : "l"(A.leaves + l));
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
    a = a > (int64_t)w.x ? a : (int64_t)w.x;
    b = b < (int64_t)w.y ? b : (int64_t)w.y;
    if (b < a) b = a;  // an empty cut (a model miss): one candidate, then the check
    lo = (uint32_t)a;
    len = (uint32_t)(b - a + 1);
    // bit 0: start[lo] <= h is proven, bit 1: start[lo + 1] > h is proven
    uint32_t known = (lo == w.x ? 1u : 0u) | ((uint32_t)b == w.y ? 2u : 0u);
    while (len > 1) {
      const uint32_t half = len >> 1;
      if (__ldg(A.start + lo + half) <= h) {
        lo += half;
        known |= 1u;
      } else {
        known |= 2u;
      }
      len -= half;
    }
    const bool ok0 = (known & 1u) || __ldg(A.start + lo) <= h;
    const bool ok1 = (known & 2u) || h < __ldg(A.start + lo + 1);
    if (ok0 && ok1) {
      add_pay<SMEM, SUM, RANGE>(__ldg(A.pay + lo), E.a, acc, A);
      return;
    }
    atomicAdd(A.fallbacks, 1ull);
    lo = w.x;
    len = w.y - w.x + 1;
  }
  while (len > 1) {
    const uint32_t half = len >> 1;
    if (__ldg(A.start + lo + half) <= h) lo += half;
    len -= half;
  }
  add_pay<SMEM, SUM, RANGE>(__ldg(A.pay + lo), E.a, acc, A);
}

// shared-memory bytes of the cell-id table: replicated per bank where every
// point encodes, one unreplicated copy for the table lookups (only points in
// mixed buckets encode there, and shared memory left unused stays L1 cache,
// which holds the lines of the table gathers in flight)
__host__ __device__ constexpr size_t hilbert_bytes(int lookup) {
  return (lookup == SDB_LOOKUP_TABLE || lookup == SDB_LOOKUP_TABLE_LEARNED)
             ? (size_t)HILBERT3_COMPACT_BYTES
             : (size_t)HILBERT3_SMEM_BYTES;
}

// shared-memory bytes of the lookup's staging area (8-byte multiple): the
// binary search's sample, the learned index's root knots, or the cell table's
// per-warp queues (blocks of tpb threads)
__host__ __device__ inline size_t stage_bytes(int lookup, const JoinArgs& A, int tpb) {
  if (lookup == SDB_LOOKUP_BINARY) return (size_t)A.sample_n * 8;
  if (lookup == SDB_LOOKUP_LEARNED) return ((size_t)A.nknots * 4 + 7) & ~(size_t)7;
  return (size_t)(tpb / 32) * QCAP * sizeof(QEnt);
}

// The table lookups with the tree's top level in shared memory run two blocks
// of TOP_THREADS per SM (the level and its palette take 65 KB per block, and
// the kernel fits 40 registers); their accumulators are flushed every
// TOP_FLUSH_TILES tiles, which keeps the same no-wrap bound.
constexpr int TOP_THREADS = 768;
constexpr int TOP_BLOCKS = 2;
constexpr uint32_t TOP_FLUSH_TILES = 20;
static_assert((uint64_t)(TOP_FLUSH_TILES * TOP_THREADS * 4 + (TOP_THREADS / 32) * (QCAP - 1)) *
                      65535u < (1ull << 32),
              "low-half counter could wrap");
static_assert((uint64_t)(TOP_FLUSH_TILES * TOP_THREADS * 4 + (TOP_THREADS / 32) * (QCAP - 1)) *
                      32768u < (1ull << 31),
              "high-half counter could wrap");

// the top level's bytes (a multiple of 16 from level 2 on) and its palette
__host__ __device__ inline size_t top_bytes(const JoinArgs& A) {
  return ((size_t)1 << (2 * A.top_lev)) + 4 * TOP_PALETTE;
}

template <int LOOKUP, bool SMEM, bool SUM, bool RANGE, bool TOP = false>
__global__ __launch_bounds__(TOP ? TOP_THREADS : THREADS, TOP ? TOP_BLOCKS : 4) void join_kernel(JoinArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int TPB = TOP ? TOP_THREADS : THREADS;
  constexpr uint32_t FT = TOP ? TOP_FLUSH_TILES : FLUSH_TILES;
  // the cell-id table, then the lookup staging (the binary search's sample of
  // range starts, the learned index's root knots, or the cell-table lookup's
  // per-warp queues), then the accumulators, then (TOP) the tree's top level
  uint32_t* s_tab = reinterpret_cast<uint32_t*>(smem);
  constexpr bool TABLE = LOOKUP == SDB_LOOKUP_TABLE || LOOKUP == SDB_LOOKUP_TABLE_LEARNED;
  static_assert(!TOP || TABLE, "the top level belongs to the table lookups");
  constexpr size_t HB = hilbert_bytes(LOOKUP);
  uint64_t* s_sample = reinterpret_cast<uint64_t*>(smem + HB);
  float* s_knots = reinterpret_cast<float*>(smem + HB);
  QEnt* s_q = reinterpret_cast<QEnt*>(smem + HB) + (threadIdx.x >> 5) * QCAP;
  const size_t off = HB + stage_bytes(LOOKUP, A, TPB);
  const Acc acc = acc_at<SUM, RANGE>(smem + off, SMEM ? A.P : 0);
  uint8_t* s_top =
      smem + ((off + acc_bytes(SMEM ? A.P : 0, SUM, RANGE) + 15) & ~(size_t)15);
  uint32_t* s_pal = reinterpret_cast<uint32_t*>(s_top + ((size_t)1 << (2 * A.top_lev)));

  if constexpr (TABLE)
    hilbert3_fill_compact(s_tab);
  else
    hilbert3_fill(s_tab);
  if constexpr (LOOKUP == SDB_LOOKUP_BINARY)
    for (uint32_t i = threadIdx.x; i < A.sample_n; i += TPB) s_sample[i] = A.sample[i];
  if constexpr (LOOKUP == SDB_LOOKUP_LEARNED)
    for (uint32_t i = threadIdx.x; i < A.nknots; i += TPB) s_knots[i] = A.knots[i];
  if constexpr (TOP) {  // 16-byte copies of the top level, then its palette
    const uint4* src = reinterpret_cast<const uint4*>(A.top);
    uint4* dst = reinterpret_cast<uint4*>(s_top);
    for (uint32_t i = threadIdx.x; i < (1u << (2 * A.top_lev)) / 16; i += TPB) dst[i] = __ldg(src + i);
    for (uint32_t i = threadIdx.x; i < TOP_PALETTE; i += TPB) s_pal[i] = __ldg(A.top_pal + i);
  }
  if (SMEM) acc_zero<SUM, RANGE>(acc, A.P);
  __syncthreads();

  const uint32_t lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t qn = 0;  // entries in this warp's queue (warp-uniform)
  const uint32_t gmask = ~((1u << A.B) - 1u);
  const uint64_t per_tile = (uint64_t)TPB * 4;
  const uint64_t ntiles = (A.n + per_tile - 1) / per_tile;
  uint32_t since_flush = 0;
  // block-uniform loop over tiles of 4 TPB consecutive points; thread t takes
  // points 4t..4t+3 of the tile (a warp reads 512 contiguous bytes per array)
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint64_t e0 = t * per_tile + (uint64_t)threadIdx.x * 4;
    uint32_t xs[4], ys[4];
    int32_t as[4];
    bool ok[4];
    if (A.vec && e0 + 3 < A.n) {
      const uint4 xv = __ldcs(reinterpret_cast<const uint4*>(A.x + e0));
      const uint4 yv = __ldcs(reinterpret_cast<const uint4*>(A.y + e0));
      xs[0] = xv.x; xs[1] = xv.y; xs[2] = xv.z; xs[3] = xv.w;
      ys[0] = yv.x; ys[1] = yv.y; ys[2] = yv.z; ys[3] = yv.w;
      if (SUM) {
        const int4 av = __ldcs(reinterpret_cast<const int4*>(A.attr + e0));
        as[0] = av.x; as[1] = av.y; as[2] = av.z; as[3] = av.w;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) ok[q] = true;
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        ok[q] = e0 + q < A.n;
        xs[q] = ok[q] ? A.x[e0 + q] : 0u;
        ys[q] = ok[q] ? A.y[e0 + q] : 0u;
        if (SUM) as[q] = ok[q] ? A.attr[e0 + q] : 0;
      }
    }
    if (!SUM) {
#pragma unroll
      for (int q = 0; q < 4; ++q) as[q] = 0;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) ok[q] = ok[q] && !((xs[q] | ys[q]) & gmask);
    if constexpr (TABLE) {
      // the entry of the point's cell at the table's level, found from the
      // coordinates (row-major table); only points in mixed cells need their
      // finest cell id
      uint32_t e[4];
      if constexpr (TOP) {
        // the top level answers points whose top cell lies in one range; the
        // others read the table as below
        bool ask[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint8_t v =
              ok[q] ? s_top[((ys[q] >> A.top_xy) << A.top_lev) | (xs[q] >> A.top_xy)] : TOP_NONE;
          ask[q] = v == TOP_ASK;
          e[q] = v >= TOP_NONE ? NONE : s_pal[v];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (ask[q]) e[q] = __ldg(A.tab + (((ys[q] >> A.txy) << A.tlev) | (xs[q] >> A.txy)));
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          e[q] = ok[q] ? __ldg(A.tab + (((ys[q] >> A.txy) << A.tlev) | (xs[q] >> A.txy))) : NONE;
      }
      if (A.sub) {  // a point in a mixed bucket reads its sub-cell's entry
        const uint32_t smask = (1u << A.s2) - 1u;
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (e[q] >= TAB_MIXED && e[q] != NONE)
            e[q] = __ldg(A.sub + (((uint64_t)(e[q] & ~TAB_MIXED) << (2 * A.s2)) |
                                  (((ys[q] >> A.txy2) & smask) << A.s2) |
                                  ((xs[q] >> A.txy2) & smask)));
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const bool mix = e[q] >= TAB_MIXED && e[q] != NONE;
        const uint32_t bal = __ballot_sync(FULL, mix);
        if (mix) {
          QEnt& E = s_q[qn + __popc(bal & lt)];
          E.x = xs[q];
          E.y = ys[q];
          E.m = e[q] & ~TAB_MIXED;
          E.a = as[q];
        } else {
          add_pay<SMEM, SUM, RANGE>(e[q], as[q], acc, A);
        }
        qn += __popc(bal);
        if (qn >= 32) {  // a full warp of held-back points: search their windows
          __syncwarp();
          qn -= 32;
          const QEnt E = s_q[qn + lane];
          __syncwarp();
          resolve_mixed<LOOKUP, SMEM, SUM, RANGE>(E, s_tab, acc, A);
        }
      }
    } else {
      uint64_t h[4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        h[q] = ok[q] ? hilbert3_encode(xs[q] >> A.k, ys[q] >> A.k, A.nsteps, A.st0, s_tab) : 0ull;
      uint32_t r[4];
      if constexpr (LOOKUP == SDB_LOOKUP_BINARY)
        find_bs<4>(h, r, s_sample, A);
      else
        find_learned<4>(h, r, s_knots, A);
      uint32_t pay[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) pay[q] = ok[q] ? __ldg(A.pay + r[q]) : NONE;
#pragma unroll
      for (int q = 0; q < 4; ++q) add_pay<SMEM, SUM, RANGE>(pay[q], as[q], acc, A);
    }
    if (SMEM && ++since_flush == FT) {
      since_flush = 0;
      __syncthreads();
      flush_acc<SUM, RANGE>(acc, A);
      __syncthreads();
    }
  }
  if constexpr (TABLE) {  // the rest of the queue
    __syncwarp();
    if (lane < qn) resolve_mixed<LOOKUP, SMEM, SUM, RANGE>(s_q[lane], s_tab, acc, A);
  }
  if (SMEM) {
    __syncthreads();
    flush_acc<SUM, RANGE>(acc, A);
  }
}

template <int LOOKUP, bool SMEM, bool SUM, bool RANGE, bool TOP = false>
sdb_status launch_t(const JoinArgs& A, cudaStream_t s) {
  constexpr int TPB = TOP ? TOP_THREADS : THREADS;
  size_t smem = hilbert_bytes(LOOKUP) + stage_bytes(LOOKUP, A, TPB);
  if (SMEM) smem += acc_bytes(A.P, SUM, RANGE);
  smem = (smem + 15) & ~(size_t)15;
  if (TOP) smem += top_bytes(A);
  auto kern = join_kernel<LOOKUP, SMEM, SUM, RANGE, TOP>;
  if (smem > 48 * 1024)
    SDB_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  SDB_TRY(occupancy(reinterpret_cast<const void*>(kern), TPB, smem, &per_sm));
  // ask for no more shared memory than the resident blocks use (plus the 1 KB
  // the system reserves per block): the rest of the SM's unified memory stays
  // L1 cache, whose lines hold the lookups' gathers in flight
  SDB_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                    carveout_pct((size_t)per_sm * (smem + 1024))));
  uint64_t blocks = (uint64_t)num_sms() * per_sm;
  const uint64_t need = (A.n + 4 * TPB - 1) / (4 * TPB);  // tiles
  if (blocks > need) blocks = need > 0 ? need : 1;
  TraceScope tr("join", s);
  kern<<<(unsigned)blocks, TPB, smem, s>>>(A);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  return SDB_OK;
}


// ------------------------------------------------ several coverings at once
// One pass over the points for up to MULTI coverings of the same polygons (an
// eps sweep): each point is loaded and its cell id computed once, at the
// finest level of the set; a coarser covering's id is a prefix of it (the
// curve's prefix property: drop 2 * (F - F') low bits).  Lookups and
// accumulators are per covering; the coverings' root knots and samples are
// read through the L1 cache.
constexpr int MULTI = 4;
struct MultiArgs {
  JoinArgs c[MULTI];       // points, grid and the finest level's encoding in c[0]
  uint32_t shift[MULTI];   // id of covering e = finest id >> shift[e]
  uint32_t E;
};

template <int LOOKUP, bool SMEM, bool SUM>
__global__ __launch_bounds__(THREADS, 4) void join_multi_kernel(MultiArgs M) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* s_tab = reinterpret_cast<uint32_t*>(smem);
  const JoinArgs& A0 = M.c[0];
  const size_t P = SMEM ? A0.P : 0;
  unsigned char* accb = smem + HILBERT3_SMEM_BYTES;
  Acc acc[MULTI];
#pragma unroll
  for (int e = 0; e < MULTI; ++e) acc[e] = acc_at<SUM, false>(accb + e * acc_bytes(P, SUM, false), P);
  hilbert3_fill(s_tab);
  if (SMEM)
#pragma unroll
    for (int e = 0; e < MULTI; ++e)
      if (e < (int)M.E) acc_zero<SUM, false>(acc[e], (uint32_t)P);
  __syncthreads();

  const uint32_t gmask = ~((1u << A0.B) - 1u);
  const uint64_t per_tile = (uint64_t)THREADS * 4;
  const uint64_t ntiles = (A0.n + per_tile - 1) / per_tile;
  uint32_t since_flush = 0;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint64_t e0 = t * per_tile + (uint64_t)threadIdx.x * 4;
    uint32_t xs[4], ys[4];
    int32_t as[4];
    bool ok[4];
    if (A0.vec && e0 + 3 < A0.n) {
      const uint4 xv = __ldcs(reinterpret_cast<const uint4*>(A0.x + e0));
      const uint4 yv = __ldcs(reinterpret_cast<const uint4*>(A0.y + e0));
      xs[0] = xv.x; xs[1] = xv.y; xs[2] = xv.z; xs[3] = xv.w;
      ys[0] = yv.x; ys[1] = yv.y; ys[2] = yv.z; ys[3] = yv.w;
      if (SUM) {
        const int4 av = __ldcs(reinterpret_cast<const int4*>(A0.attr + e0));
        as[0] = av.x; as[1] = av.y; as[2] = av.z; as[3] = av.w;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) ok[q] = true;
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        ok[q] = e0 + q < A0.n;
        xs[q] = ok[q] ? A0.x[e0 + q] : 0u;
        ys[q] = ok[q] ? A0.y[e0 + q] : 0u;
        if (SUM) as[q] = ok[q] ? A0.attr[e0 + q] : 0;
      }
    }
    uint64_t h[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      ok[q] = ok[q] && !((xs[q] | ys[q]) & gmask);
      h[q] = ok[q] ? hilbert3_encode(xs[q] >> A0.k, ys[q] >> A0.k, A0.nsteps, A0.st0, s_tab) : 0ull;
    }
#pragma unroll
    for (int e = 0; e < MULTI; ++e) {
      if (e >= (int)M.E) break;
      const JoinArgs& A = M.c[e];
      uint64_t he[4];
      uint32_t r[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) he[q] = h[q] >> M.shift[e];
      if (LOOKUP == SDB_LOOKUP_BINARY)
        find_bs<4>(he, r, A.sample, A);
      else
        find_learned<4>(he, r, A.knots, A);
      uint32_t pay[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) pay[q] = ok[q] ? __ldg(A.pay + r[q]) : NONE;
#pragma unroll
      for (int q = 0; q < 4; ++q) add_pay<SMEM, SUM, false>(pay[q], SUM ? as[q] : 0, acc[e], A);
    }
    if (SMEM && ++since_flush == FLUSH_TILES) {
      since_flush = 0;
      __syncthreads();
#pragma unroll
      for (int e = 0; e < MULTI; ++e)
        if (e < (int)M.E) flush_acc<SUM, false>(acc[e], M.c[e]);
      __syncthreads();
    }
  }
  if (SMEM) {
    __syncthreads();
#pragma unroll
    for (int e = 0; e < MULTI; ++e)
      if (e < (int)M.E) flush_acc<SUM, false>(acc[e], M.c[e]);
  }
}

template <int LOOKUP, bool SMEM, bool SUM>
sdb_status launch_multi_t(const MultiArgs& M, cudaStream_t s) {
  size_t smem = HILBERT3_SMEM_BYTES;
  if (SMEM) smem += (size_t)M.E * acc_bytes(M.c[0].P, SUM, false);
  smem = (smem + 15) & ~(size_t)15;
  auto kern = join_multi_kernel<LOOKUP, SMEM, SUM>;
  if (smem > 48 * 1024)
    SDB_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  SDB_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, smem));
  if (per_sm < 1) per_sm = 1;
  uint64_t blocks = (uint64_t)num_sms() * per_sm;
  const uint64_t need = (M.c[0].n + 4 * THREADS - 1) / (4 * THREADS);
  if (blocks > need) blocks = need > 0 ? need : 1;
  kern<<<(unsigned)blocks, THREADS, smem, s>>>(M);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  return SDB_OK;
}

// ------------------------------------------------ an eps sweep through the tables
// One pass over the points for up to MULTI coverings of the same polygons with
// cell tables (an eps sweep): each point is read once; a combined top level in
// shared memory -- a top cell whose payload is the same single polygon in
// every covering -- answers it for all coverings at once; otherwise each
// covering's table and second level answer it in turn.  Points in mixed cells
// of any covering wait in one per-warp queue (the covering's number in the top
// two bits of the queued cell index) and are searched 32 at a time, so the
// kernel holds one copy of the window search per queue drain, not one per
// covering and point (an unrolled form spent two thirds of its cycles waiting
// for instructions).
struct SweepArgs {
  JoinArgs c[MULTI];       // per covering: its table, lookup and outputs
  uint32_t E;
  const uint8_t* top;      // combined top level (nullptr: every point asks the tables)
  const uint32_t* pal;     // its palette (the first covering's)
  uint32_t top_xy, top_lev;
};

struct TopSet {
  const uint8_t* top[MULTI];
  const uint32_t* pal[MULTI];
  uint32_t E;
};

// combined top level: the first covering's byte where every covering's cell
// holds the same single polygon (or all hold none), TOP_ASK elsewhere
__global__ void sweep_top_kernel(TopSet t, uint32_t nt, uint8_t* __restrict__ out) {
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nt) return;
  const uint8_t b0 = t.top[0][c];
  uint8_t v = b0;
  if (b0 != TOP_ASK) {
    const uint32_t p0 = b0 < TOP_NONE ? t.pal[0][b0] : 0xFFFFFFFFu;
    for (uint32_t e = 1; e < t.E; ++e) {
      const uint8_t b = t.top[e][c];
      const uint32_t p = b < TOP_NONE ? t.pal[e][b] : (b == TOP_NONE ? 0xFFFFFFFFu : 0xFFFFFFFEu);
      if (p != p0) v = TOP_ASK;
    }
  }
  out[c] = v;
}

// queued cell indices carry the covering in their top two bits (mixed cell
// indices stay below TAB_MIXED_MAX < 2^30)
constexpr uint32_t SWEEP_E_SHIFT = 30;
static_assert(MULTI <= 4 && TAB_MIXED_MAX < (1u << SWEEP_E_SHIFT), "covering bits");

// shared-memory layout of the sweep: the compact cell-id table, the per-warp
// queues, MULTI accumulator sets, then (with a combined top level) its bytes
// and palette
__host__ __device__ constexpr size_t sweep_queue_off() { return HILBERT3_COMPACT_BYTES; }
__host__ __device__ constexpr size_t sweep_acc_off() {
  return sweep_queue_off() + (size_t)(TOP_THREADS / 32) * QCAP * sizeof(QEnt);
}
__host__ __device__ constexpr size_t sweep_top_off(size_t P, bool SUM) {
  return (sweep_acc_off() + MULTI * acc_bytes(P, SUM, false) + 15) & ~(size_t)15;
}

template <int LOOKUP, bool SMEM, bool SUM>
__device__ __forceinline__ void sweep_resolve(QEnt Q, const uint32_t* s_tab,
                                              unsigned char* accb, size_t ab, size_t P,
                                              const JoinArgs* s_args) {
  const uint32_t e = Q.m >> SWEEP_E_SHIFT;
  Q.m &= (1u << SWEEP_E_SHIFT) - 1u;
  resolve_mixed<LOOKUP, SMEM, SUM, false>(Q, s_tab, acc_at<SUM, false>(accb + e * ab, P),
                                          s_args[e]);
}

template <int LOOKUP, bool SMEM, bool SUM>
__global__ __launch_bounds__(TOP_THREADS, TOP_BLOCKS) void sweep_kernel(
    const __grid_constant__ SweepArgs S) {
  extern __shared__ __align__(16) unsigned char smem[];
  // the coverings' arguments, read with a covering index known only at run time
  __shared__ JoinArgs s_args[MULTI];
  constexpr int TPB = TOP_THREADS;
  const JoinArgs& A0 = S.c[0];
  const uint32_t E = S.E;
  const size_t P = SMEM ? A0.P : 0;
  const size_t ab = acc_bytes(P, SUM, false);
  uint32_t* s_tab = reinterpret_cast<uint32_t*>(smem);
  QEnt* s_q = reinterpret_cast<QEnt*>(smem + sweep_queue_off()) + (threadIdx.x >> 5) * QCAP;
  unsigned char* accb = smem + sweep_acc_off();
  uint8_t* s_top = smem + sweep_top_off(P, SUM);
  uint32_t* s_pal = reinterpret_cast<uint32_t*>(s_top + ((size_t)1 << (2 * S.top_lev)));
  hilbert3_fill_compact(s_tab);
  {
    static_assert(sizeof(JoinArgs) % 4 == 0, "word copy");
    const uint32_t* src = reinterpret_cast<const uint32_t*>(S.c);
    uint32_t* dst = reinterpret_cast<uint32_t*>(s_args);
    for (uint32_t i = threadIdx.x; i < E * (sizeof(JoinArgs) / 4); i += TPB) dst[i] = src[i];
  }
  if (S.top) {
    const uint4* src = reinterpret_cast<const uint4*>(S.top);
    uint4* dst = reinterpret_cast<uint4*>(s_top);
    for (uint32_t i = threadIdx.x; i < (1u << (2 * S.top_lev)) / 16; i += TPB) dst[i] = __ldg(src + i);
    for (uint32_t i = threadIdx.x; i < TOP_PALETTE; i += TPB) s_pal[i] = __ldg(S.pal + i);
  }
  if (SMEM)
    for (uint32_t e = 0; e < E; ++e) acc_zero<SUM, false>(acc_at<SUM, false>(accb + e * ab, P), (uint32_t)P);
  __syncthreads();

  const uint32_t lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t qn = 0;  // entries in this warp's queue (warp-uniform)
  const uint32_t gmask = ~((1u << A0.B) - 1u);
  const uint64_t per_tile = (uint64_t)TPB * 4;
  const uint64_t ntiles = (A0.n + per_tile - 1) / per_tile;
  uint32_t since_flush = 0;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint64_t e0 = t * per_tile + (uint64_t)threadIdx.x * 4;
    uint32_t xs[4], ys[4];
    int32_t as[4];
    bool ok[4];
    if (A0.vec && e0 + 3 < A0.n) {
      const uint4 xv = __ldcs(reinterpret_cast<const uint4*>(A0.x + e0));
      const uint4 yv = __ldcs(reinterpret_cast<const uint4*>(A0.y + e0));
      xs[0] = xv.x; xs[1] = xv.y; xs[2] = xv.z; xs[3] = xv.w;
      ys[0] = yv.x; ys[1] = yv.y; ys[2] = yv.z; ys[3] = yv.w;
      if (SUM) {
        const int4 av = __ldcs(reinterpret_cast<const int4*>(A0.attr + e0));
        as[0] = av.x; as[1] = av.y; as[2] = av.z; as[3] = av.w;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) ok[q] = true;
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        ok[q] = e0 + q < A0.n;
        xs[q] = ok[q] ? A0.x[e0 + q] : 0u;
        ys[q] = ok[q] ? A0.y[e0 + q] : 0u;
        as[q] = (SUM && ok[q]) ? A0.attr[e0 + q] : 0;
      }
    }
    if (!SUM) {
#pragma unroll
      for (int q = 0; q < 4; ++q) as[q] = 0;
    }
    // the combined top level: a payload shared by every covering, NONE, or ask
    bool ask[4];
    uint32_t pc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const bool in = ok[q] && !((xs[q] | ys[q]) & gmask);
      const uint8_t v = !in ? TOP_NONE
                            : (S.top ? s_top[((ys[q] >> S.top_xy) << S.top_lev) | (xs[q] >> S.top_xy)]
                                     : TOP_ASK);
      ask[q] = v == TOP_ASK;
      pc[q] = v < TOP_NONE ? s_pal[v] : NONE;
    }
    // covering by covering (a loop the compiler keeps rolled): the table
    // entries of the points the top level did not answer, all four gathers in
    // flight, then the second level; mixed cells go to the queue
#pragma unroll 1
    for (uint32_t e = 0; e < E; ++e) {
      const JoinArgs& A = s_args[e];
      const Acc acc = acc_at<SUM, false>(accb + e * ab, P);
      uint32_t en[4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        en[q] = ask[q] ? __ldg(A.tab + (((ys[q] >> A.txy) << A.tlev) | (xs[q] >> A.txy))) : pc[q];
      if (A.sub) {
        const uint32_t smask = (1u << A.s2) - 1u;
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (ask[q] && en[q] >= TAB_MIXED && en[q] != NONE)
            en[q] = __ldg(A.sub + (((uint64_t)(en[q] & ~TAB_MIXED) << (2 * A.s2)) |
                                   (((ys[q] >> A.txy2) & smask) << A.s2) |
                                   ((xs[q] >> A.txy2) & smask)));
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const bool mix = ask[q] && en[q] >= TAB_MIXED && en[q] != NONE;
        const uint32_t bal = __ballot_sync(FULL, mix);
        if (mix) {
          QEnt& Q = s_q[qn + __popc(bal & lt)];
          Q.x = xs[q];
          Q.y = ys[q];
          Q.m = (en[q] & ~TAB_MIXED) | (e << SWEEP_E_SHIFT);
          Q.a = as[q];
        } else {
          add_pay<SMEM, SUM, false>(en[q], as[q], acc, A);
        }
        qn += __popc(bal);
        if (qn >= 32) {  // a full warp of held-back points: search their windows
          __syncwarp();
          qn -= 32;
          const QEnt Q = s_q[qn + lane];
          __syncwarp();
          sweep_resolve<LOOKUP, SMEM, SUM>(Q, s_tab, accb, ab, P, s_args);
        }
      }
    }
    if (SMEM && ++since_flush == TOP_FLUSH_TILES) {
      since_flush = 0;
      __syncthreads();
      for (uint32_t e = 0; e < E; ++e) flush_acc<SUM, false>(acc_at<SUM, false>(accb + e * ab, P), s_args[e]);
      __syncthreads();
    }
  }
  __syncwarp();  // the rest of the queue
  if (lane < qn) sweep_resolve<LOOKUP, SMEM, SUM>(s_q[lane], s_tab, accb, ab, P, s_args);
  if (SMEM) {
    __syncthreads();
    for (uint32_t e = 0; e < E; ++e) flush_acc<SUM, false>(acc_at<SUM, false>(accb + e * ab, P), s_args[e]);
  }
}

template <int LOOKUP, bool SMEM, bool SUM>
sdb_status launch_sweep_t(const SweepArgs& S, cudaStream_t s) {
  size_t smem = sweep_top_off(SMEM ? S.c[0].P : 0, SUM);
  if (S.top) smem += ((size_t)1 << (2 * S.top_lev)) + 4 * TOP_PALETTE;
  smem = (smem + 15) & ~(size_t)15;
  auto kern = sweep_kernel<LOOKUP, SMEM, SUM>;
  if (smem > 48 * 1024)
    SDB_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  SDB_TRY(occupancy(reinterpret_cast<const void*>(kern), TOP_THREADS, smem, &per_sm));
  SDB_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                    carveout_pct((size_t)per_sm * (smem + sizeof(SweepArgs::c) + 1024))));
  uint64_t blocks = (uint64_t)num_sms() * per_sm;
  const uint64_t need = (S.c[0].n + 4 * TOP_THREADS - 1) / (4 * TOP_THREADS);
  if (blocks > need) blocks = need > 0 ? need : 1;
  TraceScope tr("join", s);
  kern<<<(unsigned)blocks, TOP_THREADS, smem, s>>>(S);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  return SDB_OK;
}

template <bool RANGE>
sdb_status launch_pick(const JoinArgs& A, int lookup, bool has_sum, cudaStream_t s) {
  const bool smem = A.P <= (RANGE ? SMEM_POLYS_RANGE : SMEM_POLYS);
  if (lookup == SDB_LOOKUP_BINARY) {
    if (smem)
      return has_sum ? launch_t<0, true, true, RANGE>(A, s) : launch_t<0, true, false, RANGE>(A, s);
    return has_sum ? launch_t<0, false, true, RANGE>(A, s) : launch_t<0, false, false, RANGE>(A, s);
  }
  if constexpr (!RANGE) {  // the table lookups with the top level in shared memory
    if (A.top && lookup == SDB_LOOKUP_TABLE) {
      if (smem)
        return has_sum ? launch_t<3, true, true, false, true>(A, s)
                       : launch_t<3, true, false, false, true>(A, s);
      return has_sum ? launch_t<3, false, true, false, true>(A, s)
                     : launch_t<3, false, false, false, true>(A, s);
    }
    if (A.top && lookup == SDB_LOOKUP_TABLE_LEARNED) {
      if (smem)
        return has_sum ? launch_t<4, true, true, false, true>(A, s)
                       : launch_t<4, true, false, false, true>(A, s);
      return has_sum ? launch_t<4, false, true, false, true>(A, s)
                     : launch_t<4, false, false, false, true>(A, s);
    }
  }
  if (lookup == SDB_LOOKUP_TABLE) {
    if (smem)
      return has_sum ? launch_t<3, true, true, RANGE>(A, s) : launch_t<3, true, false, RANGE>(A, s);
    return has_sum ? launch_t<3, false, true, RANGE>(A, s) : launch_t<3, false, false, RANGE>(A, s);
  }
  if (lookup == SDB_LOOKUP_TABLE_LEARNED) {
    if (smem)
      return has_sum ? launch_t<4, true, true, RANGE>(A, s) : launch_t<4, true, false, RANGE>(A, s);
    return has_sum ? launch_t<4, false, true, RANGE>(A, s) : launch_t<4, false, false, RANGE>(A, s);
  }
  if (smem)
    return has_sum ? launch_t<1, true, true, RANGE>(A, s) : launch_t<1, true, false, RANGE>(A, s);
  return has_sum ? launch_t<1, false, true, RANGE>(A, s) : launch_t<1, false, false, RANGE>(A, s);
}

}  // namespace

sdb_status launch_join(const uint32_t* x, const uint32_t* y, const int32_t* attr, uint64_t n,
                       const sdb_covering* cov, int lookup, uint64_t* count, int64_t* sum,
                       cudaStream_t s, bool zero, uint64_t* bcount, int64_t* bsum,
                       uint64_t* babs) {
  if (zero) {
    SDB_TRY_CUDA(cudaMemsetAsync(count, 0, (size_t)cov->P * 8, s));
    if (sum) SDB_TRY_CUDA(cudaMemsetAsync(sum, 0, (size_t)cov->P * 8, s));
    if (bcount) SDB_TRY_CUDA(cudaMemsetAsync(bcount, 0, (size_t)cov->P * 8, s));
    if (bsum) SDB_TRY_CUDA(cudaMemsetAsync(bsum, 0, (size_t)cov->P * 8, s));
    if (babs) SDB_TRY_CUDA(cudaMemsetAsync(babs, 0, (size_t)cov->P * 8, s));
    if (lookup == SDB_LOOKUP_LEARNED || lookup == SDB_LOOKUP_TABLE_LEARNED)
      SDB_TRY_CUDA(cudaMemsetAsync(cov->fallbacks, 0, sizeof(unsigned long long), s));
  }
  if (n == 0) return SDB_OK;
  JoinArgs A{};
  A.x = x;
  A.y = y;
  A.attr = attr;
  A.n = n;
  A.count = reinterpret_cast<unsigned long long*>(count);
  A.sum = reinterpret_cast<unsigned long long*>(sum);
  A.vec = ((((uintptr_t)x) | ((uintptr_t)y) | (attr ? (uintptr_t)attr : 0)) & 15u) == 0;
  A.start = cov->start;
  A.pay = cov->pay;
  A.list_off = cov->list_off;
  A.list_ids = cov->list_ids;
  A.sample = cov->sample;
  A.R = cov->R;
  A.sample_n = cov->sample_n;
  A.stride = cov->sample_stride;
  A.B = cov->B;
  A.k = cov->k;
  hilbert3_params(cov->F, &A.nsteps, &A.st0);
  A.P = cov->P;
  A.leaves = cov->leaves;
  A.fence = cov->fence;
  A.knots = cov->knots;
  A.nknots = cov->leaf_bits ? (1u << cov->knot_bits) + 1 : 0;
  A.wshift = cov->knot_wshift;
  A.inv_w = 1.0f / (float)(1ull << cov->knot_wshift);
  A.nleaves = cov->leaf_bits ? (1u << cov->leaf_bits) : 0u;
  A.fallbacks = cov->fallbacks;
  A.tab = cov->tab;
  A.win = cov->sub ? cov->win2 : cov->win;
  A.tlev = cov->tab_bits / 2;
  A.txy = cov->B - A.tlev;
  A.sub = cov->sub;
  A.s2 = cov->sub_bits;
  A.txy2 = A.txy - cov->sub_bits;
  A.top = cov->top;
  A.top_pal = cov->top_pal;
  A.top_lev = cov->top_level;
  A.top_xy = cov->B - cov->top_level;
  A.bcount = reinterpret_cast<unsigned long long*>(bcount);
  A.bsum = reinterpret_cast<unsigned long long*>(bsum);
  A.babs = reinterpret_cast<unsigned long long*>(babs);
  const bool has_sum = sum != nullptr;
  return bcount ? launch_pick<true>(A, lookup, has_sum, s) : launch_pick<false>(A, lookup, has_sum, s);
}

namespace {
// Sec. 6: a conservative raster errs only by false positives, all of them
// points in boundary cells, so the exact COUNT lies in [count - bcount, count]
// and the exact SUM in [sum - pos, sum + neg] with pos = (babs + bsum) / 2 and
// neg = (babs - bsum) / 2 the boundary points' positive and negative attribute
// mass (both exact: babs + bsum and babs - bsum are twice a sum of magnitudes).
__global__ void result_bounds_kernel(const uint64_t* __restrict__ count,
                                     const int64_t* __restrict__ sum,
                                     const uint64_t* __restrict__ bcount,
                                     const int64_t* __restrict__ bsum,
                                     const uint64_t* __restrict__ babs, uint32_t P,
                                     uint64_t* __restrict__ count_lo,
                                     uint64_t* __restrict__ count_hi, int64_t* __restrict__ sum_lo,
                                     int64_t* __restrict__ sum_hi) {
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= P) return;
  const uint64_t c = count[j];
  count_lo[j] = c - bcount[j];
  count_hi[j] = c;
  if (sum) {
    const uint64_t ab = babs[j], bs = (uint64_t)bsum[j];
    const uint64_t pos = (ab + bs) >> 1, neg = (ab - bs) >> 1;  // both < 2^63
    sum_lo[j] = (int64_t)((uint64_t)sum[j] - pos);
    sum_hi[j] = (int64_t)((uint64_t)sum[j] + neg);
  }
}
}  // namespace

sdb_status launch_result_bounds(const uint64_t* count, const int64_t* sum, const uint64_t* bcount,
                                const int64_t* bsum, const uint64_t* babs, uint32_t P,
                                uint64_t* count_lo, uint64_t* count_hi, int64_t* sum_lo,
                                int64_t* sum_hi, cudaStream_t s) {
  if (P == 0) return SDB_OK;
  result_bounds_kernel<<<(P + 255) / 256, 256, 0, s>>>(count, sum, bcount, bsum, babs, P,
                                                       count_lo, count_hi, sum_lo, sum_hi);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  return SDB_OK;
}

namespace {
JoinArgs join_args(const uint32_t* x, const uint32_t* y, const int32_t* attr, uint64_t n,
                   const sdb_covering* cov, uint64_t* count, int64_t* sum) {
  JoinArgs A{};
  A.x = x;
  A.y = y;
  A.attr = attr;
  A.n = n;
  A.count = reinterpret_cast<unsigned long long*>(count);
  A.sum = reinterpret_cast<unsigned long long*>(sum);
  A.vec = ((((uintptr_t)x) | ((uintptr_t)y) | (attr ? (uintptr_t)attr : 0)) & 15u) == 0;
  A.start = cov->start;
  A.pay = cov->pay;
  A.list_off = cov->list_off;
  A.list_ids = cov->list_ids;
  A.sample = cov->sample;
  A.R = cov->R;
  A.sample_n = cov->sample_n;
  A.stride = cov->sample_stride;
  A.B = cov->B;
  A.k = cov->k;
  hilbert3_params(cov->F, &A.nsteps, &A.st0);
  A.P = cov->P;
  A.leaves = cov->leaves;
  A.fence = cov->fence;
  A.knots = cov->knots;
  A.nknots = cov->leaf_bits ? (1u << cov->knot_bits) + 1 : 0;
  A.wshift = cov->knot_wshift;
  A.inv_w = 1.0f / (float)(1ull << cov->knot_wshift);
  A.nleaves = cov->leaf_bits ? (1u << cov->leaf_bits) : 0u;
  A.fallbacks = cov->fallbacks;
  A.tab = cov->tab;
  A.win = cov->sub ? cov->win2 : cov->win;
  A.tlev = cov->tab_bits / 2;
  A.txy = cov->B - A.tlev;
  A.sub = cov->sub;
  A.s2 = cov->sub_bits;
  A.txy2 = A.txy - cov->sub_bits;
  return A;
}
}  // namespace

sdb_status launch_join_multi(const uint32_t* x, const uint32_t* y, const int32_t* attr,
                             uint64_t n, const sdb_covering* const* covs, uint32_t E, int lookup,
                             uint64_t* count, int64_t* sum, cudaStream_t s, bool zero) {
  const uint32_t P = covs[0]->P;
  for (uint32_t e0 = 0; e0 < E; e0 += MULTI) {
    const uint32_t m = std::min<uint32_t>(MULTI, E - e0);
    uint32_t finest = 0;  // the covering with the largest finest level encodes the ids
    for (uint32_t e = 1; e < m; ++e)
      if (covs[e0 + e]->F > covs[e0 + finest]->F) finest = e;
    MultiArgs M{};
    M.E = m;
    for (uint32_t e = 0; e < m; ++e) {
      const sdb_covering* c = covs[e0 + e];
      if (zero) {
        SDB_TRY_CUDA(cudaMemsetAsync(count + (size_t)(e0 + e) * P, 0, (size_t)P * 8, s));
        if (sum) SDB_TRY_CUDA(cudaMemsetAsync(sum + (size_t)(e0 + e) * P, 0, (size_t)P * 8, s));
        if (lookup == SDB_LOOKUP_LEARNED || lookup == SDB_LOOKUP_TABLE_LEARNED)
          SDB_TRY_CUDA(cudaMemsetAsync(c->fallbacks, 0, sizeof(unsigned long long), s));
      }
      M.c[e] = join_args(x, y, attr, n, c, count + (size_t)(e0 + e) * P,
                         sum ? sum + (size_t)(e0 + e) * P : nullptr);
      M.shift[e] = 2 * (covs[e0 + finest]->F - c->F);
    }
    if (lookup == SDB_LOOKUP_TABLE || lookup == SDB_LOOKUP_TABLE_LEARNED) {
      if (n == 0) continue;
      SweepArgs S{};
      S.E = m;
      for (uint32_t e = 0; e < m; ++e) S.c[e] = M.c[e];
      // the combined top level when every covering has one of the same level
      Scratch sc(s);
      bool tops = true;
      for (uint32_t e = 0; e < m; ++e)
        tops = tops && covs[e0 + e]->top && covs[e0 + e]->top_level == covs[e0]->top_level;
      if (tops) {
        const uint32_t Lt = covs[e0]->top_level, nt = 1u << (2 * Lt);
        uint8_t* ctop;
        SDB_TRY(sc.get(&ctop, nt));
        TopSet ts{};
        ts.E = m;
        for (uint32_t e = 0; e < m; ++e) {
          ts.top[e] = covs[e0 + e]->top;
          ts.pal[e] = covs[e0 + e]->top_pal;
        }
        sweep_top_kernel<<<(nt + 255) / 256, 256, 0, s>>>(ts, nt, ctop);
        note_launch();
        SDB_TRY_CUDA(cudaGetLastError());
        S.top = ctop;
        S.pal = covs[e0]->top_pal;
        S.top_lev = Lt;
        S.top_xy = covs[e0]->B - Lt;
      }
      const bool smem = (uint64_t)MULTI * P <= SMEM_POLYS;
      const bool has_sum = sum != nullptr;
      sdb_status st;
      if (lookup == SDB_LOOKUP_TABLE)
        st = smem ? (has_sum ? launch_sweep_t<3, true, true>(S, s) : launch_sweep_t<3, true, false>(S, s))
                  : (has_sum ? launch_sweep_t<3, false, true>(S, s)
                             : launch_sweep_t<3, false, false>(S, s));
      else
        st = smem ? (has_sum ? launch_sweep_t<4, true, true>(S, s) : launch_sweep_t<4, true, false>(S, s))
                  : (has_sum ? launch_sweep_t<4, false, true>(S, s)
                             : launch_sweep_t<4, false, false>(S, s));
      SDB_TRY(st);
      continue;
    }
    // the encoding parameters of the finest covering go with c[0]
    const JoinArgs& Af = M.c[finest];
    M.c[0].k = Af.k;
    M.c[0].nsteps = Af.nsteps;
    M.c[0].st0 = Af.st0;
    if (n == 0) continue;
    const bool smem = (uint64_t)m * P <= SMEM_POLYS;
    const bool has_sum = sum != nullptr;
    sdb_status st;
    if (lookup == SDB_LOOKUP_BINARY)
      st = smem ? (has_sum ? launch_multi_t<0, true, true>(M, s) : launch_multi_t<0, true, false>(M, s))
                : (has_sum ? launch_multi_t<0, false, true>(M, s) : launch_multi_t<0, false, false>(M, s));
    else
      st = smem ? (has_sum ? launch_multi_t<1, true, true>(M, s) : launch_multi_t<1, true, false>(M, s))
                : (has_sum ? launch_multi_t<1, false, true>(M, s) : launch_multi_t<1, false, false>(M, s));
    SDB_TRY(st);
  }
  return SDB_OK;
}

}  // namespace sdb
