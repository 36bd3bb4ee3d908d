// Internal definitions shared by the libsdb.so translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "sdb.h"

namespace sdb {

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
sdb_status cuda_status(cudaError_t e, const char* what, const char* file, int line);

#define SDB_TRY_CUDA(call)                                                     \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess) return ::sdb::cuda_status(e_, #call, __FILE__, __LINE__); \
  } while (0)

#define SDB_TRY(call)                   \
  do {                                  \
    sdb_status s_ = (call);             \
    if (s_ != SDB_OK) return s_;        \
  } while (0)

// ---------------------------------------------------------------- memory
// Stream-ordered allocations from a library-owned pool (one per device) that
// keeps freed blocks cached, so repeated builds do not pay for cudaMalloc.
sdb_status dalloc(void** p, size_t bytes, cudaStream_t s);
void dfree(void* p, cudaStream_t s);

template <class T>
sdb_status dalloc_n(T** p, size_t n, cudaStream_t s) {
  return dalloc(reinterpret_cast<void**>(p), (n ? n : 1) * sizeof(T), s);
}

// RAII holder for temporaries of one call (freed on the call's stream).
struct Scratch {
  cudaStream_t s;
  void* ptrs[64];
  int n = 0;
  explicit Scratch(cudaStream_t st) : s(st) {}
  ~Scratch() {
    for (int i = 0; i < n; ++i) dfree(ptrs[i], s);
  }
  template <class T>
  sdb_status get(T** p, size_t count) {
    if (n >= 64) {
      set_error("internal: scratch slots exhausted");
      return SDB_ENOMEM;
    }
    SDB_TRY(dalloc_n(p, count, s));
    ptrs[n++] = *p;
    return SDB_OK;
  }
  // release one early (must have come from this scratch)
  void release(void* p) {
    for (int i = 0; i < n; ++i)
      if (ptrs[i] == p) {
        dfree(p, s);
        ptrs[i] = ptrs[--n];
        return;
      }
  }
};

// shared-memory carveout (percent of the SM's maximum shared memory, rounded up)
// that holds the given bytes of resident blocks' shared memory
int carveout_pct(size_t bytes);
// resident blocks per SM of kernel kern (at least 1) with the given threads and
// dynamic shared memory, independent of the carveout a previous launch chose
sdb_status occupancy(const void* kern, int threads, size_t smem, int* per_sm);
int num_sms();

// count of kernels this library has launched in the process (all devices)
void note_launch();

// Diagnostics: while tracing is on (sdb_trace_enable), a scope records a CUDA
// event pair around its work on stream s, filed under name (a string literal).
struct TraceScope {
  int slot = -1;
  cudaStream_t s;
  TraceScope(const char* name, cudaStream_t s);
  ~TraceScope() { end(); }
  void end();  // records the closing event now (once)
  TraceScope(const TraceScope&) = delete;
  TraceScope& operator=(const TraceScope&) = delete;
};

// ---------------------------------------------------------------- Hilbert curve
// Quadrant-digit Hilbert curve whose order-1 visit order is (0,0), (0,1), (1,1),
// (1,0).  Scanning levels from the top, the orientation inherited by the lower
// levels is one of four symmetries of the square: identity, transpose,
// anti-transpose, rotation by 180 degrees.  They form a Klein four-group, so the
// orientation is two bits (swap, complement) and composing orientations is XOR.
// Under orientation (sw, cm) the raw bits (xb, yb) of a level read as
//   xt = (sw ? yb : xb) ^ cm,  yt = (sw ? xb : yb) ^ cm,
// the level's digit is 2*xt + (xt ^ yt), and quadrant (0,0) contributes a
// transpose (sw ^= 1) while quadrant (1,0) contributes an anti-transpose
// (sw ^= 1, cm ^= 1).
__host__ __device__ inline uint64_t hilbert_id(uint32_t x, uint32_t y, uint32_t order) {
  uint64_t d = 0;
  uint32_t sw = 0, cm = 0;
  for (int lev = (int)order - 1; lev >= 0; --lev) {
    uint32_t xb = (x >> lev) & 1u, yb = (y >> lev) & 1u;
    uint32_t xt = (sw ? yb : xb) ^ cm, yt = (sw ? xb : yb) ^ cm;
    d = (d << 2) | ((xt << 1) | (xt ^ yt));
    if (!yt) {
      sw ^= 1u;
      cm ^= xt;
    }
  }
  return d;
}

// ---------------------------------------------------------------- covering
// One leaf of the learned range index, 32 bytes (one DRAM sector).  The leaf
// receives the ids h in [base, next leaf's base); its ranges are first..last.
// Prediction: first + floor(fma(a, float(h - base), b)) in FP32, clamped into
// [first, last] (monotone, and no extrapolation across a long last range); the
// true range lies in [pred - errlo, pred + errhi] for every id the leaf receives.
struct LeafRec {
  uint64_t base;
  float a, b;
  uint32_t first, last;
  int32_t errlo, errhi;
};
static_assert(sizeof(LeafRec) == 32, "leaf records are read as one 32-byte load");

__device__ __forceinline__ int64_t leaf_predict(const LeafRec& l, uint64_t h) {
  const float x = __ull2float_rn(h - l.base);
  const float pos = __fmaf_rn(l.a, x, l.b);
  int64_t p = (int64_t)l.first + (int64_t)__float2ll_rd(pos);
  p = p < (int64_t)l.first ? (int64_t)l.first : p;
  return p > (int64_t)l.last ? (int64_t)l.last : p;
}

// Root of the learned index: a piecewise-linear approximation of the ranges'
// cumulative distribution over the id space, in leaf units.  Knot j sits at
// id j << wshift and holds knot[j] = L * (#range starts below it) / R; between
// knots the value is interpolated in FP32.  The map is monotone in h (each
// piece is non-decreasing and ends at the next knot's value), so every leaf
// receives one contiguous interval of ids.
__device__ __forceinline__ uint32_t root_leaf(const float* knot, uint32_t wshift, float inv_w,
                                              uint32_t nleaves, uint64_t h) {
  const uint32_t j = (uint32_t)(h >> wshift);
  const uint64_t rem = h - ((uint64_t)j << wshift);
  const float k0 = knot[j], k1 = knot[j + 1];
  // k0 <= pos <= k1 by construction (the min guards one-ulp overshoot of the
  // rounded slope), so the map is monotone across knots as well
  const float pos =
      fminf(__fmaf_rn(k1 - k0, __fmul_rn(__ull2float_rn(rem), inv_w), k0), k1);
  int v = __float2int_rd(pos);
  v = v < 0 ? 0 : v;
  return (uint32_t)v >= nleaves ? nleaves - 1 : (uint32_t)v;
}

// Fences of the learned index: every 2^FENCE_SHIFT-th range start, so that a
// window search first narrows the window to one 128-byte line of starts
// through the (cache-resident) fences.
constexpr uint32_t FENCE_SHIFT = 4;

}  // namespace sdb

struct sdb_covering {
  int device = 0;
  uint32_t B = 0, k = 0, F = 0, P = 0;
  bool flagged = false;  // list entries and pay carry boundary flags
  uint64_t R = 0, nids = 0, ncells = 0;
  // canonical form
  uint64_t* start = nullptr;     // R+1
  uint32_t* list_off = nullptr;  // R+1
  uint32_t* list_ids = nullptr;  // nids
  // lookup acceleration
  uint32_t* pay = nullptr;       // R: 0xFFFFFFFF empty, <2^31 single polygon, else 2^31|r
  uint64_t* sample = nullptr;    // sample_n keys start[j * sample_stride]
  uint32_t sample_n = 0, sample_stride = 1;
  // learned index
  uint32_t leaf_bits = 0;
  uint32_t knot_bits = 0, knot_wshift = 0; // root: 2^knot_bits + 1 knots, spacing 2^knot_wshift ids
  float* knots = nullptr;                  // root knots (leaf units)
  sdb::LeafRec* leaves = nullptr;          // 2^leaf_bits
  uint64_t* fence = nullptr;               // start[j << FENCE_SHIFT], j = 0 .. R >> FENCE_SHIFT
  unsigned long long* fallbacks = nullptr; // device counter
  // cell table (table.cu): 2^tab_bits buckets of 2^tab_shift ids
  uint32_t* tab = nullptr;  // payload, or TAB_MIXED | index into win
  uint2* win = nullptr;     // first and last range of each mixed bucket
  uint32_t tab_bits = 0, tab_shift = 0;
  uint64_t tab_mixed = 0;
  // the table's second level: every mixed bucket split into 2^sub_bits x
  // 2^sub_bits sub-cells (row-major), each a payload or TAB_MIXED | index into
  // win2 (sub_bits = 0: no second level)
  uint32_t* sub = nullptr;
  uint2* win2 = nullptr;
  uint32_t sub_bits = 0;
  uint64_t sub_mixed = 0;
  // the tree's top level, small enough for shared memory: 4^top_level cells of
  // level top_level, row-major, 1 byte each (TOP_ASK: consult the table,
  // TOP_NONE: no polygon, else an index into top_pal, the single-polygon
  // payloads of the level's cells, at most TOP_PALETTE of them, the most
  // frequent first); top == nullptr: none
  uint8_t* top = nullptr;
  uint32_t* top_pal = nullptr;
  uint32_t top_level = 0;
  size_t bytes = 0;
};

// resident point set ordered by full-resolution Hilbert id (batch.cu)
struct sdb_points {
  int device = 0;
  uint32_t B = 0;
  uint64_t n = 0;
  uint64_t* key = nullptr;
  uint32_t* x = nullptr;
  uint32_t* y = nullptr;
  int32_t* attr = nullptr;
  // point index (sdb_points_build_index): prefix sums and a RadixSpline
  int64_t* prefix = nullptr;  // n + 1
  uint64_t* rs_key = nullptr;
  uint32_t* rs_pos = nullptr;
  uint32_t* rs_table = nullptr;  // 2^rs_radix_bits + 1
  unsigned long long* rs_fallbacks = nullptr;
  uint64_t rs_n = 0, rs_min = 0, rs_max = 0;
  uint32_t rs_radix_bits = 0, rs_error = 0, rs_shift = 0;
};

namespace sdb {

// api.cu ---------------------------------------------------------------------
// Polygons as edge sets: polygon j owns edges [edge_off[j], edge_off[j+1]) and
// edge v runs from vertex v to vertex next[v], the following vertex of its
// ring.  A polygon of several rings (outer boundaries and holes) is the
// even-odd region of all its edges.
struct PolyEdges {
  uint32_t P = 0, V = 0;
  const uint32_t* x = nullptr;  // caller-owned vertex arrays
  const uint32_t* y = nullptr;
  std::vector<uint32_t> edge_off;
  std::vector<uint32_t> next;
};
PolyEdges poly_edges(const sdb_polygons* p);
PolyEdges poly_edges(const sdb_multipolygons* p);
sdb_status validate_polygons(const sdb_polygons* polys, uint32_t grid_bits);
sdb_status validate_multipolygons(const sdb_multipolygons* polys, uint32_t grid_bits);

// raster.cu ------------------------------------------------------------------
// Bounded Raster Join: counts (and sums, when sum != nullptr) per polygon over
// a canvas of 2^(B-k) x 2^(B-k) pixels, cut into tiles of 2^tile_bits pixels a
// side, as many tiles at once as fit in budget_bytes (16 bytes per pixel).
sdb_status raster_join(const PolyEdges& pe, uint32_t B, uint32_t k, const uint32_t* x,
                       const uint32_t* y, const int32_t* attr, uint64_t n, uint32_t tile_bits,
                       uint64_t budget_bytes, uint64_t* count, int64_t* sum, cudaStream_t s);

// pointindex.cu --------------------------------------------------------------
sdb_status build_point_index(sdb_points* p, uint32_t radix_bits, uint32_t spline_error,
                             cudaStream_t s);
void release_point_index(sdb_points* p, cudaStream_t s);
sdb_status point_index_aggregate(const sdb_points* p, const sdb_covering* cov, int lookup,
                                 uint64_t* count, int64_t* sum, cudaStream_t s);
sdb_status point_index_stats(const sdb_points* p, uint64_t* n_spline, uint64_t* max_error,
                             uint64_t* fallbacks, cudaStream_t s);

// cover.cu -------------------------------------------------------------------
// Several coverings can be built in one level-synchronous pass.  Query q covers
// the polygons of its (query, polygon) pairs at finest level F, keeping only
// cells that hold lattice points of its box [x0, x1) x [y0, y1); each pair's
// polygon is reported under the pair's slot id.  A single covering is one
// query over the whole grid whose slots are the polygon ids.
struct CoverQuery {
  uint32_t F, x0, y0, x1, y1;
};
struct CoverSpec {
  uint32_t B = 0;
  uint32_t Q = 0;
  const CoverQuery* q = nullptr;        // host, Q entries
  uint32_t NP = 0;                      // pairs
  const uint32_t* pair_poly = nullptr;  // host, NP entries each
  const uint32_t* pair_query = nullptr;
  const uint32_t* pair_slot = nullptr;
  bool flags = false;    // boundary flags on list entries (result range, Sec. 6)
  bool noncons = false;  // finest boundary cells kept only when their centre is inside
};
// Result, device arrays from the library pool.  Query q's ranges are entries
// [qoff[q], qoff[q+1] - 1) of start/list_off/pay; entry qoff[q+1] - 1 is a
// sentinel with start 4^F and an empty list, so list_off[i+1] - list_off[i] is
// the length of range i's list for every range.
struct CoverSet {
  uint64_t* start = nullptr;     // E
  uint32_t* list_off = nullptr;  // E
  uint32_t* list_ids = nullptr;  // nids (slot ids)
  uint32_t* pay = nullptr;       // E: empty / single slot / 2^31 | entry index
  uint64_t E = 0, nids = 0, ncells = 0;
  std::vector<uint64_t> qoff;    // host, Q + 1
  std::vector<uint64_t> qcells;  // host, raster cells (records) of each query
  void release(cudaStream_t s);
};
sdb_status build_coverings(const PolyEdges& pe, const CoverSpec& spec, cudaStream_t s,
                           CoverSet* out);
// options: SDB_COVER_BOUNDARY_FLAGS, SDB_COVER_NONCONSERVATIVE
sdb_status build_covering_device(const PolyEdges& pe, uint32_t B, uint32_t k, uint32_t options,
                                 cudaStream_t s, sdb_covering* cov);
// several finest shifts ks[0..nq) of the same polygons in one level-synchronous
// pass (one covering per shift, as build_covering_device would make it);
// polygons that overlap fall back to one pass per shift
sdb_status build_coverings_multi(const PolyEdges& pe, uint32_t B, const uint32_t* ks, uint32_t nq,
                                 uint32_t options, cudaStream_t s, sdb_covering* const* covs);
// batch.cu ------------------------------------------------------------------
// Per-query parameters of a batched join, and the covering arrays a query's
// slice lives in (one chunk may serve many queries).
struct BatchQueryDev {
  uint64_t sbase;  // first entry of the query's covering slice in its chunk
  uint32_t R;      // ranges in the slice (the sentinel follows)
  uint32_t chunk;
  uint32_t k, nsteps, st0;
  uint32_t x0, y0, x1, y1;
  uint32_t out_off;
  // learned index of the slice (nleaves = 0: binary search): ids below llo lie
  // in range 0, ids from lhi on in range R - 1; between them leaf
  // min(nleaves - 1, (h - llo) >> lwshift) of the batch's leaf array, from loff
  uint32_t nleaves, loff, lwshift;
  uint32_t npoly;  // output slots of the query (its subset's size)
  uint64_t llo, lhi;
};
struct BatchChunkDev {
  const uint64_t* start;
  const uint32_t* pay;
  const uint32_t* list_off;
  const uint32_t* list_ids;
};
struct BatchTile {
  uint32_t q, begin, end, pad;
};
// Everything a batched join needs besides the coverings themselves.
struct BatchCore {
  const sdb_points* pts = nullptr;
  // learned lookup (batch_core_index): per-query leaves, fallback counter
  bool learned = false;
  LeafRec* leaves = nullptr;
  uint64_t nleaves = 0;
  uint32_t indexed = 0;  // queries with leaves
  unsigned long long* fallbacks = nullptr;
  uint32_t Q = 0;
  uint64_t out_len = 0, candidates = 0;
  std::vector<BatchQueryDev> hq;
  std::vector<BatchChunkDev> hchunks;
  BatchQueryDev* dq = nullptr;
  BatchChunkDev* dchunks = nullptr;
  uint32_t* cand = nullptr;   // per query up to 81 candidate point index ranges
  uint32_t* ncand = nullptr;
  uint32_t tile = 4096, ppt = 2;
  BatchTile* tiles = nullptr;
  uint64_t ntiles = 0;
  std::vector<uint64_t> qtile;  // host, Q + 1: tiles of query q
  unsigned long long* heads = nullptr;  // Q + 1 work counters
  void release(cudaStream_t s);
};
// viewport, level and output slot of one query (sbase/R/chunk left to the caller)
sdb_status batch_query_dev(uint32_t B, const sdb_query& q, uint64_t out_off, BatchQueryDev* d,
                           uint32_t* F_out);
// upload hq/hchunks, candidate ranges, work list (candidate counts computed)
sdb_status batch_core_prepare(BatchCore* c, cudaStream_t s);
sdb_status batch_core_tiles(BatchCore* c, uint32_t T, cudaStream_t s);
// mode SDB_BATCH_PERSISTENT or SDB_BATCH_PER_QUERY; outputs cleared first
// fit the per-query learned index of every query with at least min_ranges
// ranges (about ranges_per_leaf ranges per leaf, at most 2^16 leaves a query)
sdb_status batch_core_index(BatchCore* c, uint32_t min_ranges, uint32_t ranges_per_leaf,
                            cudaStream_t s);
sdb_status batch_core_run(BatchCore* c, int mode, uint64_t* count, int64_t* sum, cudaStream_t s);
// coverings for queries cq (pairs in query order), chunked; fills sbase/R/chunk
// of hq with chunk indices starting at chunk_base
sdb_status build_query_coverings(const PolyEdges& pe, uint32_t B,
                                 const std::vector<CoverQuery>& cq,
                                 const std::vector<uint32_t>& pp, const std::vector<uint32_t>& pq,
                                 const std::vector<uint32_t>& ps, std::vector<BatchQueryDev>& hq,
                                 std::vector<CoverSet>* sets, uint32_t chunk_base,
                                 cudaStream_t s, uint64_t* n_ranges, uint64_t* n_cells,
                                 uint64_t* max_ranges);
// pairs of query q whose polygon (bounding boxes bb, 4 per polygon) can reach
// its viewport at finest shift k; ids = the query's subset
void viewport_pairs(const std::vector<uint32_t>& bb, uint32_t q, const sdb_query& Qu, uint32_t k,
                    const uint32_t* ids, std::vector<uint32_t>& pp, std::vector<uint32_t>& pq,
                    std::vector<uint32_t>& ps);
sdb_status polygon_bboxes(const sdb_polygons* polys, uint32_t B, std::vector<uint32_t>* bb);

// learned.cu
sdb_status build_learned_index(sdb_covering* cov, uint32_t leaf_bits, uint32_t root_bits,
                               cudaStream_t s);

// cell table entries: a range payload, or TAB_MIXED | m for the m-th bucket that
// meets several ranges (m < TAB_MIXED_MAX - 1; payload values 2^31 | r need
// r < 2^30 - 1, so the two never collide)
constexpr uint32_t TAB_MIXED = 0xC0000000u;
// top-level entries: an index into the level's palette of payloads, or one of these
constexpr uint8_t TOP_ASK = 0xFFu;
constexpr uint8_t TOP_NONE = 0xFEu;
constexpr uint32_t TOP_PALETTE = 254;  // palette slots (indices 0 .. 253)
constexpr uint32_t TOP_MAX_LEVEL = 8;  // 4^8 cells, 64 KB of shared memory
constexpr uint32_t TAB_MIXED_MAX = 0x3fffffffu;
// Sec. 6 intervals from the range join's partials (join.cu)
sdb_status launch_result_bounds(const uint64_t* count, const int64_t* sum, const uint64_t* bcount,
                                const int64_t* bsum, const uint64_t* babs, uint32_t P,
                                uint64_t* count_lo, uint64_t* count_hi, int64_t* sum_lo,
                                int64_t* sum_hi, cudaStream_t s);
sdb_status build_cell_table(sdb_covering* cov, uint32_t table_bits, cudaStream_t s);
// A covering record's value: polygon slot (bits 0..25), level above the finest
// (26..30), boundary flag (31).  Packed record (one 64-bit word, sb slot bits):
// key << (sb + 6) | flag << (sb + 5) | level << sb | slot.
__host__ __device__ inline uint64_t record_pack(uint64_t key, uint32_t val, uint32_t sb) {
  return (key << (sb + 6)) | ((uint64_t)(val >> 31) << (sb + 5)) |
         ((uint64_t)((val >> 26) & 31u) << sb) | (uint64_t)(val & ((1u << 26) - 1u));
}
__host__ __device__ inline uint32_t record_val(uint64_t w, uint32_t sb) {
  return (uint32_t)(w & ((1ull << sb) - 1ull)) | ((uint32_t)((w >> sb) & 31u) << 26) |
         ((uint32_t)((w >> (sb + 5)) & 1u) << 31);
}

// lookup is known and the covering has what it needs (api.cu)
sdb_status check_lookup(const sdb_covering* cov, int lookup);
// join.cu
// zero = true: outputs (and the fallback counter) are cleared first;
// zero = false: the launch adds into them (chunked joins)
// one pass over the points for E coverings of the same polygons and grid;
// count / sum hold E rows of P entries (row e for covs[e])
sdb_status launch_join_multi(const uint32_t* x, const uint32_t* y, const int32_t* attr,
                             uint64_t n, const sdb_covering* const* covs, uint32_t E, int lookup,
                             uint64_t* count, int64_t* sum, cudaStream_t s, bool zero);
// bcount / bsum / babs (nullable; the covering must be flagged): result-range
// partials of Sec. 6 (boundary count, boundary attribute sum, sum of magnitudes)
sdb_status launch_join(const uint32_t* x, const uint32_t* y, const int32_t* attr, uint64_t n,
                       const sdb_covering* cov, int lookup, uint64_t* count, int64_t* sum,
                       cudaStream_t s, bool zero, uint64_t* bcount = nullptr,
                       int64_t* bsum = nullptr, uint64_t* babs = nullptr);

// sort.cu: device-wide primitives
template <class T>
sdb_status exclusive_scan(const T* in, T* out, size_t n, T* d_total, cudaStream_t s);
// keys-only LSD sort of packed covering records (record_pack) on their key
// bits [first_bit, first_bit + bits); the result is split into keys
// (*keys_out, one of keys / tmp) and standard values (vals_out)
sdb_status radix_sort_split(uint64_t* keys, uint64_t* tmp, size_t n, int bits, int first_bit,
                            uint32_t sb, uint32_t* vals_out, cudaStream_t s, uint64_t** keys_out);
// keys-only LSD sort on bits [first_bit, first_bit + bits) (stable)
sdb_status radix_sort_keys(uint64_t* keys, uint64_t* tmp, size_t n, int bits, cudaStream_t s,
                           uint64_t** result, int first_bit = 0);
sdb_status radix_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* ktmp, uint32_t* vtmp,
                            size_t n, int bits, cudaStream_t s, uint64_t** kres, uint32_t** vres);
// unique of a sorted array: writes out[0..m), returns m via host sync
sdb_status unique_sorted(const uint64_t* in, size_t n, uint64_t* out, size_t* m, cudaStream_t s);

inline unsigned grid_for(size_t n, unsigned block) {
  size_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > 0x7fffffffu) g = 0x7fffffffu;
  return (unsigned)g;
}

}  // namespace sdb
