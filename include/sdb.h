/*
 * sdb.h - distance-bounded approximate spatial aggregation on the GPU.
 *
 * C ABI of libsdb.so.  The library answers the spatial aggregation query of
 * Sec. 5 of "The Case for Distance-Bounded Spatial Approximations" (CIDR 2021):
 *
 *     SELECT COUNT(*), SUM(a) FROM P, R WHERE P.loc INSIDE R.geometry GROUP BY R.id
 *
 * without any exact geometric test.  Each polygon is replaced by a conservative
 * hierarchical raster (Sec. 2.1, Fig. 1c) whose boundary cells have a diagonal
 * of at most eps (Sec. 2.2), so every point counted for a polygon it does not
 * contain lies within eps of that polygon's boundary, and no contained point is
 * missed.  Cells are linearised with a Hilbert curve and stored as disjoint,
 * sorted id ranges that each carry a polygon list (Sec. 3, "Polygon
 * Indexing"); each point is mapped to its finest-level cell id and looked up
 * (Sec. 3), and the join is fused with the aggregation (Sec. 5.1).
 *
 * Conventions shared by every call:
 *   - Coordinates are unsigned integers on the grid [0, 2^grid_bits)^2,
 *     1 <= grid_bits <= 30.  eps is in grid units.
 *   - A cell is a closed square and a polygon a closed region; a cell belongs to
 *     a polygon's covering when the two intersect (a touch is enough).
 *   - The finest cell side is s = 2^k, the largest power of two with
 *     2 s^2 <= eps^2 (diagonal <= eps); k is capped at grid_bits.  The finest
 *     level is F = grid_bits - k.  A point (x, y) lies in finest cell
 *     (x >> k, y >> k).
 *   - "d_" pointers are device memory owned by the caller; "h_" pointers are
 *     host memory owned by the caller (pinned memory is faster, pageable works).
 *     Nothing the caller passes is retained after the call returns, except that
 *     device work enqueued on cuda_stream reads d_ inputs until it completes.
 *   - cuda_stream is a cudaStream_t (NULL = the legacy default stream).  Device
 *     work is enqueued on it and the call returns without waiting, unless the
 *     call's description says it synchronises.
 *   - Every call returns a status; nothing aborts or throws.  On any status but
 *     SDB_OK the outputs are unspecified and sdb_last_error() describes the
 *     failure (thread-local text).
 *   - Points outside [0, 2^grid_bits)^2 match no polygon.
 */
#ifndef SDB_H
#define SDB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum sdb_status {
  SDB_OK = 0,
  SDB_EINVAL = 1,   /* invalid argument (message in sdb_last_error) */
  SDB_ENOMEM = 2,   /* device or host allocation failed */
  SDB_ECUDA = 3,    /* a CUDA runtime call failed */
  SDB_ETIMEOUT = 4, /* a bounded wait ran out */
  SDB_EBUSY = 5     /* the object is in use (e.g. a batch still running) */
} sdb_status;

/* Covering lookups: binary search over the range starts, the learned index
 * (sdb_covering_build_index), the cell table (sdb_covering_build_table), the
 * cell table as the first level with the learned index searching inside the
 * table's mixed buckets (needs both; the layout of the paper's RadixSpline, a
 * radix table over the key's top bits in front of the model); and, for
 * resident point sets only, the RadixSpline over the sorted point keys. */
enum {
  SDB_LOOKUP_BINARY = 0,
  SDB_LOOKUP_LEARNED = 1,
  SDB_LOOKUP_RADIX_SPLINE = 2,
  SDB_LOOKUP_TABLE = 3,
  SDB_LOOKUP_TABLE_LEARNED = 4
};

/* Polygons in host memory, read during the call only.  One simple ring per
 * polygon (no holes, no self-contact), vertices in [0, 2^grid_bits), either
 * orientation, no closing duplicate vertex.  Polygon j's vertices are
 * x[ring_off[j]] .. x[ring_off[j+1]-1]; the output index of polygon j is j.
 * Simplicity is the caller's responsibility (it is not checked). */
typedef struct sdb_polygons {
  uint32_t n_polygons;      /* P, 1 <= P < 2^26 */
  const uint32_t *ring_off; /* P+1 offsets, ring_off[0] = 0, each ring >= 3 vertices */
  const uint32_t *x;        /* ring_off[P] vertex x coordinates */
  const uint32_t *y;        /* ring_off[P] vertex y coordinates */
} sdb_polygons;

/* Polygons of one or more rings in host memory, read during the call only:
 * multi-polygons and polygons with holes (the paper's neighbourhood regions
 * include multi-polygons, Sec. 5.2).  Polygon j owns rings
 * poly_ring_off[j] .. poly_ring_off[j+1]-1; ring r owns vertices
 * x[ring_off[r]] .. x[ring_off[r+1]-1] (no closing duplicate, either
 * orientation).  The polygon's region is the set of points with an odd
 * crossing number over all of its rings, together with the rings (closed):
 * outer boundaries and holes need no orientation or order.  Rings of one
 * polygon must not cross each other (not checked). */
typedef struct sdb_multipolygons {
  uint32_t n_polygons;           /* P, 1 <= P < 2^26 */
  uint32_t n_rings;              /* >= P */
  const uint32_t *poly_ring_off; /* P+1, poly_ring_off[0] = 0, each polygon >= 1 ring,
                                    poly_ring_off[P] = n_rings */
  const uint32_t *ring_off;      /* n_rings+1, ring_off[0] = 0, each ring >= 3 vertices */
  const uint32_t *x;             /* ring_off[n_rings] vertex coordinates */
  const uint32_t *y;
} sdb_multipolygons;

/* Opaque device-resident covering (library-owned device memory). */
typedef struct sdb_covering sdb_covering;

typedef struct sdb_covering_info {
  uint32_t grid_bits;      /* B */
  uint32_t finest_shift;   /* k: finest side 2^k */
  uint32_t finest_level;   /* F = B - k */
  uint32_t n_polygons;     /* P */
  uint64_t n_ranges;       /* R: ranges partition [0, 4^F) */
  uint64_t n_list_ids;     /* total length of all polygon lists */
  uint64_t n_cells;        /* raster cells emitted before merging into ranges */
  uint64_t device_bytes;   /* device memory held by the covering */
  uint32_t index_leaf_bits;/* leaves = 2^index_leaf_bits, 0 = no learned index */
  uint32_t boundary_flags; /* 1 if built with SDB_COVER_BOUNDARY_FLAGS */
  uint32_t table_bits;     /* cell table: 2^table_bits buckets (0: no table, or F = 0) */
  uint64_t table_mixed;    /* buckets of the cell table that hold several ranges */
  uint32_t table_sub_bits; /* second level: 2^s x 2^s sub-cells per mixed bucket (0: none) */
  uint64_t table_sub_mixed;/* sub-cells that hold several ranges */
  uint32_t index_root_bits;/* learned index root: 2^index_root_bits segments (0: one line) */
} sdb_covering_info;

/* Finest level for (grid_bits, eps), Sec. 2.2 (side eps/sqrt(2), so the
 * diagonal is eps; the side is rounded down to a power of two so cells nest
 * in the quadtree).  Host only.  SDB_EINVAL if grid_bits is outside 1..30 or
 * eps < 2 (no side s >= 1 has diagonal <= eps). */
sdb_status sdb_finest_level(uint32_t grid_bits, uint64_t eps, uint32_t *shift_out,
                            uint32_t *level_out);

/* Build the conservative hierarchical raster covering of every polygon
 * (Sec. 2.1-2.2, Sec. 3 "Polygon Indexing"): per polygon, quadtree cells from
 * the whole grid down; a cell that meets no edge and lies inside is emitted
 * whole (interior cell, any level); a cell that meets an edge is split until
 * the finest level and emitted there (boundary cell); all other cells are
 * dropped.  Each emitted cell becomes the Hilbert-id range of its finest-level
 * descendants; the ranges of all polygons are merged into maximal disjoint
 * ranges partitioning [0, 4^F), each with its ascending, duplicate-free polygon
 * list (possibly empty).
 *
 * Synchronises cuda_stream (the per-level frontier sizes are read on the host).
 * *out receives a new covering to be released with sdb_covering_free.
 * SDB_EINVAL: bad grid_bits/eps (see sdb_finest_level), P = 0 or P >= 2^26,
 * a ring with < 3 vertices, a vertex outside the grid, a null pointer.
 * SDB_ENOMEM: device memory ran out. */
sdb_status sdb_build_covering(const sdb_polygons *polys, uint32_t grid_bits, uint64_t eps,
                              void *cuda_stream, sdb_covering **out);

/* Result range estimation (Sec. 6): errors of a conservative raster occur only
 * in boundary cells, so counting the points that fall in a polygon's boundary
 * cells bounds the exact answer.  With SDB_COVER_BOUNDARY_FLAGS every list
 * entry is polygon | 1 << 31 when the range lies in boundary cells of that
 * polygon (finest-level cells meeting its boundary) and polygon otherwise
 * (interior cells); ranges are maximal for the flagged lists, so a covering has
 * at least as many ranges as the plain one.  Stripping the flags and merging
 * equal neighbours gives exactly the plain covering.  Every join accepts a
 * flagged covering; sdb_join_aggregate_range requires one. */
#define SDB_COVER_BOUNDARY_FLAGS 1u

/* Non-conservative raster (Sec. 2.2: boundary cells with a small overlap may
 * be omitted, trading false positives for false negatives): a finest-level
 * boundary cell is kept only when its centre lies in the closed polygon;
 * interior cells are kept as always.  Every answer error still lies within
 * eps of the boundary.  Not combinable with SDB_COVER_BOUNDARY_FLAGS (the
 * result-range interval assumes a conservative raster). */
#define SDB_COVER_NONCONSERVATIVE 2u

/* sdb_build_covering with options: flags = 0, SDB_COVER_BOUNDARY_FLAGS or
 * SDB_COVER_NONCONSERVATIVE.  SDB_EINVAL as sdb_build_covering, an unknown flag
 * bit, or both flags together. */
sdb_status sdb_build_covering_ex(const sdb_polygons *polys, uint32_t grid_bits, uint64_t eps,
                                 uint32_t flags, void *cuda_stream, sdb_covering **out);

/* The coverings of the same polygons at n_eps distance bounds, built together
 * in one level-synchronous pass (an eps sweep, as in the paper's experiments):
 * out[i] receives the covering for eps[i], identical to what
 * sdb_build_covering_ex(polys, grid_bits, eps[i], flags) returns, each to be
 * released with sdb_covering_free.  Polygons that overlap one another are
 * built one eps at a time.  Synchronises cuda_stream.  SDB_EINVAL: as
 * sdb_build_covering_ex, NULL eps/out, n_eps outside 1..64.  On failure no
 * covering is returned. */
sdb_status sdb_build_coverings(const sdb_polygons *polys, uint32_t grid_bits, const uint64_t *eps,
                               uint32_t n_eps, uint32_t flags, void *cuda_stream,
                               sdb_covering **out);

/* sdb_build_covering_ex for polygons of several rings (holes, multi-polygons):
 * a cell is a boundary cell of polygon j when it meets any of j's rings, an
 * interior cell when it meets none and lies in j's even-odd region.  The
 * covering is used like any other.  SDB_EINVAL as sdb_build_covering_ex, a
 * polygon without rings, a ring with < 3 vertices, inconsistent offsets. */
sdb_status sdb_build_covering_multi(const sdb_multipolygons *polys, uint32_t grid_bits,
                                    uint64_t eps, uint32_t flags, void *cuda_stream,
                                    sdb_covering **out);

sdb_status sdb_covering_get_info(const sdb_covering *cov, sdb_covering_info *info);

/* Fit the learned range index (Sec. 3, "Point Indexing": a learned model
 * predicts a key's position in the sorted array, after RadixSpline): a root
 * maps a cell id to one of 2^leaf_bits leaves, each leaf a linear model in FP32
 * on leaf-relative ids, plus the leaf's maximum prediction error below and
 * above, measured with the same FP32 arithmetic the lookup uses over every id
 * the root sends to that leaf, and the fences of the range starts (every 16th
 * start, which the lookup searches before the starts).  The root is piecewise linear in FP32 over
 * 2^root_bits equal segments of [0, 4^F): at each segment end it takes the
 * fraction of range starts below that id (the starts' cumulative distribution,
 * so leaves receive about equal numbers of ranges); root_bits = 0 is a single
 * root line from 0 to 4^F (the plain two-level model).  The fit (least squares
 * per leaf) runs on the device.  Replaces a previous index.  Synchronises
 * cuda_stream.  sdb_covering_build_index uses SDB_INDEX_ROOT_BITS_DEFAULT.
 * SDB_EINVAL: leaf_bits outside 4..20, root_bits above SDB_INDEX_ROOT_BITS_MAX. */
#define SDB_INDEX_ROOT_BITS_DEFAULT 12u
#define SDB_INDEX_ROOT_BITS_MAX 12u
sdb_status sdb_covering_build_index(sdb_covering *cov, uint32_t leaf_bits, void *cuda_stream);
sdb_status sdb_covering_build_index_ex(sdb_covering *cov, uint32_t leaf_bits, uint32_t root_bits,
                                       void *cuda_stream);

/* Build the cell table: a direct-mapped first level of a radix tree over the
 * finest cell ids (the role of ACT's upper levels in Sec. 3, "Polygon
 * Indexing": cells of large interior ranges are resolved at once).  With
 * T = min(table_bits rounded down to even, 2F) the ids [0, 4^F) fall into 2^T
 * buckets of 4^F / 2^T consecutive ids, the descendants of one cell of level
 * T / 2 each.  The table lists those cells in row-major order, so a point's
 * entry follows from its coordinates without encoding its cell id.  A bucket that lies inside one range stores that range's
 * polygon payload, so a point in it needs one table read; a bucket that meets
 * several ranges stores the first and last of them, and the lookup binary
 * searches that window of range starts.  A second level (the tree's next
 * levels) splits every mixed bucket into s x s sub-cells, s = 2^min(3, F - T/2),
 * stored the same way, so a point in a mixed bucket makes one more read and
 * searches only inside a sub-cell that meets several ranges.  Table: 4 bytes
 * per bucket, 8 per mixed bucket, 4 s^2 per mixed bucket for the second level
 * and 8 per mixed sub-cell.  Replaces a previous table.  Synchronises
 * cuda_stream.  SDB_EINVAL: table_bits outside 8..26, or R >= 2^30 - 1. */
sdb_status sdb_covering_build_table(sdb_covering *cov, uint32_t table_bits, void *cuda_stream);

/* Index-nested-loop join fused with COUNT and SUM (Sec. 5.1): for each point i
 * with finest cell id h, the range r with start[r] <= h < start[r+1] is found
 * (lookup = SDB_LOOKUP_BINARY: binary search over the range starts;
 * SDB_LOOKUP_LEARNED: the learned index's prediction, a search bounded by the
 * stored error window (first over the index's fences, every 16th range start,
 * then inside one fence's block), verified, with binary search as the fallback;
 * requires sdb_covering_build_index; SDB_LOOKUP_TABLE: the cell table's bucket, then a
 * binary search of the bucket's window if it holds several ranges; requires
 * sdb_covering_build_table; SDB_LOOKUP_TABLE_LEARNED: the cell table's bucket,
 * and in a bucket of several ranges -- when its window holds more than 64 of
 * them -- the learned index's error window cut to the bucket's window, searched
 * and verified, with the bucket's window as the counted fallback; requires
 * both), and for every polygon j on r's list
 * d_count[j] += 1 and d_sum[j] += d_attr[i].  All three lookups give
 * identical results.  d_count and d_sum (P entries each) are zeroed by the call.
 * d_x, d_y, d_attr: n device values (SoA).  d_attr and d_sum may be NULL
 * (COUNT only).  n = 0 just zeroes the outputs.  Asynchronous.
 * SDB_EINVAL: null cov/d_count, n > 0 with null d_x/d_y, n > 0 with d_sum but no
 * d_attr, a lookup whose index or table was not built. */
sdb_status sdb_join_aggregate(const uint32_t *d_x, const uint32_t *d_y, const int32_t *d_attr,
                              uint64_t n, const sdb_covering *cov, int lookup,
                              uint64_t *d_count, int64_t *d_sum, void *cuda_stream);

/* sdb_join_aggregate plus the result-range partials of Sec. 6, on a covering
 * built with SDB_COVER_BOUNDARY_FLAGS: for every polygon j on the range of
 * point i where j is flagged, d_bcount[j] += 1, d_bsum[j] += d_attr[i] and
 * d_babs[j] += |d_attr[i]|.  With a conservative raster the exact answers lie in
 *   COUNT: [d_count - d_bcount, d_count]
 *   SUM:   [d_sum - (d_babs + d_bsum) / 2, d_sum + (d_babs - d_bsum) / 2]
 * (the false positives are a subset of the boundary points; (d_babs + d_bsum)/2
 * and (d_bsum - d_babs)/2 are their positive and negative parts).  All output
 * arrays have P entries, are zeroed by the call and are device memory;
 * d_sum, d_bsum and d_babs are given together or all NULL (COUNT only).
 * Asynchronous.  SDB_EINVAL: as sdb_join_aggregate, a null d_bcount, a covering
 * without boundary flags, or only some of d_sum / d_bsum / d_babs. */
sdb_status sdb_join_aggregate_range(const uint32_t *d_x, const uint32_t *d_y,
                                    const int32_t *d_attr, uint64_t n, const sdb_covering *cov,
                                    int lookup, uint64_t *d_count, int64_t *d_sum,
                                    uint64_t *d_bcount, int64_t *d_bsum, uint64_t *d_babs,
                                    void *cuda_stream);

/* The result ranges of Sec. 6 ("the exact answer lies in [alpha - beta,
 * alpha]") from the partials of sdb_join_aggregate_range, computed on the
 * device: for every polygon j < n_polygons
 *   d_count_lo[j] = d_count[j] - d_bcount[j],  d_count_hi[j] = d_count[j],
 *   d_sum_lo[j] = d_sum[j] - (d_babs[j] + d_bsum[j]) / 2,
 *   d_sum_hi[j] = d_sum[j] + (d_babs[j] - d_bsum[j]) / 2
 * (exact integers: the false positives of a conservative raster are a subset
 * of the boundary points, whose positive and negative attribute parts are the
 * two halves).  All arrays are device memory of n_polygons entries owned by
 * the caller; the five sum arrays are given together or all NULL (COUNT only).
 * Asynchronous on cuda_stream.  SDB_EINVAL: a NULL count array, or only some of
 * the sum arrays. */
sdb_status sdb_result_bounds(const uint64_t *d_count, const int64_t *d_sum,
                             const uint64_t *d_bcount, const int64_t *d_bsum,
                             const uint64_t *d_babs, uint32_t n_polygons, uint64_t *d_count_lo,
                             uint64_t *d_count_hi, int64_t *d_sum_lo, int64_t *d_sum_hi,
                             void *cuda_stream);

/* sdb_join_aggregate for n_covs coverings of the same polygons on the same grid
 * (an eps sweep) in one pass over the points: each point is read once.  With
 * the binary or learned lookup its cell id is computed once, at the finest
 * level among the coverings (a coarser id is its prefix), then looked up in
 * every covering.  With the table lookups (SDB_LOOKUP_TABLE,
 * SDB_LOOKUP_TABLE_LEARNED; every covering needs its cell table, and the
 * learned one its index) a combined top level -- the cells whose payload is
 * the same single polygon in every covering -- answers a point for all
 * coverings with one shared-memory read, and the other points go through each
 * covering's table in turn.  d_count and d_sum hold n_covs rows of P entries
 * (row c for covs[c]), zeroed by the call; results equal n_covs separate
 * sdb_join_aggregate calls.  Asynchronous.
 * SDB_EINVAL: as sdb_join_aggregate, a NULL covering, coverings that differ in
 * polygon count or grid bits, n_covs = 0, a covering without the table or
 * index its lookup needs. */
sdb_status sdb_join_aggregate_multi(const uint32_t *d_x, const uint32_t *d_y,
                                    const int32_t *d_attr, uint64_t n,
                                    const sdb_covering *const *covs, uint32_t n_covs, int lookup,
                                    uint64_t *d_count, int64_t *d_sum, void *cuda_stream);

/* The same join for points in host memory against n_covs coverings at once
 * (e.g. the same polygons at several eps).  Points are streamed to the device
 * in chunks; each chunk is joined against every covering while the next chunk
 * is copied.  All coverings must have the same n_polygons P.  h_count and h_sum
 * are host arrays of n_covs * P entries (covering c's results at [c*P, c*P+P)).
 * Synchronises cuda_stream before returning (results are in host memory).
 * Device staging buffers are allocated and freed by the call. */
sdb_status sdb_join_aggregate_host(const uint32_t *h_x, const uint32_t *h_y, const int32_t *h_attr,
                                   uint64_t n, const sdb_covering *const *covs, uint32_t n_covs,
                                   int lookup, uint64_t *h_count, int64_t *h_sum,
                                   void *cuda_stream);

/* Allocation-free variant of sdb_join_aggregate_host for one covering.  The paper
 * has no counterpart: this serves callers that cannot allocate device memory
 * while they call in -- services that reserve their whole device-memory budget
 * when they start and must not allocate afterwards, and plugins inside a
 * process whose own allocator owns the device and forbids allocations made
 * behind its back.
 *
 * Staging buffers and per-polygon accumulators live in one file-scope device
 * array of SDB_NOALLOC_CHUNK * 12 + SDB_NOALLOC_MAX_POLYGONS * 16 bytes (13 MiB)
 * that every GPU which loads the library holds until the process exits.  The
 * call makes no cudaMalloc/cudaFree or other allocating call; it streams the
 * points SDB_NOALLOC_CHUNK at a time on cuda_stream alone and synchronises it
 * before returning (results in h_count/h_sum, P entries each).  Each call
 * looks up the array's device address in the current context
 * (cudaGetSymbolAddress, which allocates nothing), so calls after a
 * cudaDeviceReset find the reloaded array.  Every call shares the array and clears the accumulators itself; calls whose GPU work
 * overlaps (other streams or threads) race on it.
 * SDB_EINVAL: more than SDB_NOALLOC_MAX_POLYGONS polygons, and the argument
 * errors of sdb_join_aggregate_host. */
#define SDB_NOALLOC_CHUNK (1u << 20)
#define SDB_NOALLOC_MAX_POLYGONS (1u << 16)
sdb_status sdb_join_aggregate_host_noalloc(const uint32_t *h_x, const uint32_t *h_y,
                                           const int32_t *h_attr, uint64_t n,
                                           const sdb_covering *cov, int lookup, uint64_t *h_count,
                                           int64_t *h_sum, void *cuda_stream);

/* Bounded Raster Join (Sec. 5.2), restated on device buffers without a
 * graphics API: the points are blended into a uniform canvas whose pixels are
 * the finest cells of eps (each pixel keeps the COUNT and SUM of its points),
 * every polygon is rasterised conservatively onto the same pixels (a pixel is
 * masked in when the closed pixel meets the closed polygon; exact integer
 * scanline rasterisation), and the masked pixels' aggregates are summed per
 * polygon.  No covering and no precomputation; the result equals
 * sdb_join_aggregate with a covering of the same polygons and eps.  The canvas
 * of 4^F pixels is processed in tiles of 2^tile_bits x 2^tile_bits pixels
 * (0 = 2^13), as many at a time as fit in 8 GiB (16 bytes per pixel), so the
 * cost grows with the canvas: quadratically as eps shrinks.
 * polys: host arrays as for sdb_build_covering; d_x, d_y, d_attr: n device
 * points (d_attr and d_sum may be NULL); d_count, d_sum: P device entries,
 * zeroed by the call.  Synchronises cuda_stream.
 * SDB_EINVAL: as sdb_build_covering, NULL outputs or coordinates, n >= 2^32,
 * tile_bits > 14, more than 2^16 tiles (finest level - tile_bits > 8), or a
 * polygon row whose rasterisation needs more than 128 spans or crossings.
 * SDB_ENOMEM: device memory ran out. */
sdb_status sdb_raster_join(const sdb_polygons *polys, uint32_t grid_bits, uint64_t eps,
                           const uint32_t *d_x, const uint32_t *d_y, const int32_t *d_attr,
                           uint64_t n, uint32_t tile_bits, uint64_t *d_count, int64_t *d_sum,
                           void *cuda_stream);

/* sdb_raster_join for polygons of several rings (the crossings of all rings
 * decide the interior; every ring's edges mark boundary pixels). */
sdb_status sdb_raster_join_multi(const sdb_multipolygons *polys, uint32_t grid_bits, uint64_t eps,
                                 const uint32_t *d_x, const uint32_t *d_y, const int32_t *d_attr,
                                 uint64_t n, uint32_t tile_bits, uint64_t *d_count,
                                 int64_t *d_sum, void *cuda_stream);

/* ---------------------------------------------------------------------------
 * Batched level-of-detail queries (Sec. 1: users explore at several levels of
 * detail, an overview first, then zooms into regions of interest).  A query is
 * an axis-aligned viewport [x0, x1) x [y0, y1), a subset of the polygons and a
 * distance bound eps; it asks, for each polygon of the subset, COUNT and SUM of
 * the points inside the viewport whose finest cell (at the query's eps) meets
 * the polygon -- the eps-bounded join of sdb_join_aggregate restricted to the
 * viewport and the subset.
 * ------------------------------------------------------------------------- */

/* A resident point set on the device, ordered by full-resolution Hilbert id so
 * a viewport is a few contiguous index ranges.  Library-owned copy. */
typedef struct sdb_points sdb_points;

/* Copy n device points (SoA; d_attr may be NULL = zeros) into a resident set.
 * Synchronises cuda_stream.  SDB_EINVAL: grid_bits outside 1..30, n = 0 or
 * n >= 2^32, NULL coordinates, a point outside the grid. */
sdb_status sdb_points_create(const uint32_t *d_x, const uint32_t *d_y, const int32_t *d_attr,
                             uint64_t n, uint32_t grid_bits, void *cuda_stream, sdb_points **out);
void sdb_points_free(sdb_points *pts);

/* ---------------------------------------------------------------------------
 * Point-indexed aggregation (Sec. 3, "Point Indexing"): the points' cells are
 * linearised by the same curve at full resolution and kept as a sorted array
 * (the resident set above); a polygon's covering ranges select contiguous
 * slices of it, so per covering range COUNT = ub - lb and SUM = prefix[ub] -
 * prefix[lb] with lb / ub the lower bounds of the range's first id and of the
 * next range's first id, both scaled to full resolution (<< 2 * finest_shift).
 * The results equal sdb_join_aggregate on the same points exactly.
 * ------------------------------------------------------------------------- */

/* Build the point index: int64 prefix sums of the attribute in key order and
 * a RadixSpline over the distinct keys (the paper's learned index, with radix
 * bits 25 and spline error 32 in its experiments): spline points such that
 * linear interpolation between consecutive ones is within spline_error of every
 * key's first position (greedy spline corridor, exact integer slopes, built in
 * independent chunks of 4096 keys), and a table of 2^radix_bits + 1 entries
 * giving, per prefix of the key range, the first spline point at or above it.
 * Replaces a previous index.  Synchronises cuda_stream.
 * SDB_EINVAL: NULL pts, radix_bits outside 1..30, spline_error outside
 * 1..2^20, another current device.  SDB_ENOMEM: device memory ran out. */
sdb_status sdb_points_build_index(sdb_points *pts, uint32_t radix_bits, uint32_t spline_error,
                                  void *cuda_stream);

/* COUNT and SUM per polygon of cov over the resident points by range counting:
 * one lower-bound lookup per range boundary (lookup = SDB_LOOKUP_BINARY: binary
 * search over the keys; SDB_LOOKUP_RADIX_SPLINE: radix table -> spline segment
 * -> exact integer interpolation -> search within +-(spline_error + 1), the
 * bracket verified, binary search as the counted fallback), then the slice's
 * length and prefix-sum difference added to every polygon on the range's list.
 * d_count, d_sum (P device entries; d_sum may be NULL) are zeroed by the call.
 * Asynchronous.  SDB_EINVAL: NULL pts/cov/d_count, another lookup, grid bits of
 * cov and pts differ, SUM or the spline requested before sdb_points_build_index,
 * objects on another device. */
sdb_status sdb_points_aggregate(const sdb_points *pts, const sdb_covering *cov, int lookup,
                                uint64_t *d_count, int64_t *d_sum, void *cuda_stream);

/* Spline diagnostics: number of spline points, the largest interpolation error
 * over all distinct keys (measured on the device; <= spline_error by
 * construction) and the fallbacks of the last spline aggregation.
 * Synchronises cuda_stream.  SDB_EINVAL: NULL arguments, no index. */
sdb_status sdb_points_index_stats(const sdb_points *pts, uint64_t *n_spline, uint64_t *max_error,
                                  uint64_t *fallbacks, void *cuda_stream);

typedef struct sdb_query {
  uint32_t x0, y0, x1, y1; /* viewport, half-open, inside the grid, non-empty */
  uint64_t eps;            /* distance bound in grid units (>= 2) */
  uint32_t poly_off;       /* the subset is subset_ids[poly_off .. poly_off + poly_cnt) */
  uint32_t poly_cnt;       /* its output slot i holds polygon subset_ids[poly_off + i] */
} sdb_query;

typedef struct sdb_batch sdb_batch;

typedef struct sdb_batch_info {
  uint32_t n_queries;
  uint32_t n_pairs;        /* (query, polygon) pairs that can reach their viewport */
  uint64_t out_len;        /* sum of poly_cnt: length of the output arrays */
  uint64_t n_ranges;       /* covering ranges over all queries */
  uint64_t max_ranges;     /* largest covering of one query */
  uint64_t n_cells;        /* raster cells emitted before merging */
  uint64_t candidates;     /* points in the viewports' candidate index ranges */
  uint64_t n_tiles;        /* work items of the persistent launch */
  uint32_t tile;           /* points per work item */
  uint32_t points_per_thread;
  uint32_t lookup;         /* SDB_LOOKUP_BINARY or SDB_LOOKUP_LEARNED */
  uint32_t indexed_queries;/* queries searched through their learned index */
  uint64_t n_leaves;       /* learned leaves over all queries */
} sdb_batch_info;

enum { SDB_BATCH_PERSISTENT = 0, SDB_BATCH_PER_QUERY = 1, SDB_BATCH_GRAPH = 2 };

/* Prepare a batch: every query's covering (the conservative raster of its
 * subset at its eps, cells restricted to those holding viewport points; all
 * queries in one level-synchronous pass), the viewport's candidate point
 * ranges, and the work list.  polygons/queries/subset_ids are host arrays read
 * during the call; pts must outlive the batch.  Output slices: query q's
 * results are entries [off_q, off_q + poly_cnt_q) of the output arrays, off_q
 * the sum of the preceding queries' poly_cnt.  Synchronises cuda_stream.
 * SDB_EINVAL: bad viewport/eps/subset, polygons that overlap inside one query
 * (batched coverings assume disjoint polygons, e.g. a tiling). */
sdb_status sdb_batch_create(const sdb_points *pts, const sdb_polygons *polys,
                            const sdb_query *queries, uint32_t n_queries,
                            const uint32_t *subset_ids, uint64_t n_subset_ids, void *cuda_stream,
                            sdb_batch **out);
sdb_status sdb_batch_get_info(const sdb_batch *b, sdb_batch_info *info);
/* Covering ranges of every query (host array of n_queries). */
sdb_status sdb_batch_query_ranges(const sdb_batch *b, uint32_t *h_ranges);

/* Run all queries into d_count / d_sum (out_len device entries each, zeroed by
 * the call; d_sum may be NULL).  mode SDB_BATCH_PERSISTENT: one persistent
 * launch whose blocks pull (query, point tile) work items from a device
 * counter; SDB_BATCH_PER_QUERY: one launch per query; SDB_BATCH_GRAPH: the
 * persistent launch captured once into a CUDA graph (per output pointers) and
 * replayed -- needs a created stream, not the legacy default stream.  All modes
 * give identical results.  Asynchronous. */
sdb_status sdb_batch_run(sdb_batch *b, int mode, uint64_t *d_count, int64_t *d_sum,
                         void *cuda_stream);

/* Lookup of later runs (sdb_batch_run, sdb_batch_autotune).  SDB_LOOKUP_BINARY
 * (the default): binary search over each query's ranges.  SDB_LOOKUP_LEARNED
 * (Sec. 3, learned index): every query covering of at least
 * SDB_BATCH_LEARNED_MIN_RANGES ranges gets a two-level model fitted on the
 * device -- a linear root over the span of its range starts picking one of up
 * to 2^16 leaves (about SDB_BATCH_RANGES_PER_LEAF ranges each), each leaf an
 * FP32 least-squares line with the largest prediction errors below and above
 * measured by the lookup's own arithmetic; a point searches its leaf's error
 * window, the result is verified and binary search over the query's ranges is
 * the counted fallback, so results are identical to binary search.  Smaller
 * coverings keep binary search.  Synchronises cuda_stream.  SDB_EINVAL: another
 * lookup. */
#define SDB_BATCH_LEARNED_MIN_RANGES 64u
#define SDB_BATCH_RANGES_PER_LEAF 8u
sdb_status sdb_batch_set_lookup(sdb_batch *b, int lookup, void *cuda_stream);
/* Learned searches of the most recent run that fell back to binary search.
 * Synchronises cuda_stream. */
sdb_status sdb_batch_fallbacks(const sdb_batch *b, void *cuda_stream, uint64_t *out);

/* Autotuner: times the persistent launch on this batch for tiles of 1024,
 * 4096, 16384 points and 1, 2, 4 points per thread, keeps the fastest.
 * Synchronises cuda_stream. */
sdb_status sdb_batch_autotune(sdb_batch *b, void *cuda_stream, uint32_t *tile_out,
                              uint32_t *ppt_out);
/* Set the tile size (>= 1) and points per thread (1, 2 or 4) directly. */
sdb_status sdb_batch_set_tuning(sdb_batch *b, uint32_t tile, uint32_t points_per_thread,
                                void *cuda_stream);
void sdb_batch_free(sdb_batch *b);

/* ---------------------------------------------------------------------------
 * Serving (Sec. 1: interactive exploration needs fast answers while users zoom):
 * points stay resident; queries arrive at any time and are answered by
 * continuous batching.  A pool of workers, each with its own CUDA stream, takes
 * every pending query (up to max_batch) as one batch whenever a worker is free,
 * so queries arriving while other batches run join the next free slot and the
 * batches overlap on the device.  Per query a viewport-clipped covering comes
 * from a device-memory cache (LRU under cache_bytes; coverings of running
 * batches are pinned) or is built with the batch's other missing queries in one
 * pass; a worker takes new work only while the coverings of running batches fit
 * cache_bytes.  Each batch's join is one persistent launch, or one launch per
 * query in the plain form (per_query = 1), searching each query's ranges by
 * binary search or, with lookup = SDB_LOOKUP_LEARNED, through a learned index
 * fitted to the batch's coverings (sdb_batch_set_lookup).  Results are the same as the batch
 * API's for the same query, alone or in any mix.
 * ------------------------------------------------------------------------- */
typedef struct sdb_server sdb_server;

typedef struct sdb_server_config {
  uint32_t workers;           /* batches in flight, one stream each, 1..64 */
  uint32_t max_batch;         /* queries per batch, >= 1 */
  uint64_t cache_bytes;       /* device-memory budget for coverings */
  uint32_t use_cache;         /* 0: every query's covering is built afresh */
  uint32_t per_query;         /* 1: one launch per query instead of one per batch */
  uint32_t tile;              /* points per work item, 0 = default */
  uint32_t points_per_thread; /* 1, 2, 4, or 0 = default */
  uint32_t lookup;            /* SDB_LOOKUP_BINARY (0) or SDB_LOOKUP_LEARNED: each batch
                                 fits the learned index of sdb_batch_set_lookup */
} sdb_server_config;

typedef struct sdb_ticket_info {
  double latency_ms;  /* submit until the result is in host memory */
  double queue_ms;    /* submit until a worker took the query */
  uint32_t batch_size;
  uint32_t cache_hit; /* the covering came from the cache */
  uint64_t ranges;    /* covering ranges of the query */
} sdb_ticket_info;

typedef struct sdb_server_stats {
  uint64_t submitted, completed, batches;
  uint64_t cache_hits, cache_misses, evictions;
  uint64_t cache_bytes, cache_entries, peak_bytes;
} sdb_server_stats;

/* Start the workers.  pts must outlive the server; polygons are copied.
 * SDB_EINVAL: bad config or polygons, points on another device. */
sdb_status sdb_server_create(const sdb_points *pts, const sdb_polygons *polys,
                             const sdb_server_config *cfg, sdb_server **out);
/* Queue one query (q->poly_off is ignored: subset_ids holds its q->poly_cnt
 * polygon ids; both are copied).  Returns at once with a ticket.
 * SDB_EINVAL: bad viewport, eps or polygon id; SDB_EBUSY: shutting down. */
sdb_status sdb_server_submit(sdb_server *srv, const sdb_query *q, const uint32_t *subset_ids,
                             uint64_t *ticket);
/* Wait up to timeout_ms for a ticket; on success copy its poly_cnt counts and
 * sums to host arrays (either may be NULL) and the timing to info (nullable),
 * and retire the ticket.  SDB_ETIMEOUT: not done yet (the ticket stays valid);
 * SDB_EINVAL: unknown or retired ticket; otherwise the batch's own status. */
sdb_status sdb_server_wait(sdb_server *srv, uint64_t ticket, uint32_t timeout_ms,
                           uint64_t *h_count, int64_t *h_sum, sdb_ticket_info *info);
sdb_status sdb_server_get_stats(sdb_server *srv, sdb_server_stats *stats);
/* Finish every queued query, stop the workers, free the cache.  Tickets not
 * yet waited for are discarded. */
void sdb_server_destroy(sdb_server *srv);

/* Number of learned-index lookups of the covering's most recent learned join
 * (SDB_LOOKUP_LEARNED or SDB_LOOKUP_TABLE_LEARNED) whose bounded search missed
 * and fell back to binary search.  Synchronises cuda_stream. */
sdb_status sdb_covering_fallbacks(const sdb_covering *cov, void *cuda_stream, uint64_t *out);

/* Learned-index window sizes (errlo + errhi + 1 per leaf): mean weighted by the
 * ranges each leaf spans, and maximum.  Zeros without an index.  Synchronous. */
sdb_status sdb_covering_index_stats(const sdb_covering *cov, double *mean_window,
                                    uint32_t *max_window);

/* Copy the canonical covering to host memory: start[R+1] (start[0] = 0,
 * start[R] = 4^F, strictly increasing), list_off[R+1], list_ids[n_list_ids];
 * range r holds finest ids [start[r], start[r+1]) and polygons
 * list_ids[list_off[r] .. list_off[r+1]-1], ascending.  Adjacent ranges have
 * different lists.  Synchronous.  Array sizes come from sdb_covering_get_info. */
sdb_status sdb_covering_export(const sdb_covering *cov, uint64_t *h_start, uint32_t *h_list_off,
                               uint32_t *h_list_ids);

/* Release a covering (waits for the device to finish with it).  NULL is a no-op. */
void sdb_covering_free(sdb_covering *cov);

const char *sdb_status_string(sdb_status s);
const char *sdb_last_error(void);

/* Number of CUDA kernels this library has launched in this process so far (all
 * devices, all threads).  A diagnostic counter; host only, never fails. */
uint64_t sdb_launch_count(void);

/* Device memory of the library's stream-ordered pool on the current device:
 * bytes handed out and not yet freed (used) and bytes the pool holds from the
 * driver (reserved; freed blocks are kept for reuse).  Diagnostics; host only.
 * SDB_EINVAL: a NULL output. */
sdb_status sdb_memory_stats(uint64_t *pool_used, uint64_t *pool_reserved);

/* Device time of the library's phases (diagnostics).  While tracing is on, each
 * traced phase records a CUDA event before and after its work on the stream it
 * runs on: "cover.build" (a whole covering build), "cover.expand" (one level of
 * the quadtree expansion), "cover.merge" (record sort and range merge, made
 * of "cover.sort", "cover.count" and "cover.emit"),
 * "sort.hist", "sort.scan", "sort.scatter" (one 8-bit pass of the record sort
 * each), "index.build", "table.build", "join" (one join launch).  Time spent
 * by the host between launches falls inside the enclosing phases only.
 * sdb_trace_enable(1) drops earlier records and starts recording; (0) stops.
 * sdb_trace_read waits for the recorded events and writes, per phase name in
 * order of first appearance, the number of intervals and their total time in
 * ms (at most capacity entries; *n_out = the number of names).  Host only;
 * calls racing with traced library calls in other threads are not supported.
 * SDB_EINVAL: n_out NULL, or out NULL with capacity > 0. */
typedef struct sdb_trace_stat {
  char name[32];
  uint64_t count;
  double total_ms;
} sdb_trace_stat;
sdb_status sdb_trace_enable(int on);
sdb_status sdb_trace_read(sdb_trace_stat *out, uint32_t capacity, uint32_t *n_out);

#ifdef __cplusplus
}
#endif

#endif /* SDB_H */
