// C ABI entry points of libsdb.so (declared in include/sdb.h).  Host-side
// argument checks, the per-device memory pool, covering lifetime, and the
// host-buffer join that streams point chunks through the device.
#include "sdb_internal.cuh"

#include <atomic>
#include <cstring>
#include <mutex>
#include <string>

namespace sdb {

namespace {
thread_local char g_err[512] = "";
std::mutex g_mu;
cudaMemPool_t g_pool[64];
bool g_pool_ok[64];
int g_sms[64];
std::atomic<unsigned long long> g_launches{0};
}  // namespace

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace {
struct TraceRec {
  const char* name;
  cudaEvent_t a, b;
};
std::mutex g_tmu;
std::atomic<bool> g_trace_on{false};
std::vector<TraceRec> g_trace;
std::vector<cudaEvent_t> g_evpool;

cudaEvent_t take_event() {
  if (!g_evpool.empty()) {
    cudaEvent_t e = g_evpool.back();
    g_evpool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}
}  // namespace

TraceScope::TraceScope(const char* name, cudaStream_t st) : s(st) {
  if (!g_trace_on.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(g_tmu);
  TraceRec r{name, take_event(), take_event()};
  if (!r.a || !r.b || cudaEventRecord(r.a, s) != cudaSuccess) {
    cudaGetLastError();
    if (r.a) g_evpool.push_back(r.a);
    if (r.b) g_evpool.push_back(r.b);
    return;
  }
  slot = (int)g_trace.size();
  g_trace.push_back(r);
}

void TraceScope::end() {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_tmu);
  if ((size_t)slot < g_trace.size() && cudaEventRecord(g_trace[slot].b, s) != cudaSuccess) {
    cudaGetLastError();
    g_trace[slot].name = nullptr;
  }
  slot = -1;
}

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

sdb_status cuda_status(cudaError_t e, const char* what, const char* file, int line) {
  set_error("%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  return e == cudaErrorMemoryAllocation ? SDB_ENOMEM : SDB_ECUDA;
}

static sdb_status get_pool(cudaMemPool_t* pool) {
  int dev = 0;
  SDB_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("device %d out of range", dev);
    return SDB_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_pool_ok[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    SDB_TRY_CUDA(cudaMemPoolCreate(&g_pool[dev], &props));
    // keep freed blocks for reuse by later calls of this process
    uint64_t keep = ~0ull;
    SDB_TRY_CUDA(cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep));
    g_pool_ok[dev] = true;
  }
  *pool = g_pool[dev];
  return SDB_OK;
}

sdb_status dalloc(void** p, size_t bytes, cudaStream_t s) {
  cudaMemPool_t pool;
  SDB_TRY(get_pool(&pool));
  cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, s);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    set_error("device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    return SDB_ENOMEM;
  }
  return SDB_OK;
}

void dfree(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

int num_sms() {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 1;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_sms[dev]) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    g_sms[dev] = n > 0 ? n : 1;
  }
  return g_sms[dev];
}

sdb_status occupancy(const void* kern, int threads, size_t smem, int* per_sm) {
  // the occupancy calculator honours the kernel's preferred carveout, which
  // the previous launch may have set for a smaller footprint: ask with the
  // whole unified memory available to shared memory
  SDB_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                    (int)cudaSharedmemCarveoutMaxShared));
  SDB_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, threads, smem));
  if (*per_sm < 1) *per_sm = 1;
  return SDB_OK;
}

int carveout_pct(size_t bytes) {
  int dev = 0, max_smem = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
          cudaSuccess ||
      max_smem <= 0) {
    cudaGetLastError();
    return -1;  // no preference
  }
  const size_t pct = (bytes * 100 + (size_t)max_smem - 1) / (size_t)max_smem;
  return pct > 100 ? 100 : (int)pct;
}

static sdb_status finest(uint32_t B, uint64_t eps, uint32_t* k_out) {
  if (B < 1 || B > 30) {
    set_error("grid_bits %u outside 1..30", B);
    return SDB_EINVAL;
  }
  if (eps < 2) {
    set_error("eps %llu < 2: no cell side >= 1 has a diagonal <= eps", (unsigned long long)eps);
    return SDB_EINVAL;
  }
  // largest k with 2 * (2^k)^2 <= eps^2
  unsigned __int128 e2 = (unsigned __int128)eps * eps;
  uint32_t k = 0;
  while (k < B && ((unsigned __int128)2 << (2 * (k + 1))) <= e2) ++k;
  *k_out = k;
  return SDB_OK;
}

static void free_covering(sdb_covering* c) {
  if (!c) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  void* ps[] = {c->start,  c->list_off, c->list_ids, c->pay,    c->sample,
                c->leaves, c->knots,    c->fallbacks, c->tab,   c->win,
                c->sub,    c->win2,     c->top,       c->top_pal, c->fence};
  for (void* p : ps)
    if (p) cudaFreeAsync(p, 0);
  cudaStreamSynchronize(0);
  cudaSetDevice(prev);
  delete c;
}

static sdb_status check_device(const sdb_covering* cov) {
  int dev = 0;
  SDB_TRY_CUDA(cudaGetDevice(&dev));
  if (dev != cov->device) {
    set_error("covering lives on device %d, current device is %d", cov->device, dev);
    return SDB_EINVAL;
  }
  return SDB_OK;
}

sdb_status check_lookup(const sdb_covering* cov, int lookup) {
  if (lookup != SDB_LOOKUP_BINARY && lookup != SDB_LOOKUP_LEARNED && lookup != SDB_LOOKUP_TABLE &&
      lookup != SDB_LOOKUP_TABLE_LEARNED) {
    set_error("unknown lookup %d", lookup);
    return SDB_EINVAL;
  }
  if (lookup == SDB_LOOKUP_LEARNED && !cov->leaves) {
    set_error("learned lookup requested but the covering has no index");
    return SDB_EINVAL;
  }
  if (lookup == SDB_LOOKUP_TABLE_LEARNED && (!cov->tab || !cov->leaves)) {
    set_error("table + learned lookup requested but the covering lacks %s",
              !cov->tab ? "a cell table" : "a learned index");
    return SDB_EINVAL;
  }
  if (lookup == SDB_LOOKUP_TABLE && !cov->tab) {
    set_error("table lookup requested but the covering has no cell table");
    return SDB_EINVAL;
  }
  return SDB_OK;
}

sdb_status check_cover_flags(uint32_t flags) {
  if (flags & ~(SDB_COVER_BOUNDARY_FLAGS | SDB_COVER_NONCONSERVATIVE)) {
    set_error("unknown covering flags 0x%x", flags);
    return SDB_EINVAL;
  }
  if ((flags & SDB_COVER_BOUNDARY_FLAGS) && (flags & SDB_COVER_NONCONSERVATIVE)) {
    set_error("boundary flags need a conservative covering");
    return SDB_EINVAL;
  }
  return SDB_OK;
}

sdb_status new_covering(const PolyEdges& pe, uint32_t grid_bits, uint32_t k, uint32_t flags,
                        cudaStream_t s, sdb_covering** out) {
  sdb_covering* cov = new (std::nothrow) sdb_covering();
  if (!cov) {
    set_error("host allocation failed");
    return SDB_ENOMEM;
  }
  if (cudaGetDevice(&cov->device) != cudaSuccess) {
    delete cov;
    set_error("no CUDA device");
    return SDB_ECUDA;
  }
  sdb_status st = build_covering_device(pe, grid_bits, k, flags, s, cov);
  if (st != SDB_OK) {
    std::string msg = sdb_last_error();
    free_covering(cov);
    set_error("%s", msg.c_str());
    return st;
  }
  *out = cov;
  return SDB_OK;
}

PolyEdges poly_edges(const sdb_polygons* p) {
  PolyEdges e;
  e.P = p->n_polygons;
  e.V = p->ring_off[e.P];
  e.x = p->x;
  e.y = p->y;
  e.edge_off.assign(p->ring_off, p->ring_off + e.P + 1);
  e.next.resize(e.V);
  for (uint32_t j = 0; j < e.P; ++j)
    for (uint32_t v = p->ring_off[j]; v < p->ring_off[j + 1]; ++v)
      e.next[v] = v + 1 < p->ring_off[j + 1] ? v + 1 : p->ring_off[j];
  return e;
}

PolyEdges poly_edges(const sdb_multipolygons* p) {
  PolyEdges e;
  e.P = p->n_polygons;
  e.V = p->ring_off[p->n_rings];
  e.x = p->x;
  e.y = p->y;
  e.edge_off.resize(e.P + 1);
  for (uint32_t j = 0; j <= e.P; ++j) e.edge_off[j] = p->ring_off[p->poly_ring_off[j]];
  e.next.resize(e.V);
  for (uint32_t r = 0; r < p->n_rings; ++r)
    for (uint32_t v = p->ring_off[r]; v < p->ring_off[r + 1]; ++v)
      e.next[v] = v + 1 < p->ring_off[r + 1] ? v + 1 : p->ring_off[r];
  return e;
}

sdb_status validate_multipolygons(const sdb_multipolygons* p, uint32_t grid_bits) {
  if (!p || !p->poly_ring_off || !p->ring_off || !p->x || !p->y) {
    set_error("polygons or one of their arrays is NULL");
    return SDB_EINVAL;
  }
  const uint32_t P = p->n_polygons, R = p->n_rings;
  if (P == 0 || P >= (1u << 26) || R < P) {
    set_error("n_polygons %u outside 1..2^26-1 or fewer rings (%u)", P, R);
    return SDB_EINVAL;
  }
  if (p->poly_ring_off[0] != 0 || p->poly_ring_off[P] != R || p->ring_off[0] != 0) {
    set_error("offsets must start at 0 and poly_ring_off[P] must equal n_rings");
    return SDB_EINVAL;
  }
  for (uint32_t j = 0; j < P; ++j)
    if (p->poly_ring_off[j + 1] <= p->poly_ring_off[j]) {
      set_error("polygon %u has no ring", j);
      return SDB_EINVAL;
    }
  for (uint32_t r = 0; r < R; ++r)
    if (p->ring_off[r + 1] < p->ring_off[r] + 3) {
      set_error("ring %u has fewer than 3 vertices", r);
      return SDB_EINVAL;
    }
  const uint32_t V = p->ring_off[R];
  if (V >= 0x7fffffffu) {
    set_error("too many vertices (%u)", V);
    return SDB_EINVAL;
  }
  const uint32_t G = 1u << grid_bits;
  for (uint32_t v = 0; v < V; ++v)
    if (p->x[v] >= G || p->y[v] >= G) {
      set_error("vertex %u (%u, %u) outside the grid [0, 2^%u)", v, p->x[v], p->y[v], grid_bits);
      return SDB_EINVAL;
    }
  return SDB_OK;
}

sdb_status raster_common(const PolyEdges& pe, uint32_t grid_bits, uint32_t k,
                                const uint32_t* d_x, const uint32_t* d_y, const int32_t* d_attr,
                                uint64_t n, uint32_t tile_bits, uint64_t* d_count, int64_t* d_sum,
                                void* cuda_stream) {
  if (!d_count || (n > 0 && (!d_x || !d_y))) {
    set_error("d_count is NULL, or n > 0 with NULL coordinates");
    return SDB_EINVAL;
  }
  if (d_sum && !d_attr && n > 0) {
    set_error("d_sum requested without d_attr");
    return SDB_EINVAL;
  }
  if (n >= (1ull << 32)) {
    set_error("n = %llu points: at most 2^32 - 1 per call", (unsigned long long)n);
    return SDB_EINVAL;
  }
  if (tile_bits == 0) tile_bits = 13;
  if (tile_bits > 14) {
    set_error("tile_bits %u outside 1..14 (0 = default 13)", tile_bits);
    return SDB_EINVAL;
  }
  return raster_join(pe, grid_bits, k, d_x, d_y, d_attr, n, tile_bits, 8ull << 30, d_count, d_sum,
                     (cudaStream_t)cuda_stream);
}

}  // namespace sdb

using namespace sdb;

extern "C" {

sdb_status sdb_finest_level(uint32_t grid_bits, uint64_t eps, uint32_t* shift_out,
                            uint32_t* level_out) {
  uint32_t k = 0;
  SDB_TRY(finest(grid_bits, eps, &k));
  if (shift_out) *shift_out = k;
  if (level_out) *level_out = grid_bits - k;
  return SDB_OK;
}

sdb_status sdb_build_covering(const sdb_polygons* polys, uint32_t grid_bits, uint64_t eps,
                              void* cuda_stream, sdb_covering** out) {
  return sdb_build_covering_ex(polys, grid_bits, eps, 0u, cuda_stream, out);
}

sdb_status sdb_build_covering_ex(const sdb_polygons* polys, uint32_t grid_bits, uint64_t eps,
                                 uint32_t flags, void* cuda_stream, sdb_covering** out) {
  if (!out) {
    set_error("out is NULL");
    return SDB_EINVAL;
  }
  *out = nullptr;
  SDB_TRY(check_cover_flags(flags));
  uint32_t k = 0;
  SDB_TRY(finest(grid_bits, eps, &k));
  SDB_TRY(validate_polygons(polys, grid_bits));
  return new_covering(poly_edges(polys), grid_bits, k, flags, (cudaStream_t)cuda_stream, out);
}

sdb_status sdb_build_coverings(const sdb_polygons* polys, uint32_t grid_bits, const uint64_t* eps,
                               uint32_t n_eps, uint32_t flags, void* cuda_stream,
                               sdb_covering** out) {
  if (!out || !eps || n_eps == 0 || n_eps > 64) {
    set_error("out or eps is NULL, or n_eps outside 1..64");
    return SDB_EINVAL;
  }
  for (uint32_t i = 0; i < n_eps; ++i) out[i] = nullptr;
  SDB_TRY(check_cover_flags(flags));
  std::vector<uint32_t> ks(n_eps);
  for (uint32_t i = 0; i < n_eps; ++i) SDB_TRY(finest(grid_bits, eps[i], &ks[i]));
  SDB_TRY(validate_polygons(polys, grid_bits));
  std::vector<sdb_covering*> covs(n_eps, nullptr);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    set_error("no CUDA device");
    return SDB_ECUDA;
  }
  for (uint32_t i = 0; i < n_eps; ++i) {
    covs[i] = new (std::nothrow) sdb_covering();
    if (!covs[i]) {
      for (auto* c : covs) delete c;
      set_error("host allocation failed");
      return SDB_ENOMEM;
    }
    covs[i]->device = dev;
  }
  sdb_status st = build_coverings_multi(poly_edges(polys), grid_bits, ks.data(), n_eps, flags,
                                        (cudaStream_t)cuda_stream, covs.data());
  if (st != SDB_OK) {
    std::string msg = sdb_last_error();
    for (auto* c : covs) free_covering(c);
    set_error("%s", msg.c_str());
    return st;
  }
  for (uint32_t i = 0; i < n_eps; ++i) out[i] = covs[i];
  return SDB_OK;
}

sdb_status sdb_build_covering_multi(const sdb_multipolygons* polys, uint32_t grid_bits,
                                    uint64_t eps, uint32_t flags, void* cuda_stream,
                                    sdb_covering** out) {
  if (!out) {
    set_error("out is NULL");
    return SDB_EINVAL;
  }
  *out = nullptr;
  SDB_TRY(check_cover_flags(flags));
  uint32_t k = 0;
  SDB_TRY(finest(grid_bits, eps, &k));
  SDB_TRY(validate_multipolygons(polys, grid_bits));
  return new_covering(poly_edges(polys), grid_bits, k, flags, (cudaStream_t)cuda_stream, out);
}

}  // extern "C"

namespace sdb {
sdb_status validate_polygons(const sdb_polygons* polys, uint32_t grid_bits) {
  if (!polys || !polys->ring_off || !polys->x || !polys->y) {
    set_error("polygons or one of their arrays is NULL");
    return SDB_EINVAL;
  }
  const uint32_t P = polys->n_polygons;
  if (P == 0 || P >= (1u << 26)) {
    set_error("n_polygons %u outside 1..2^26-1", P);
    return SDB_EINVAL;
  }
  if (polys->ring_off[0] != 0) {
    set_error("ring_off[0] must be 0");
    return SDB_EINVAL;
  }
  for (uint32_t j = 0; j < P; ++j) {
    if (polys->ring_off[j + 1] < polys->ring_off[j] + 3) {
      set_error("polygon %u has fewer than 3 vertices", j);
      return SDB_EINVAL;
    }
  }
  const uint32_t V = polys->ring_off[P];
  if (V >= 0x7fffffffu) {
    set_error("too many vertices (%u)", V);
    return SDB_EINVAL;
  }
  const uint32_t G = 1u << grid_bits;
  for (uint32_t v = 0; v < V; ++v) {
    if (polys->x[v] >= G || polys->y[v] >= G) {
      set_error("vertex %u (%u, %u) outside the grid [0, 2^%u)", v, polys->x[v], polys->y[v],
                grid_bits);
      return SDB_EINVAL;
    }
  }
  return SDB_OK;
}
}  // namespace sdb

extern "C" {

sdb_status sdb_raster_join(const sdb_polygons* polys, uint32_t grid_bits, uint64_t eps,
                           const uint32_t* d_x, const uint32_t* d_y, const int32_t* d_attr,
                           uint64_t n, uint32_t tile_bits, uint64_t* d_count, int64_t* d_sum,
                           void* cuda_stream) {
  uint32_t k = 0;
  SDB_TRY(finest(grid_bits, eps, &k));
  SDB_TRY(validate_polygons(polys, grid_bits));
  return raster_common(poly_edges(polys), grid_bits, k, d_x, d_y, d_attr, n, tile_bits, d_count,
                       d_sum, cuda_stream);
}

sdb_status sdb_raster_join_multi(const sdb_multipolygons* polys, uint32_t grid_bits, uint64_t eps,
                                 const uint32_t* d_x, const uint32_t* d_y, const int32_t* d_attr,
                                 uint64_t n, uint32_t tile_bits, uint64_t* d_count,
                                 int64_t* d_sum, void* cuda_stream) {
  uint32_t k = 0;
  SDB_TRY(finest(grid_bits, eps, &k));
  SDB_TRY(validate_multipolygons(polys, grid_bits));
  return raster_common(poly_edges(polys), grid_bits, k, d_x, d_y, d_attr, n, tile_bits, d_count,
                       d_sum, cuda_stream);
}


sdb_status sdb_covering_get_info(const sdb_covering* cov, sdb_covering_info* info) {
  if (!cov || !info) {
    set_error("covering or info is NULL");
    return SDB_EINVAL;
  }
  memset(info, 0, sizeof(*info));
  info->grid_bits = cov->B;
  info->finest_shift = cov->k;
  info->finest_level = cov->F;
  info->n_polygons = cov->P;
  info->n_ranges = cov->R;
  info->n_list_ids = cov->nids;
  info->n_cells = cov->ncells;
  info->device_bytes =
      cov->bytes + (cov->leaf_bits ? (32ull << cov->leaf_bits) + (4ull << cov->knot_bits) + 4 +
                                         8ull * ((cov->R >> FENCE_SHIFT) + 1)
                                   : 0);
  if (cov->tab)
    info->device_bytes += (4ull << cov->tab_bits) + 8ull * cov->tab_mixed +
                          (cov->top ? (1ull << (2 * cov->top_level)) + 4 * TOP_PALETTE : 0) +
                          (4ull << (2 * cov->sub_bits)) * (cov->sub ? cov->tab_mixed : 0) +
                          8ull * cov->sub_mixed;
  info->index_leaf_bits = cov->leaf_bits;
  info->index_root_bits = cov->leaf_bits ? cov->knot_bits : 0u;
  info->boundary_flags = cov->flagged ? 1u : 0u;
  info->table_bits = cov->tab ? cov->tab_bits : 0u;
  info->table_mixed = cov->tab_mixed;
  info->table_sub_bits = cov->sub ? cov->sub_bits : 0u;
  info->table_sub_mixed = cov->sub_mixed;
  return SDB_OK;
}

sdb_status sdb_covering_build_index_ex(sdb_covering* cov, uint32_t leaf_bits, uint32_t root_bits,
                                       void* cuda_stream) {
  if (!cov) {
    set_error("covering is NULL");
    return SDB_EINVAL;
  }
  if (leaf_bits < 4 || leaf_bits > 20) {
    set_error("leaf_bits %u outside 4..20", leaf_bits);
    return SDB_EINVAL;
  }
  if (root_bits > SDB_INDEX_ROOT_BITS_MAX) {
    set_error("root_bits %u above %u", root_bits, SDB_INDEX_ROOT_BITS_MAX);
    return SDB_EINVAL;
  }
  SDB_TRY(check_device(cov));
  return build_learned_index(cov, leaf_bits, root_bits, (cudaStream_t)cuda_stream);
}

sdb_status sdb_covering_build_index(sdb_covering* cov, uint32_t leaf_bits, void* cuda_stream) {
  return sdb_covering_build_index_ex(cov, leaf_bits, SDB_INDEX_ROOT_BITS_DEFAULT, cuda_stream);
}

sdb_status sdb_covering_build_table(sdb_covering* cov, uint32_t table_bits, void* cuda_stream) {
  if (!cov) {
    set_error("covering is NULL");
    return SDB_EINVAL;
  }
  if (table_bits < 8 || table_bits > 26) {
    set_error("table_bits %u outside 8..26", table_bits);
    return SDB_EINVAL;
  }
  SDB_TRY(check_device(cov));
  return build_cell_table(cov, table_bits, (cudaStream_t)cuda_stream);
}

sdb_status sdb_join_aggregate(const uint32_t* d_x, const uint32_t* d_y, const int32_t* d_attr,
                              uint64_t n, const sdb_covering* cov, int lookup, uint64_t* d_count,
                              int64_t* d_sum, void* cuda_stream) {
  if (!cov || !d_count) {
    set_error("covering or d_count is NULL");
    return SDB_EINVAL;
  }
  if (n > 0 && (!d_x || !d_y)) {
    set_error("n > 0 with NULL coordinates");
    return SDB_EINVAL;
  }
  if (d_sum && !d_attr && n > 0) {
    set_error("d_sum requested without d_attr");
    return SDB_EINVAL;
  }
  SDB_TRY(check_lookup(cov, lookup));
  SDB_TRY(check_device(cov));
  return launch_join(d_x, d_y, d_attr, n, cov, lookup, d_count, d_sum, (cudaStream_t)cuda_stream,
                     true);
}

sdb_status sdb_join_aggregate_range(const uint32_t* d_x, const uint32_t* d_y, const int32_t* d_attr,
                                    uint64_t n, const sdb_covering* cov, int lookup,
                                    uint64_t* d_count, int64_t* d_sum, uint64_t* d_bcount,
                                    int64_t* d_bsum, uint64_t* d_babs, void* cuda_stream) {
  if (!cov || !d_count || !d_bcount) {
    set_error("covering, d_count or d_bcount is NULL");
    return SDB_EINVAL;
  }
  if (!cov->flagged) {
    set_error("covering was built without boundary flags (SDB_COVER_BOUNDARY_FLAGS)");
    return SDB_EINVAL;
  }
  if (n > 0 && (!d_x || !d_y)) {
    set_error("n > 0 with NULL coordinates");
    return SDB_EINVAL;
  }
  if ((d_sum != nullptr) != (d_bsum != nullptr) || (d_sum != nullptr) != (d_babs != nullptr)) {
    set_error("d_sum, d_bsum and d_babs must be given together");
    return SDB_EINVAL;
  }
  if (d_sum && !d_attr && n > 0) {
    set_error("d_sum requested without d_attr");
    return SDB_EINVAL;
  }
  SDB_TRY(check_lookup(cov, lookup));
  SDB_TRY(check_device(cov));
  return launch_join(d_x, d_y, d_attr, n, cov, lookup, d_count, d_sum, (cudaStream_t)cuda_stream,
                     true, d_bcount, d_bsum, d_babs);
}

sdb_status sdb_result_bounds(const uint64_t* d_count, const int64_t* d_sum,
                             const uint64_t* d_bcount, const int64_t* d_bsum,
                             const uint64_t* d_babs, uint32_t n_polygons, uint64_t* d_count_lo,
                             uint64_t* d_count_hi, int64_t* d_sum_lo, int64_t* d_sum_hi,
                             void* cuda_stream) {
  if (!d_count || !d_bcount || !d_count_lo || !d_count_hi) {
    set_error("d_count, d_bcount, d_count_lo or d_count_hi is NULL");
    return SDB_EINVAL;
  }
  const bool any = d_sum || d_bsum || d_babs || d_sum_lo || d_sum_hi;
  const bool all = d_sum && d_bsum && d_babs && d_sum_lo && d_sum_hi;
  if (any && !all) {
    set_error("d_sum, d_bsum, d_babs, d_sum_lo and d_sum_hi must be given together");
    return SDB_EINVAL;
  }
  return launch_result_bounds(d_count, d_sum, d_bcount, d_bsum, d_babs, n_polygons, d_count_lo,
                              d_count_hi, d_sum_lo, d_sum_hi, (cudaStream_t)cuda_stream);
}

sdb_status sdb_join_aggregate_multi(const uint32_t* d_x, const uint32_t* d_y, const int32_t* d_attr,
                                    uint64_t n, const sdb_covering* const* covs, uint32_t n_covs,
                                    int lookup, uint64_t* d_count, int64_t* d_sum,
                                    void* cuda_stream) {
  if (!covs || n_covs == 0 || !d_count) {
    set_error("covs or d_count is NULL, or n_covs = 0");
    return SDB_EINVAL;
  }
  if (n > 0 && (!d_x || !d_y)) {
    set_error("n > 0 with NULL coordinates");
    return SDB_EINVAL;
  }
  if (d_sum && !d_attr && n > 0) {
    set_error("d_sum requested without d_attr");
    return SDB_EINVAL;
  }
  for (uint32_t c = 0; c < n_covs; ++c) {
    if (!covs[c] || covs[c]->P != covs[0]->P || covs[c]->B != covs[0]->B) {
      set_error("covering %u is NULL or differs in polygon count or grid bits", c);
      return SDB_EINVAL;
    }
    SDB_TRY(check_lookup(covs[c], lookup));
    SDB_TRY(check_device(covs[c]));
  }
  return launch_join_multi(d_x, d_y, d_attr, n, covs, n_covs, lookup, d_count, d_sum,
                           (cudaStream_t)cuda_stream, true);
}

sdb_status sdb_join_aggregate_host(const uint32_t* h_x, const uint32_t* h_y, const int32_t* h_attr,
                                   uint64_t n, const sdb_covering* const* covs, uint32_t n_covs,
                                   int lookup, uint64_t* h_count, int64_t* h_sum,
                                   void* cuda_stream) {
  if (!covs || n_covs == 0 || !h_count) {
    set_error("coverings or h_count missing");
    return SDB_EINVAL;
  }
  if (n > 0 && (!h_x || !h_y)) {
    set_error("n > 0 with NULL coordinates");
    return SDB_EINVAL;
  }
  if (h_sum && !h_attr && n > 0) {
    set_error("h_sum requested without h_attr");
    return SDB_EINVAL;
  }
  const uint32_t P = covs[0] ? covs[0]->P : 0;
  for (uint32_t c = 0; c < n_covs; ++c) {
    if (!covs[c] || covs[c]->P != P) {
      set_error("covering %u is NULL or has a different polygon count", c);
      return SDB_EINVAL;
    }
    SDB_TRY(check_lookup(covs[c], lookup));
    SDB_TRY(check_device(covs[c]));
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  Scratch sc(s);
  const size_t outn = (size_t)n_covs * P;
  uint64_t* d_cnt;
  int64_t* d_sum = nullptr;
  SDB_TRY(sc.get(&d_cnt, outn));
  if (h_sum) SDB_TRY(sc.get(&d_sum, outn));
  SDB_TRY_CUDA(cudaMemsetAsync(d_cnt, 0, outn * 8, s));
  if (d_sum) SDB_TRY_CUDA(cudaMemsetAsync(d_sum, 0, outn * 8, s));
  if (lookup == SDB_LOOKUP_LEARNED || lookup == SDB_LOOKUP_TABLE_LEARNED)
    for (uint32_t c = 0; c < n_covs; ++c)
      SDB_TRY_CUDA(cudaMemsetAsync(covs[c]->fallbacks, 0, sizeof(unsigned long long), s));
  // points per chunk: the joins of the last chunk are not hidden by a copy,
  // but smaller chunks issue more launches per call, and a host whose API calls
  // are slow then falls behind the copies (2^22: 6.00 ms on some hosts, 7.81 on
  // another, for 100M points at four eps; 2^24: 6.05 ms)
  const uint64_t CH = 1ull << 24;
  const uint64_t nch = (n + CH - 1) / CH;
  uint32_t* dx[2];
  uint32_t* dy[2];
  int32_t* da[2] = {nullptr, nullptr};
  for (int b = 0; b < 2; ++b) {
    SDB_TRY(sc.get(&dx[b], CH));
    SDB_TRY(sc.get(&dy[b], CH));
    if (h_sum) SDB_TRY(sc.get(&da[b], CH));
  }
  cudaStream_t cs;
  SDB_TRY_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaEvent_t copied[2], done[2];
  for (int b = 0; b < 2; ++b) {
    cudaEventCreateWithFlags(&copied[b], cudaEventDisableTiming);
    cudaEventCreateWithFlags(&done[b], cudaEventDisableTiming);
  }
  sdb_status st = SDB_OK;
  for (uint64_t c = 0; c < nch && st == SDB_OK; ++c) {
    const int b = (int)(c & 1);
    const uint64_t a0 = c * CH, m = (n - a0 < CH) ? n - a0 : CH;
    cudaError_t e = cudaSuccess;
    if (c >= 2) e = cudaStreamWaitEvent(cs, done[b], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dx[b], h_x + a0, m * 4, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dy[b], h_y + a0, m * 4, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess && h_sum)
      e = cudaMemcpyAsync(da[b], h_attr + a0, m * 4, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaEventRecord(copied[b], cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, copied[b], 0);
    if (e != cudaSuccess) {
      st = cuda_status(e, "chunk copy", __FILE__, __LINE__);
      break;
    }
    for (uint32_t k = 0; k < n_covs && st == SDB_OK; ++k)
      st = launch_join(dx[b], dy[b], da[b], m, covs[k], lookup, d_cnt + (size_t)k * P,
                       d_sum ? d_sum + (size_t)k * P : nullptr, s, false);
    if (st == SDB_OK && cudaEventRecord(done[b], s) != cudaSuccess)
      st = cuda_status(cudaGetLastError(), "event record", __FILE__, __LINE__);
  }
  if (st == SDB_OK) {
    cudaError_t e = cudaMemcpyAsync(h_count, d_cnt, outn * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && h_sum)
      e = cudaMemcpyAsync(h_sum, d_sum, outn * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_status(e, "result copy", __FILE__, __LINE__);
  }
  cudaStreamSynchronize(cs);
  for (int b = 0; b < 2; ++b) {
    cudaEventDestroy(copied[b]);
    cudaEventDestroy(done[b]);
  }
  cudaStreamDestroy(cs);
  return st;
}

sdb_status sdb_covering_fallbacks(const sdb_covering* cov, void* cuda_stream, uint64_t* out) {
  if (!cov || !out) {
    set_error("covering or out is NULL");
    return SDB_EINVAL;
  }
  *out = 0;
  if (!cov->fallbacks) return SDB_OK;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  unsigned long long v = 0;
  SDB_TRY_CUDA(cudaMemcpyAsync(&v, cov->fallbacks, sizeof(v), cudaMemcpyDeviceToHost, s));
  SDB_TRY_CUDA(cudaStreamSynchronize(s));
  *out = v;
  return SDB_OK;
}

sdb_status sdb_covering_index_stats(const sdb_covering* cov, double* mean_window,
                                    uint32_t* max_window) {
  if (!cov || !mean_window || !max_window) {
    set_error("covering or an output is NULL");
    return SDB_EINVAL;
  }
  *mean_window = 0;
  *max_window = 0;
  if (!cov->leaves) return SDB_OK;
  SDB_TRY(check_device(cov));
  const size_t L = (size_t)1 << cov->leaf_bits;
  LeafRec* h = new (std::nothrow) LeafRec[L];
  if (!h) {
    set_error("host allocation failed");
    return SDB_ENOMEM;
  }
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(h, cov->leaves, L * sizeof(LeafRec), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    delete[] h;
    return cuda_status(e, "leaf copy", __FILE__, __LINE__);
  }
  double wsum = 0, rsum = 0;
  uint32_t wmax = 0;
  for (size_t l = 0; l < L; ++l) {
    const double w = (double)h[l].errlo + (double)h[l].errhi + 1.0;
    const double r = (double)h[l].last - (double)h[l].first + 1.0;
    wsum += w * r;
    rsum += r;
    if (w > wmax) wmax = (uint32_t)w;
  }
  delete[] h;
  *mean_window = rsum > 0 ? wsum / rsum : 0;
  *max_window = wmax;
  return SDB_OK;
}

sdb_status sdb_covering_export(const sdb_covering* cov, uint64_t* h_start, uint32_t* h_list_off,
                               uint32_t* h_list_ids) {
  if (!cov || !h_start || !h_list_off || (cov->nids && !h_list_ids)) {
    set_error("covering or an output array is NULL");
    return SDB_EINVAL;
  }
  SDB_TRY(check_device(cov));
  SDB_TRY_CUDA(cudaDeviceSynchronize());
  SDB_TRY_CUDA(cudaMemcpy(h_start, cov->start, (cov->R + 1) * 8, cudaMemcpyDeviceToHost));
  SDB_TRY_CUDA(cudaMemcpy(h_list_off, cov->list_off, (cov->R + 1) * 4, cudaMemcpyDeviceToHost));
  if (cov->nids)
    SDB_TRY_CUDA(cudaMemcpy(h_list_ids, cov->list_ids, cov->nids * 4, cudaMemcpyDeviceToHost));
  return SDB_OK;
}

void sdb_covering_free(sdb_covering* cov) { free_covering(cov); }

const char* sdb_status_string(sdb_status s) {
  switch (s) {
    case SDB_OK: return "ok";
    case SDB_EINVAL: return "invalid argument";
    case SDB_ENOMEM: return "out of memory";
    case SDB_ECUDA: return "CUDA error";
    case SDB_ETIMEOUT: return "timed out";
    case SDB_EBUSY: return "busy";
  }
  return "unknown status";
}

const char* sdb_last_error(void) { return g_err; }

uint64_t sdb_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

sdb_status sdb_memory_stats(uint64_t* pool_used, uint64_t* pool_reserved) {
  if (!pool_used || !pool_reserved) {
    set_error("pool_used or pool_reserved is NULL");
    return SDB_EINVAL;
  }
  cudaMemPool_t pool;
  SDB_TRY(get_pool(&pool));
  unsigned long long used = 0, reserved = 0;  // the attributes are 64-bit counters
  SDB_TRY_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used));
  SDB_TRY_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved));
  *pool_used = used;
  *pool_reserved = reserved;
  return SDB_OK;
}

sdb_status sdb_trace_enable(int on) {
  std::lock_guard<std::mutex> lk(g_tmu);
  if (on) {
    for (TraceRec& r : g_trace) {
      if (r.a) g_evpool.push_back(r.a);
      if (r.b) g_evpool.push_back(r.b);
    }
    g_trace.clear();
  }
  g_trace_on.store(on != 0);
  return SDB_OK;
}

sdb_status sdb_trace_read(sdb_trace_stat* out, uint32_t capacity, uint32_t* n_out) {
  if (!n_out || (capacity > 0 && !out)) {
    set_error("n_out is NULL, or out is NULL with capacity > 0");
    return SDB_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_tmu);
  std::vector<sdb_trace_stat> agg;
  for (const TraceRec& r : g_trace) {
    if (!r.name) continue;
    SDB_TRY_CUDA(cudaEventSynchronize(r.b));
    float ms = 0.f;
    SDB_TRY_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
    size_t i = 0;
    while (i < agg.size() && strncmp(agg[i].name, r.name, sizeof(agg[i].name) - 1) != 0) ++i;
    if (i == agg.size()) {
      agg.emplace_back();
      memset(&agg[i], 0, sizeof(agg[i]));
      strncpy(agg[i].name, r.name, sizeof(agg[i].name) - 1);
    }
    agg[i].count += 1;
    agg[i].total_ms += ms;
  }
  for (size_t i = 0; i < agg.size() && i < capacity; ++i) out[i] = agg[i];
  *n_out = (uint32_t)agg.size();
  return SDB_OK;
}

}  // extern "C"
