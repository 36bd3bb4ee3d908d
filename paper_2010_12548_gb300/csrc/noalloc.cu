// Host-buffer join that allocates no device memory.
//
// Some callers cannot allocate device memory while they call into this
// library: services that reserve their whole device-memory budget when they
// start and must not allocate afterwards (an allocation could fail or stall at
// an arbitrary moment under load), and plugins loaded into a process whose own
// allocator owns the device and forbids allocations made behind its back.
// For them this entry point streams host points through a fixed-size staging
// area and keeps the per-polygon accumulators in the same area: a file-scope
// device array that every GPU which loads the library holds until the process
// exits.
//
// Limits: at most SDB_NOALLOC_MAX_POLYGONS polygons per covering; any number of
// points (they are processed SDB_NOALLOC_CHUNK at a time).  The array is shared
// by every call: each call clears the accumulators before use, and calls whose
// GPU work overlaps (on different streams or threads) race on the array.  Each
// call looks up the array's device address in the current context, so calls
// made after a device reset (which reloads the module) find it afresh.
#include "sdb_internal.cuh"

namespace sdb {

namespace {

constexpr uint64_t CHUNK = SDB_NOALLOC_CHUNK;
constexpr uint64_t MAXP = SDB_NOALLOC_MAX_POLYGONS;
constexpr size_t SCRATCH_BYTES = CHUNK * 12 + MAXP * 16;

// staging: x[CHUNK] | y[CHUNK] | attr[CHUNK] | count[MAXP] | sum[MAXP]
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

// Device address of the array in the current context (host code only sees a
// host-side stand-in for the symbol).  Looked up on every call -- the lookup
// allocates nothing -- so a context recreated after a device reset never sees
// a stale address.
sdb_status scratch_address(unsigned char** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress", __FILE__, __LINE__);
  *out = static_cast<unsigned char*>(p);
  return SDB_OK;
}

}  // namespace

}  // namespace sdb

using namespace sdb;

extern "C" sdb_status sdb_join_aggregate_host_noalloc(const uint32_t* h_x, const uint32_t* h_y,
                                                      const int32_t* h_attr, uint64_t n,
                                                      const sdb_covering* cov, int lookup,
                                                      uint64_t* h_count, int64_t* h_sum,
                                                      void* cuda_stream) {
  if (!cov || !h_count) {
    set_error("covering or h_count is NULL");
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
  SDB_TRY(check_lookup(cov, lookup));
  if (cov->P > MAXP) {
    set_error("%u polygons exceed the allocation-free join's maximum of %llu", cov->P,
              (unsigned long long)MAXP);
    return SDB_EINVAL;
  }
  int dev = 0;
  SDB_TRY_CUDA(cudaGetDevice(&dev));
  if (dev != cov->device) {
    set_error("covering lives on device %d, current device is %d", cov->device, dev);
    return SDB_EINVAL;
  }
  unsigned char* base = nullptr;
  SDB_TRY(scratch_address(&base));
  uint32_t* dx = reinterpret_cast<uint32_t*>(base);
  uint32_t* dy = dx + CHUNK;
  int32_t* da = reinterpret_cast<int32_t*>(dy + CHUNK);
  uint64_t* dcnt = reinterpret_cast<uint64_t*>(base + CHUNK * 12);
  int64_t* dsum = reinterpret_cast<int64_t*>(dcnt + MAXP);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const size_t P = cov->P;
  // the array keeps the previous call's contents: clear the accumulators
  SDB_TRY_CUDA(cudaMemsetAsync(dcnt, 0, P * 8, s));
  SDB_TRY_CUDA(cudaMemsetAsync(dsum, 0, P * 8, s));
  if (lookup == SDB_LOOKUP_LEARNED || lookup == SDB_LOOKUP_TABLE_LEARNED)
    SDB_TRY_CUDA(cudaMemsetAsync(cov->fallbacks, 0, sizeof(unsigned long long), s));
  for (uint64_t a0 = 0; a0 < n; a0 += CHUNK) {
    const uint64_t m = (n - a0 < CHUNK) ? n - a0 : CHUNK;
    // one stream: the next chunk's copy waits for this chunk's join
    SDB_TRY_CUDA(cudaMemcpyAsync(dx, h_x + a0, m * 4, cudaMemcpyHostToDevice, s));
    SDB_TRY_CUDA(cudaMemcpyAsync(dy, h_y + a0, m * 4, cudaMemcpyHostToDevice, s));
    if (h_sum) SDB_TRY_CUDA(cudaMemcpyAsync(da, h_attr + a0, m * 4, cudaMemcpyHostToDevice, s));
    SDB_TRY(launch_join(dx, dy, h_sum ? da : nullptr, m, cov, lookup, dcnt, h_sum ? dsum : nullptr,
                        s, false));
  }
  SDB_TRY_CUDA(cudaMemcpyAsync(h_count, dcnt, P * 8, cudaMemcpyDeviceToHost, s));
  if (h_sum) SDB_TRY_CUDA(cudaMemcpyAsync(h_sum, dsum, P * 8, cudaMemcpyDeviceToHost, s));
  SDB_TRY_CUDA(cudaStreamSynchronize(s));
  return SDB_OK;
}
