// Device-wide primitives used by the covering builder: exclusive scan,
// stable LSD radix sort of uint64 keys (optionally carrying uint32 values),
// and unique of a sorted array.  Hand-written; no library sort.
#include "sdb_internal.cuh"

namespace sdb {

namespace {

constexpr unsigned FULL = 0xffffffffu;

// ------------------------------------------------------------------ scan
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <class T>
__device__ T block_exclusive_scan(T v, T* s_warp, T* total) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T t = __shfl_up_sync(FULL, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) s_warp[w] = inc;
  __syncthreads();
  if (w == 0) {
    T ws = lane < (SCAN_THREADS / 32) ? s_warp[lane] : T(0);
    T wi = ws;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T t = __shfl_up_sync(FULL, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < (SCAN_THREADS / 32)) s_warp[lane] = wi - ws;
    if (lane == (SCAN_THREADS / 32) - 1) s_warp[SCAN_THREADS / 32] = wi;
  }
  __syncthreads();
  T r = s_warp[w] + inc - v;
  *total = s_warp[SCAN_THREADS / 32];
  __syncthreads();
  return r;
}

template <class T>
__global__ __launch_bounds__(SCAN_THREADS) void scan_reduce_kernel(const T* in, size_t n, T* sums) {
  __shared__ T s_warp[SCAN_THREADS / 32 + 1];
  size_t base = (size_t)blockIdx.x * SCAN_TILE;
  T acc = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    size_t g = base + (size_t)i * SCAN_THREADS + threadIdx.x;
    if (g < n) acc += in[g];
  }
  T tot;
  block_exclusive_scan<T>(acc, s_warp, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

template <class T>
__global__ __launch_bounds__(SCAN_THREADS) void scan_tile_kernel(const T* in, T* out, size_t n,
                                                                 const T* block_off, T* d_total) {
  __shared__ T s_warp[SCAN_THREADS / 32 + 1];
  size_t base = (size_t)blockIdx.x * SCAN_TILE + (size_t)threadIdx.x * SCAN_ITEMS;
  T v[SCAN_ITEMS];
  T acc = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    size_t g = base + i;
    v[i] = g < n ? in[g] : T(0);
    acc += v[i];
  }
  T tot;
  T pre = block_exclusive_scan<T>(acc, s_warp, &tot);
  T off = (block_off ? block_off[blockIdx.x] : T(0)) + pre;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    size_t g = base + i;
    if (g < n) out[g] = off;
    off += v[i];
  }
  if (d_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == SCAN_THREADS - 1) {
    *d_total = off;  // last thread holds the grand total after its items
  }
}

// ------------------------------------------------------------------ radix sort
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 16;  // per lane
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
static_assert(RS_THREADS == 256, "one thread per digit in the scatter's digit scans");

// Per-block digit histogram of one 8-bit digit.  A full tile is read with
// 16-byte loads, all issued before any counting; counts go to per-warp
// shared-memory histograms with shared atomics.
__global__ __launch_bounds__(RS_THREADS) void radix_hist_kernel(const uint64_t* __restrict__ keys,
                                                               size_t n, int shift,
                                                               uint32_t* __restrict__ hist,
                                                               uint32_t nblocks) {
  __shared__ uint32_t h[RS_WARPS][256];
  const int w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS) (&h[0][0])[i] = 0;
  __syncthreads();
  const size_t tile0 = (size_t)blockIdx.x * RS_TILE;
  if (tile0 + RS_TILE <= n && (reinterpret_cast<uintptr_t>(keys) & 15u) == 0) {
    const ulonglong2* k2 = reinterpret_cast<const ulonglong2*>(keys + tile0);
    ulonglong2 r[RS_ITEMS / 2];
#pragma unroll
    for (int it = 0; it < RS_ITEMS / 2; ++it) r[it] = k2[it * RS_THREADS + threadIdx.x];
#pragma unroll
    for (int it = 0; it < RS_ITEMS / 2; ++it) {
      atomicAdd(&h[w][(uint32_t)(r[it].x >> shift) & 255u], 1u);
      atomicAdd(&h[w][(uint32_t)(r[it].y >> shift) & 255u], 1u);
    }
  } else {
    for (size_t g = tile0 + threadIdx.x; g < n; g += RS_THREADS)
      atomicAdd(&h[w][(uint32_t)(keys[g] >> shift) & 255u], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += RS_THREADS) {
    uint32_t t = 0;
    for (int ww = 0; ww < RS_WARPS; ++ww) t += h[ww][d];
    hist[(size_t)d * nblocks + blockIdx.x] = t;
  }
}

// Stable scatter of one 8-bit digit.  Each warp ranks its 512 keys (in order)
// by digit with a warp match; the block then lays its tile out in shared memory
// sorted by digit (stable), and writes it back so that consecutive threads
// write consecutive slots of the same digit's output run (coalesced), starting
// at the block's global offset for that digit.  Only the ranks stay in
// registers across the block's digit prefix: the keys are read again (from L2,
// four at a time) to lay the tile out, which keeps the keys-only form at five
// resident blocks per SM instead of three.
// SPLIT (keys only): the output is the packed covering record split into its
// key (kout) and standard value (vout), sb slot bits.
template <bool VALS>
constexpr int scatter_blocks() { return VALS ? 3 : 5; }

template <bool VALS, bool SPLIT = false>
__global__ __launch_bounds__(RS_THREADS, scatter_blocks<VALS>()) void radix_scatter_kernel(
    const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint64_t* __restrict__ kout,
    uint32_t* __restrict__ vout, size_t n, int shift, const uint32_t* __restrict__ offs,
    uint32_t nblocks, uint32_t sb = 0) {
  extern __shared__ __align__(16) unsigned char dyn[];
  uint64_t* sk = reinterpret_cast<uint64_t*>(dyn);                 // RS_TILE keys
  uint32_t* sv = reinterpret_cast<uint32_t*>(dyn + RS_TILE * 8);   // RS_TILE values
  uint32_t* vin_s = sv + RS_TILE;  // the tile's values as read, staged asynchronously
  __shared__ uint32_t cnt[RS_WARPS][256];  // per warp and digit: count, then warp prefix
  __shared__ uint32_t dstart[256];         // digit's first slot in the tile
  __shared__ uint32_t gbase[256];          // digit's first global slot for this block
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS) (&cnt[0][0])[i] = 0;
  __syncthreads();
  const size_t tile0 = (size_t)blockIdx.x * RS_TILE;
  const size_t base = tile0 + (size_t)w * (32 * RS_ITEMS);
  const unsigned lt = (1u << lane) - 1u;
  // a full tile's values travel to shared memory while the keys are ranked
  // (16-byte asynchronous copies; tiles start 16 KB apart in a 256-byte
  // aligned buffer); a partial last tile reads them directly later
  const bool full = tile0 + RS_TILE <= n && (reinterpret_cast<uintptr_t>(vin) & 15u) == 0;
  if (VALS && full) {
    for (int c = threadIdx.x; c < RS_TILE / 4; c += RS_THREADS) {
      const unsigned dst = (unsigned)__cvta_generic_to_shared(vin_s + 4 * c);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst),
                   "l"(vin + tile0 + 4 * c)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  // the keys are loaded for their digits only (each dies once ranked), half
  // of them in flight at a time; values are read only when the tile's layout
  // is known.  Ranks, later tile slots (< RS_TILE), go two to a register.
  uint32_t rank[RS_ITEMS / 2] = {};
  static_assert(RS_TILE <= 65536, "16-bit slots");
  constexpr int RS_HALF = RS_ITEMS / 2;
  uint64_t k[RS_HALF];
#pragma unroll
  for (int it = 0; it < RS_ITEMS; ++it) {
    if (it % RS_HALF == 0) {
#pragma unroll
      for (int j = 0; j < RS_HALF; ++j) {
        const size_t g = base + (size_t)(it + j) * 32 + lane;
        k[j] = g < n ? kin[g] : 0ull;
      }
    }
    const size_t g = base + (size_t)it * 32 + lane;
    const bool ok = g < n;
    const uint32_t d = ok ? (uint32_t)((k[it % RS_HALF] >> shift) & 255u) : 256u;
    // one lane per digit reads and advances the warp's counter (fewer
    // shared-memory bank conflicts than every lane reading it)
    const unsigned peers = __match_any_sync(FULL, d);
    const int lead = __ffs(peers) - 1;
    uint32_t before = (ok && lane == lead) ? cnt[w][d] : 0u;
    before = __shfl_sync(FULL, before, lead);
    if (ok && lane == lead) cnt[w][d] = before + __popc(peers);
    __syncwarp();
    rank[it >> 1] |= (before + __popc(peers & lt)) << (16 * (it & 1));
  }
  __syncthreads();
  // digit totals of the tile -> warp prefixes; thread d owns digit d
  uint32_t total = 0;
  {
    const int d = threadIdx.x;  // RS_THREADS == 256
    for (int ww = 0; ww < RS_WARPS; ++ww) {
      const uint32_t t = cnt[ww][d];
      cnt[ww][d] = total;
      total += t;
    }
    gbase[d] = offs[(size_t)d * nblocks + blockIdx.x];
  }
  // exclusive scan of the 256 digit totals (block-wide, two levels of warps)
  {
    __shared__ uint32_t wsum[RS_WARPS];
    uint32_t inc = total;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(FULL, inc, o);
      if (lane >= o) inc += t;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    uint32_t wpre = 0;
    for (int ww = 0; ww < w; ++ww) wpre += wsum[ww];
    dstart[threadIdx.x] = wpre + inc - total;
  }
  __syncthreads();
  // stable layout of the tile by digit in shared memory (rank becomes the
  // slot); the keys come back from L2 four at a time
#pragma unroll
  for (int it0 = 0; it0 < RS_ITEMS; it0 += 4) {
    uint64_t kk[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const size_t g = base + (size_t)(it0 + j) * 32 + lane;
      kk[j] = g < n ? __ldcg(kin + g) : 0ull;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const size_t g = base + (size_t)(it0 + j) * 32 + lane;
      if (g < n) {
        const uint32_t d = (uint32_t)((kk[j] >> shift) & 255u);
        const int it = it0 + j;
        const uint32_t slot = ((rank[it >> 1] >> (16 * (it & 1))) & 0xffffu) + dstart[d] + cnt[w][d];
        rank[it >> 1] += (slot - ((rank[it >> 1] >> (16 * (it & 1))) & 0xffffu)) << (16 * (it & 1));
        sk[slot] = kk[j];
      }
    }
  }
  if (VALS) {
    uint32_t v[RS_ITEMS];
    if (full) {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
      __syncthreads();  // every thread's copies have landed
#pragma unroll
      for (int it = 0; it < RS_ITEMS; ++it) v[it] = vin_s[w * (32 * RS_ITEMS) + it * 32 + lane];
    } else {
#pragma unroll
      for (int it = 0; it < RS_ITEMS; ++it) {
        const size_t g = base + (size_t)it * 32 + lane;
        v[it] = g < n ? vin[g] : 0u;
      }
    }
#pragma unroll
    for (int it = 0; it < RS_ITEMS; ++it)
      if (base + (size_t)it * 32 + lane < n) sv[(rank[it >> 1] >> (16 * (it & 1))) & 0xffffu] = v[it];
  }
  __syncthreads();
  const uint32_t tile_n = (uint32_t)min((size_t)RS_TILE, n - tile0);
  for (uint32_t i = threadIdx.x; i < tile_n; i += RS_THREADS) {
    const uint64_t key = sk[i];
    const uint32_t d = (uint32_t)((key >> shift) & 255u);
    const uint32_t pos = gbase[d] + (i - dstart[d]);
    if (SPLIT) {
      kout[pos] = key >> (sb + 6);
      vout[pos] = record_val(key, sb);
    } else {
      kout[pos] = key;
      if (VALS) vout[pos] = sv[i];
    }
  }
}

template <bool VALS>
sdb_status radix_sort_impl(uint64_t* keys, uint32_t* vals, uint64_t* ktmp, uint32_t* vtmp, size_t n,
                           int bits, cudaStream_t s, uint64_t** kres, uint32_t** vres,
                           int first_bit = 0, uint32_t* split_vals = nullptr, uint32_t sb = 0) {
  *kres = keys;
  if (VALS) *vres = vals;
  if (n <= 1 || bits <= 0) return SDB_OK;
  if (n >= 0xffffffffull) {
    set_error("radix sort: %zu elements exceeds the 32-bit rank range", n);
    return SDB_EINVAL;
  }
  uint32_t nblocks = (uint32_t)((n + RS_TILE - 1) / RS_TILE);
  // keys (8 B each), and with values the values' slots and their staging
  constexpr size_t SCATTER_SMEM = (size_t)RS_TILE * (VALS ? 16 : 8);
  SDB_TRY_CUDA(cudaFuncSetAttribute(radix_scatter_kernel<VALS>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)SCATTER_SMEM));
  if (!VALS && split_vals)
    SDB_TRY_CUDA(cudaFuncSetAttribute(radix_scatter_kernel<false, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)SCATTER_SMEM));
  Scratch sc(s);
  uint32_t *hist, *offs;
  SDB_TRY(sc.get(&hist, (size_t)256 * nblocks));
  SDB_TRY(sc.get(&offs, (size_t)256 * nblocks));
  uint64_t *ka = keys, *kb = ktmp;
  uint32_t *va = vals, *vb = vtmp;
  for (int shift = first_bit; shift < first_bit + bits; shift += 8) {
    {
      TraceScope tr("sort.hist", s);
      radix_hist_kernel<<<nblocks, RS_THREADS, 0, s>>>(ka, n, shift, hist, nblocks);
      note_launch();
      SDB_TRY_CUDA(cudaGetLastError());
    }
    {
      TraceScope tr("sort.scan", s);
      SDB_TRY(exclusive_scan<uint32_t>(hist, offs, (size_t)256 * nblocks, nullptr, s));
    }
    {
      TraceScope tr("sort.scatter", s);
      if (!VALS && split_vals && shift + 8 >= first_bit + bits)  // the last pass splits
        radix_scatter_kernel<false, true><<<nblocks, RS_THREADS, SCATTER_SMEM, s>>>(
            ka, nullptr, kb, split_vals, n, shift, offs, nblocks, sb);
      else
        radix_scatter_kernel<VALS><<<nblocks, RS_THREADS, SCATTER_SMEM, s>>>(ka, va, kb, vb, n,
                                                                              shift, offs, nblocks);
      note_launch();
      SDB_TRY_CUDA(cudaGetLastError());
    }
    uint64_t* t = ka;
    ka = kb;
    kb = t;
    uint32_t* u = va;
    va = vb;
    vb = u;
  }
  *kres = ka;
  if (VALS) *vres = va;
  return SDB_OK;
}

__global__ void flag_new_kernel(const uint64_t* in, size_t n, uint32_t* flags) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flags[i] = (i == 0 || in[i] != in[i - 1]) ? 1u : 0u;
}

__global__ void compact_flagged_kernel(const uint64_t* in, size_t n, const uint32_t* flags,
                                       const uint32_t* pos, uint64_t* out) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && flags[i]) out[pos[i]] = in[i];
}

}  // namespace

template <class T>
sdb_status exclusive_scan(const T* in, T* out, size_t n, T* d_total, cudaStream_t s) {
  if (n == 0) {
    if (d_total) SDB_TRY_CUDA(cudaMemsetAsync(d_total, 0, sizeof(T), s));
    return SDB_OK;
  }
  size_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (nb == 1) {
    scan_tile_kernel<T><<<1, SCAN_THREADS, 0, s>>>(in, out, n, nullptr, d_total);
    note_launch();
    SDB_TRY_CUDA(cudaGetLastError());
    return SDB_OK;
  }
  Scratch sc(s);
  T *sums, *soff;
  SDB_TRY(sc.get(&sums, nb));
  SDB_TRY(sc.get(&soff, nb));
  scan_reduce_kernel<T><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, sums);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  SDB_TRY(exclusive_scan<T>(sums, soff, nb, nullptr, s));
  scan_tile_kernel<T><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, out, n, soff, d_total);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  return SDB_OK;
}

template sdb_status exclusive_scan<uint32_t>(const uint32_t*, uint32_t*, size_t, uint32_t*, cudaStream_t);
template sdb_status exclusive_scan<uint64_t>(const uint64_t*, uint64_t*, size_t, uint64_t*, cudaStream_t);

sdb_status radix_sort_keys(uint64_t* keys, uint64_t* tmp, size_t n, int bits, cudaStream_t s,
                           uint64_t** result, int first_bit) {
  uint32_t* dummy = nullptr;
  return radix_sort_impl<false>(keys, nullptr, tmp, nullptr, n, bits, s, result, &dummy,
                                first_bit);
}

sdb_status radix_sort_split(uint64_t* keys, uint64_t* tmp, size_t n, int bits, int first_bit,
                            uint32_t sb, uint32_t* vals_out, cudaStream_t s, uint64_t** keys_out) {
  uint32_t* dummy = nullptr;
  if (n <= 1) {  // no pass runs: split in place
    if (n == 1) {
      uint64_t w = 0;
      SDB_TRY_CUDA(cudaMemcpyAsync(&w, keys, 8, cudaMemcpyDeviceToHost, s));
      SDB_TRY_CUDA(cudaStreamSynchronize(s));
      const uint64_t k = w >> (sb + 6);
      const uint32_t v = record_val(w, sb);
      SDB_TRY_CUDA(cudaMemcpyAsync(keys, &k, 8, cudaMemcpyHostToDevice, s));
      SDB_TRY_CUDA(cudaMemcpyAsync(vals_out, &v, 4, cudaMemcpyHostToDevice, s));
      SDB_TRY_CUDA(cudaStreamSynchronize(s));
    }
    *keys_out = keys;
    return SDB_OK;
  }
  return radix_sort_impl<false>(keys, nullptr, tmp, nullptr, n, bits, s, keys_out, &dummy,
                                first_bit, vals_out, sb);
}

sdb_status radix_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* ktmp, uint32_t* vtmp, size_t n,
                            int bits, cudaStream_t s, uint64_t** kres, uint32_t** vres) {
  return radix_sort_impl<true>(keys, vals, ktmp, vtmp, n, bits, s, kres, vres);
}

sdb_status unique_sorted(const uint64_t* in, size_t n, uint64_t* out, size_t* m, cudaStream_t s) {
  if (n == 0) {
    *m = 0;
    return SDB_OK;
  }
  if (n >= 0xffffffffull) {
    set_error("unique: %zu elements exceeds the 32-bit index range", n);
    return SDB_EINVAL;
  }
  Scratch sc(s);
  uint32_t *flags, *pos, *tot;
  SDB_TRY(sc.get(&flags, n));
  SDB_TRY(sc.get(&pos, n));
  SDB_TRY(sc.get(&tot, 1));
  flag_new_kernel<<<grid_for(n, 256), 256, 0, s>>>(in, n, flags);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  SDB_TRY(exclusive_scan<uint32_t>(flags, pos, n, tot, s));
  compact_flagged_kernel<<<grid_for(n, 256), 256, 0, s>>>(in, n, flags, pos, out);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  uint32_t h = 0;
  SDB_TRY_CUDA(cudaMemcpyAsync(&h, tot, sizeof(h), cudaMemcpyDeviceToHost, s));
  SDB_TRY_CUDA(cudaStreamSynchronize(s));
  *m = h;
  return SDB_OK;
}

}  // namespace sdb
