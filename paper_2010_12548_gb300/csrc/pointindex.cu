// Point-indexed aggregation (Sec. 3, "Point Indexing").  The resident points
// are already ordered by their full-resolution Hilbert id (level B); a covering
// range [h, h') at the finest level F holds exactly the points whose ids lie in
// [h << 2k, h' << 2k) (the curve's prefix property), a contiguous slice of the
// sorted array.  COUNT is the slice's length and SUM a difference of prefix
// sums, so one lower-bound lookup per range boundary answers the whole
// covering.  The lookups use binary search or a RadixSpline (the paper's learned
// index: spline points with a bounded interpolation error and a radix table over
// the keys' top bits).
//
//  * prefix[i] = attr[0] + ... + attr[i-1] in key order, int64 (n + 1 entries).
//  * spline: over the distinct keys (each at its first position), the greedy
//    spline corridor: from the last spline point, keep the narrowest cone of
//    slopes that passes within +-E of every point seen; when a point leaves the
//    cone the previous point becomes a spline point.  Slopes are compared exactly
//    (128-bit cross products).  The array is cut into chunks of CHUNK keys, each
//    scanned by one thread, every chunk starting and ending with a spline point
//    (one pass, in parallel; the bound holds on every segment).
//  * radix table: entry j = first spline point whose key, minus the smallest
//    key, shifted right so that 2^radix_bits prefixes cover the key range, is
//    >= j.  A lookup reads two entries, searches the few spline points between
//    them, interpolates exactly in integers, and searches +-(E + 1) around the
//    estimate; the bracket is verified and plain binary search is the fallback
//    (counted).
#include "sdb_internal.cuh"

namespace sdb {

namespace {

constexpr uint64_t CHUNK = 4096;  // keys per spline-building thread
constexpr uint32_t NONE = 0xffffffffu;

struct SplinePt {
  uint64_t k;
  int64_t p;
};

// slope(a -> b1) < slope(a -> b2), both keys above a's
__device__ __forceinline__ bool slope_less(const SplinePt& a, const SplinePt& b1,
                                           const SplinePt& b2) {
  const __int128 l = (__int128)(b1.p - a.p) * (__int128)(b2.k - a.k);
  const __int128 r = (__int128)(b2.p - a.p) * (__int128)(b1.k - a.k);
  return l < r;
}

// The greedy corridor over chunk c's distinct keys; emit(point) in key order.
template <class Emit>
__device__ void corridor(const uint64_t* __restrict__ key, uint64_t n, uint64_t c, int64_t E,
                         Emit emit) {
  uint64_t i = c * CHUNK;
  const uint64_t end = min(n, i + CHUNK);
  while (i < end && i > 0 && key[i] == key[i - 1]) ++i;  // a run begun in the previous chunk
  if (i >= end) return;
  SplinePt base{key[i], (int64_t)i}, prev = base, up{0, 0}, lo{0, 0};
  emit(base);
  bool cone = false;
  for (uint64_t j = i + 1; j < end; ++j) {
    const uint64_t k = key[j];
    if (k == prev.k) continue;  // distinct keys at their first position
    const SplinePt cp{k, (int64_t)j};
    const SplinePt u2{k, (int64_t)j + E}, l2{k, (int64_t)j - E};
    if (!cone) {
      up = u2;
      lo = l2;
      cone = true;
    } else if (slope_less(base, up, cp) || slope_less(base, cp, lo)) {
      emit(prev);  // cp leaves the cone: prev ends the segment
      base = prev;
      up = u2;
      lo = l2;
    } else {
      if (slope_less(base, u2, up)) up = u2;
      if (slope_less(base, lo, l2)) lo = l2;
    }
    prev = cp;
  }
  if (prev.k != base.k) emit(prev);  // the chunk's last distinct key closes it
}

__global__ void spline_count_kernel(const uint64_t* __restrict__ key, uint64_t n, uint64_t nchunks,
                                    int64_t E, uint64_t* __restrict__ cnt) {
  const uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nchunks) return;
  uint64_t m = 0;
  corridor(key, n, c, E, [&](const SplinePt&) { ++m; });
  cnt[c] = m;
}

__global__ void spline_write_kernel(const uint64_t* __restrict__ key, uint64_t n,
                                    uint64_t nchunks, int64_t E,
                                    const uint64_t* __restrict__ off, uint64_t* __restrict__ sk,
                                    uint32_t* __restrict__ sp) {
  const uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nchunks) return;
  uint64_t o = off[c];
  corridor(key, n, c, E, [&](const SplinePt& q) {
    sk[o] = q.k;
    sp[o] = (uint32_t)q.p;
    ++o;
  });
}

// table[j] = first spline point with prefix >= j, j in [0, 2^r]: the prefix of
// key x is (x - kmin) >> shift, which is >= j exactly when x >= kmin + (j << shift)
__global__ void radix_table_kernel(const uint64_t* __restrict__ sk, uint64_t ns, uint64_t kmin,
                                   uint32_t shift, uint32_t r, uint32_t* __restrict__ table) {
  const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j > (1ull << r)) return;
  const uint64_t q = kmin + (j << shift);
  uint64_t lo = 0, len = ns;
  while (len > 0) {
    const uint64_t half = len >> 1;
    if (sk[lo + half] < q) {
      lo += half + 1;
      len -= half + 1;
    } else {
      len = half;
    }
  }
  table[j] = (uint32_t)lo;
}

__global__ void widen_attr_kernel(const int32_t* __restrict__ a, uint64_t n,
                                  uint64_t* __restrict__ w) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) w[i] = (uint64_t)(int64_t)a[i];
}

struct Spline {
  const uint64_t* key;  // the points' sorted keys
  uint64_t n;
  const uint64_t* sk;
  const uint32_t* sp;
  uint64_t ns;
  const uint32_t* table;
  uint64_t kmin, kmax;
  uint32_t shift;
  int64_t E;
  unsigned long long* fallbacks;
};

// first index in [lo, hi) with key >= q, hi if none
__device__ __forceinline__ uint64_t lower_bound_in(const uint64_t* __restrict__ key, uint64_t lo,
                                                   uint64_t hi, uint64_t q) {
  uint64_t len = hi - lo;
  while (len > 0) {
    const uint64_t half = len >> 1;
    if (__ldg(key + lo + half) < q) {
      lo += half + 1;
      len -= half + 1;
    } else {
      len = half;
    }
  }
  return lo;
}

__device__ uint64_t spline_lower_bound(const Spline& S, uint64_t q) {
  if (q <= S.kmin) return 0;
  if (q > S.kmax) return S.n;
  const uint64_t j = (q - S.kmin) >> S.shift;
  // the last spline point with key <= q lies in [table[j] - 1, table[j + 1])
  uint64_t a = __ldg(S.table + j), b = __ldg(S.table + j + 1);
  a = a > 0 ? a - 1 : 0;
  uint64_t len = b - a;  // last index in [a, b) with sk <= q (sk[a] <= q holds)
  while (len > 1) {
    const uint64_t half = len >> 1;
    if (__ldg(S.sk + a + half) <= q) a += half;
    len -= half;
  }
  uint64_t est;
  if (a + 1 >= S.ns) {
    est = __ldg(S.sp + a);
  } else {
    const uint64_t k0 = __ldg(S.sk + a), k1 = __ldg(S.sk + a + 1);
    const uint64_t p0 = __ldg(S.sp + a), p1 = __ldg(S.sp + a + 1);
    est = p0 + (uint64_t)((unsigned __int128)(q - k0) * (p1 - p0) / (k1 - k0));
  }
  const uint64_t lo = est > (uint64_t)S.E + 1 ? est - (uint64_t)S.E - 1 : 0;
  const uint64_t hi = min(S.n, est + (uint64_t)S.E + 2);
  const uint64_t pos = lower_bound_in(S.key, lo, hi, q);
  const bool ok = (pos == 0 || __ldg(S.key + pos - 1) < q) && (pos == S.n || __ldg(S.key + pos) >= q);
  if (ok) return pos;
  atomicAdd(S.fallbacks, 1ull);
  return lower_bound_in(S.key, 0, S.n, q);
}

// pos[r] = lower bound of start[r] << sh, r in [0, R]
template <bool RS>
__global__ void boundary_pos_kernel(const uint64_t* __restrict__ start, uint64_t R, uint32_t sh,
                                    Spline S, uint32_t* __restrict__ pos) {
  const uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r > R) return;
  const uint64_t q = __ldg(start + r) << sh;
  pos[r] = (uint32_t)(RS ? spline_lower_bound(S, q) : lower_bound_in(S.key, 0, S.n, q));
}

template <bool SUM>
__global__ void range_aggregate_kernel(const uint32_t* __restrict__ pos, uint64_t R,
                                       const uint32_t* __restrict__ pay,
                                       const uint32_t* __restrict__ list_off,
                                       const uint32_t* __restrict__ list_ids,
                                       const int64_t* __restrict__ prefix,
                                       unsigned long long* __restrict__ count,
                                       unsigned long long* __restrict__ sum) {
  const uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  const uint32_t py = __ldg(pay + r);
  if (py == NONE) return;
  const uint32_t a = __ldg(pos + r), b = __ldg(pos + r + 1);
  if (a == b) return;
  const unsigned long long c = b - a;
  const unsigned long long s = SUM ? (unsigned long long)(__ldg(prefix + b) - __ldg(prefix + a)) : 0;
  if (py < 0x80000000u) {
    const uint32_t p = py & 0x3fffffffu;
    atomicAdd(count + p, c);
    if (SUM) atomicAdd(sum + p, s);
  } else {
    const uint32_t rr = py & 0x7fffffffu;
    for (uint32_t e = __ldg(list_off + rr); e < __ldg(list_off + rr + 1); ++e) {
      const uint32_t p = __ldg(list_ids + e) & 0x7fffffffu;
      atomicAdd(count + p, c);
      if (SUM) atomicAdd(sum + p, s);
    }
  }
}

// largest |interpolated - true position| over the distinct keys
__global__ void spline_error_kernel(Spline S, unsigned long long* __restrict__ worst) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S.n || (i > 0 && S.key[i] == S.key[i - 1])) return;
  const uint64_t q = S.key[i];
  uint64_t a = 0, len = S.ns;  // last spline point with key <= q
  while (len > 1) {
    const uint64_t half = len >> 1;
    if (S.sk[a + half] <= q) a += half;
    len -= half;
  }
  uint64_t est = S.sp[a];
  if (a + 1 < S.ns) {
    const uint64_t k0 = S.sk[a], k1 = S.sk[a + 1], p0 = S.sp[a], p1 = S.sp[a + 1];
    est = p0 + (uint64_t)((unsigned __int128)(q - k0) * (p1 - p0) / (k1 - k0));
  }
  const unsigned long long d = est > i ? est - i : i - est;
  atomicMax(worst, d);
}

Spline spline_of(const sdb_points* p) {
  Spline S{};
  S.key = p->key;
  S.n = p->n;
  S.sk = p->rs_key;
  S.sp = p->rs_pos;
  S.ns = p->rs_n;
  S.table = p->rs_table;
  S.kmin = p->rs_min;
  S.kmax = p->rs_max;
  S.shift = p->rs_shift;
  S.E = (int64_t)p->rs_error;
  S.fallbacks = p->rs_fallbacks;
  return S;
}

}  // namespace

void release_point_index(sdb_points* p, cudaStream_t s) {
  void* ps[] = {p->prefix, p->rs_key, p->rs_pos, p->rs_table, p->rs_fallbacks};
  for (void* q : ps)
    if (q) dfree(q, s);
  p->prefix = nullptr;
  p->rs_key = nullptr;
  p->rs_pos = nullptr;
  p->rs_table = nullptr;
  p->rs_fallbacks = nullptr;
  p->rs_n = 0;
  p->rs_radix_bits = 0;
}

sdb_status build_point_index(sdb_points* p, uint32_t radix_bits, uint32_t spline_error,
                             cudaStream_t s) {
  release_point_index(p, s);
  Scratch sc(s);
  const uint64_t n = p->n;
  // prefix sums of the attribute in key order
  SDB_TRY(dalloc_n(&p->prefix, n + 1, s));
  uint64_t* w;
  SDB_TRY(sc.get(&w, n));
  widen_attr_kernel<<<grid_for(n, 256), 256, 0, s>>>(p->attr, n, w);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  uint64_t* pre = reinterpret_cast<uint64_t*>(p->prefix);
  SDB_TRY(exclusive_scan<uint64_t>(w, pre, n, pre + n, s));
  sc.release(w);
  // spline points, chunk by chunk
  const uint64_t nchunks = (n + CHUNK - 1) / CHUNK;
  uint64_t *cnt, *off, *dns;
  SDB_TRY(sc.get(&cnt, nchunks));
  SDB_TRY(sc.get(&off, nchunks));
  SDB_TRY(sc.get(&dns, 1));
  spline_count_kernel<<<grid_for(nchunks, 128), 128, 0, s>>>(p->key, n, nchunks,
                                                              (int64_t)spline_error, cnt);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  SDB_TRY(exclusive_scan<uint64_t>(cnt, off, nchunks, dns, s));
  uint64_t ns = 0, ends[2] = {0, 0};
  SDB_TRY_CUDA(cudaMemcpyAsync(&ns, dns, 8, cudaMemcpyDeviceToHost, s));
  SDB_TRY_CUDA(cudaMemcpyAsync(&ends[0], p->key, 8, cudaMemcpyDeviceToHost, s));
  SDB_TRY_CUDA(cudaMemcpyAsync(&ends[1], p->key + n - 1, 8, cudaMemcpyDeviceToHost, s));
  SDB_TRY_CUDA(cudaStreamSynchronize(s));
  if (ns >= 0xffffffffull) {
    set_error("radix spline: %llu spline points exceed 32-bit indices", (unsigned long long)ns);
    return SDB_ENOMEM;
  }
  SDB_TRY(dalloc_n(&p->rs_key, ns, s));
  SDB_TRY(dalloc_n(&p->rs_pos, ns, s));
  spline_write_kernel<<<grid_for(nchunks, 128), 128, 0, s>>>(p->key, n, nchunks,
                                                              (int64_t)spline_error, off, p->rs_key,
                                                              p->rs_pos);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  // radix table over the key range
  const uint64_t span = ends[1] - ends[0];
  const uint32_t span_bits = span ? 64 - __builtin_clzll(span) : 0;
  p->rs_shift = span_bits > radix_bits ? span_bits - radix_bits : 0;
  SDB_TRY(dalloc_n(&p->rs_table, (1ull << radix_bits) + 1, s));
  radix_table_kernel<<<grid_for((1ull << radix_bits) + 1, 256), 256, 0, s>>>(
      p->rs_key, ns, ends[0], p->rs_shift, radix_bits, p->rs_table);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  SDB_TRY(dalloc_n(&p->rs_fallbacks, 1, s));
  SDB_TRY_CUDA(cudaMemsetAsync(p->rs_fallbacks, 0, 8, s));
  SDB_TRY_CUDA(cudaStreamSynchronize(s));
  p->rs_n = ns;
  p->rs_min = ends[0];
  p->rs_max = ends[1];
  p->rs_radix_bits = radix_bits;
  p->rs_error = spline_error;
  return SDB_OK;
}

sdb_status point_index_aggregate(const sdb_points* p, const sdb_covering* cov, int lookup,
                                 uint64_t* count, int64_t* sum, cudaStream_t s) {
  SDB_TRY_CUDA(cudaMemsetAsync(count, 0, (size_t)cov->P * 8, s));
  if (sum) SDB_TRY_CUDA(cudaMemsetAsync(sum, 0, (size_t)cov->P * 8, s));
  const bool rs = lookup == SDB_LOOKUP_RADIX_SPLINE;
  if (rs) SDB_TRY_CUDA(cudaMemsetAsync(p->rs_fallbacks, 0, 8, s));
  Scratch sc(s);
  const uint64_t R = cov->R;
  uint32_t* pos;
  SDB_TRY(sc.get(&pos, R + 1));
  const Spline S = spline_of(p);
  const uint32_t sh = 2 * cov->k;
  if (rs)
    boundary_pos_kernel<true><<<grid_for(R + 1, 256), 256, 0, s>>>(cov->start, R, sh, S, pos);
  else
    boundary_pos_kernel<false><<<grid_for(R + 1, 256), 256, 0, s>>>(cov->start, R, sh, S, pos);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  auto* c = reinterpret_cast<unsigned long long*>(count);
  auto* su = reinterpret_cast<unsigned long long*>(sum);
  if (sum)
    range_aggregate_kernel<true><<<grid_for(R, 256), 256, 0, s>>>(
        pos, R, cov->pay, cov->list_off, cov->list_ids, p->prefix, c, su);
  else
    range_aggregate_kernel<false><<<grid_for(R, 256), 256, 0, s>>>(
        pos, R, cov->pay, cov->list_off, cov->list_ids, p->prefix, c, su);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  return SDB_OK;
}

sdb_status point_index_stats(const sdb_points* p, uint64_t* n_spline, uint64_t* max_error,
                             uint64_t* fallbacks, cudaStream_t s) {
  *n_spline = p->rs_n;
  unsigned long long h[2] = {0, 0};
  Scratch sc(s);
  unsigned long long* worst;
  SDB_TRY(sc.get(&worst, 1));
  SDB_TRY_CUDA(cudaMemsetAsync(worst, 0, 8, s));
  spline_error_kernel<<<grid_for(p->n, 256), 256, 0, s>>>(spline_of(p), worst);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  SDB_TRY_CUDA(cudaMemcpyAsync(&h[0], worst, 8, cudaMemcpyDeviceToHost, s));
  SDB_TRY_CUDA(cudaMemcpyAsync(&h[1], p->rs_fallbacks, 8, cudaMemcpyDeviceToHost, s));
  SDB_TRY_CUDA(cudaStreamSynchronize(s));
  *max_error = h[0];
  *fallbacks = h[1];
  return SDB_OK;
}

}  // namespace sdb

extern "C" {

sdb_status sdb_points_build_index(sdb_points* pts, uint32_t radix_bits, uint32_t spline_error,
                                  void* cuda_stream) {
  if (!pts) {
    sdb::set_error("points is NULL");
    return SDB_EINVAL;
  }
  if (radix_bits < 1 || radix_bits > 30) {
    sdb::set_error("radix_bits %u outside 1..30", radix_bits);
    return SDB_EINVAL;
  }
  if (spline_error < 1 || spline_error > (1u << 20)) {
    sdb::set_error("spline_error %u outside 1..2^20", spline_error);
    return SDB_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != pts->device) {
    sdb::set_error("points live on device %d, current device is %d", pts->device, dev);
    return SDB_EINVAL;
  }
  return sdb::build_point_index(pts, radix_bits, spline_error, (cudaStream_t)cuda_stream);
}

sdb_status sdb_points_aggregate(const sdb_points* pts, const sdb_covering* cov, int lookup,
                                uint64_t* d_count, int64_t* d_sum, void* cuda_stream) {
  if (!pts || !cov || !d_count) {
    sdb::set_error("points, covering or d_count is NULL");
    return SDB_EINVAL;
  }
  if (lookup != SDB_LOOKUP_BINARY && lookup != SDB_LOOKUP_RADIX_SPLINE) {
    sdb::set_error("point aggregation takes SDB_LOOKUP_BINARY or SDB_LOOKUP_RADIX_SPLINE, not %d",
                   lookup);
    return SDB_EINVAL;
  }
  if (cov->B != pts->B) {
    sdb::set_error("covering grid bits %u differ from the points' %u", cov->B, pts->B);
    return SDB_EINVAL;
  }
  if ((d_sum || lookup == SDB_LOOKUP_RADIX_SPLINE) && !pts->prefix) {
    sdb::set_error("SUM and the RadixSpline lookup need sdb_points_build_index first");
    return SDB_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != pts->device || dev != cov->device) {
    sdb::set_error("points, covering and current device differ");
    return SDB_EINVAL;
  }
  return sdb::point_index_aggregate(pts, cov, lookup, d_count, d_sum, (cudaStream_t)cuda_stream);
}

sdb_status sdb_points_index_stats(const sdb_points* pts, uint64_t* n_spline, uint64_t* max_error,
                                  uint64_t* fallbacks, void* cuda_stream) {
  if (!pts || !n_spline || !max_error || !fallbacks) {
    sdb::set_error("NULL argument");
    return SDB_EINVAL;
  }
  if (!pts->prefix) {
    sdb::set_error("no point index (sdb_points_build_index)");
    return SDB_EINVAL;
  }
  return sdb::point_index_stats(pts, n_spline, max_error, fallbacks, (cudaStream_t)cuda_stream);
}

}  // extern "C"
