// Join fused with aggregation (Sec. 5.1): per point, its finest-level cell id
// (Sec. 3, "a query point is mapped to a cell on the most fine-grained grid
// level"), the covering range holding that id, and COUNT/SUM for every polygon
// on the range's list.  No exact geometric test.
//
// Layout and mapping:
//  * points are SoA uint32 x[], y[], int32 attr[]; each lane takes 4 consecutive
//    points per step (one 16-byte load per array, streaming cache hint), a warp
//    covers 128 consecutive points, all warps stride over the array;
//  * the cell id is computed 4 levels at a time from a 1024-entry table in
//    shared memory (each block builds it at start);
//  * binary search: the top ~11 levels come from a sample of the range starts
//    staged in shared memory, the rest from global memory with a fixed number
//    of steps, the 4 points of a lane searched in lockstep so their loads
//    overlap;
//  * learned search: root model -> 32-byte leaf record -> FP32 prediction ->
//    search inside the leaf's error window -> bracket verified, binary search
//    as the fallback (counted);
//  * aggregation: lanes holding the same polygon are grouped with a warp match,
//    the group's count and (split 16/16-bit, exact) attribute sum are reduced
//    in registers and added once by the group leader, into shared memory
//    (P <= SMEM_POLYS, flushed once per block) or straight into global memory.
#include "sdb_internal.cuh"

namespace sdb {

void make_hilbert_lut(HilbertLut* t) {
  for (uint32_t idx = 0; idx < 1024; ++idx) {
    uint32_t sw = (idx >> 9) & 1u, cm = (idx >> 8) & 1u;
    uint32_t xn = (idx >> 4) & 15u, yn = idx & 15u, out = 0;
    for (int lev = 3; lev >= 0; --lev) {
      uint32_t xb = (xn >> lev) & 1u, yb = (yn >> lev) & 1u;
      uint32_t xt = (sw ? yb : xb) ^ cm, yt = (sw ? xb : yb) ^ cm;
      out = (out << 2) | (xt << 1) | (xt ^ yt);
      if (!yt) {
        sw ^= 1u;
        cm ^= xt;
      }
    }
    t->e[idx] = (uint16_t)(out | (((sw << 1) | cm) << 8));
  }
}

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr uint32_t NONE = 0xffffffffu;
constexpr int THREADS = 256;
constexpr uint32_t SMEM_POLYS = 2048;

struct JoinArgs {
  const uint32_t* x;
  const uint32_t* y;
  const int32_t* attr;
  uint64_t n;
  unsigned long long* count;
  unsigned long long* sum;
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
  // learned index
  const LeafRec* leaves;
  float root_a, root_b;
  uint32_t nleaves;
  unsigned long long* fallbacks;
};

__device__ __forceinline__ uint16_t lut_entry(uint32_t idx) {
  uint32_t sw = (idx >> 9) & 1u, cm = (idx >> 8) & 1u;
  uint32_t xn = (idx >> 4) & 15u, yn = idx & 15u, out = 0;
#pragma unroll
  for (int lev = 3; lev >= 0; --lev) {
    uint32_t xb = (xn >> lev) & 1u, yb = (yn >> lev) & 1u;
    uint32_t xt = (sw ? yb : xb) ^ cm, yt = (sw ? xb : yb) ^ cm;
    out = (out << 2) | (xt << 1) | (xt ^ yt);
    if (!yt) {
      sw ^= 1u;
      cm ^= xt;
    }
  }
  return (uint16_t)(out | (((sw << 1) | cm) << 8));
}

// Finest cell id of cell (cx, cy): nsteps table steps of 4 levels each, the
// top step padded with zero levels; st0 cancels the padding's orientation
// changes (each zero level transposes), so the result equals the plain
// F-level id.
__device__ __forceinline__ uint64_t encode_cell(uint32_t cx, uint32_t cy, uint32_t nsteps,
                                                uint32_t st0, const uint16_t* lut) {
  uint64_t h = 0;
  uint32_t st = st0;
  for (int s = (int)nsteps - 1; s >= 0; --s) {
    uint32_t idx = (st << 8) | (((cx >> (4 * s)) & 15u) << 4) | ((cy >> (4 * s)) & 15u);
    uint32_t e = lut[idx];
    h = (h << 8) | (e & 255u);
    st = e >> 8;
  }
  return h;
}

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
                                             const JoinArgs& A) {
  uint64_t lo[G], wlo[G], whi[G];
  uint32_t len[G];
#pragma unroll
  for (int q = 0; q < G; ++q) {
    uint32_t l = root_leaf(A.root_a, A.root_b, A.nleaves, h[q]);
    const uint4* p = reinterpret_cast<const uint4*>(A.leaves + l);
    uint4 u0 = __ldg(p), u1 = __ldg(p + 1);
    LeafRec lr;
    lr.base = (uint64_t)u0.x | ((uint64_t)u0.y << 32);
    lr.a = __uint_as_float(u0.z);
    lr.b = __uint_as_float(u0.w);
    lr.first = u1.x;
    lr.last = u1.y;
    lr.errlo = (int32_t)u1.z;
    lr.errhi = (int32_t)u1.w;
    int64_t pr = leaf_predict(lr, h[q]);
    int64_t a = pr - lr.errlo, b = pr + lr.errhi;
    if (a < (int64_t)lr.first) a = lr.first;
    if (b > (int64_t)lr.last) b = lr.last;
    if (b < a) b = a;
    wlo[q] = (uint64_t)a;
    whi[q] = (uint64_t)b;
    lo[q] = wlo[q];
    len[q] = (uint32_t)(b - a + 1);
  }
  // bracket checks issued with the search: start[wlo] <= h < start[whi + 1]
  uint64_t c0[G], c1[G];
#pragma unroll
  for (int q = 0; q < G; ++q) {
    c0[q] = __ldg(A.start + wlo[q]);
    c1[q] = __ldg(A.start + whi[q] + 1);
  }
  bool more = true;
  while (more) {
    more = false;
    uint64_t v[G];
#pragma unroll
    for (int q = 0; q < G; ++q)
      if (len[q] > 1) v[q] = __ldg(A.start + lo[q] + (len[q] >> 1));
#pragma unroll
    for (int q = 0; q < G; ++q) {
      if (len[q] > 1) {
        uint32_t half = len[q] >> 1;
        if (v[q] <= h[q]) lo[q] += half;
        len[q] -= half;
        more |= len[q] > 1;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < G; ++q) {
    if (c0[q] <= h[q] && h[q] < c1[q]) {
      r[q] = (uint32_t)lo[q];
    } else {
      atomicAdd(A.fallbacks, 1ull);
      r[q] = bs_global(A.start, A.R, h[q]);
    }
  }
}

template <bool SMEM, bool SUM>
__device__ __forceinline__ void agg_warp(uint32_t p, int32_t a, uint32_t* s_cnt,
                                         unsigned long long* s_sum, const JoinArgs& A) {
  unsigned peers = __match_any_sync(FULL, p);
  if (p == NONE) return;
  unsigned c = __popc(peers);
  long long tot = 0;
  if (SUM) {
    int lo = __reduce_add_sync(peers, a & 0xffff);
    int hi = __reduce_add_sync(peers, a >> 16);
    tot = (long long)hi * 65536 + lo;
  }
  if ((threadIdx.x & 31) == (unsigned)(__ffs(peers) - 1)) {
    if (SMEM) {
      atomicAdd(&s_cnt[p], c);
      if (SUM) atomicAdd(&s_sum[p], (unsigned long long)tot);
    } else {
      atomicAdd(&A.count[p], (unsigned long long)c);
      if (SUM) atomicAdd(&A.sum[p], (unsigned long long)tot);
    }
  }
}

template <int LOOKUP, bool SMEM, bool SUM>
__global__ __launch_bounds__(THREADS) void join_kernel(JoinArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long* s_sum = reinterpret_cast<unsigned long long*>(smem);
  size_t off = (SMEM && SUM) ? (size_t)A.P * 8 : 0;
  uint64_t* s_sample = reinterpret_cast<uint64_t*>(smem + off);
  off += (LOOKUP == SDB_LOOKUP_BINARY) ? (size_t)A.sample_n * 8 : 0;
  uint32_t* s_cnt = reinterpret_cast<uint32_t*>(smem + off);
  off += SMEM ? (size_t)A.P * 4 : 0;
  uint16_t* s_lut = reinterpret_cast<uint16_t*>(smem + off);

  for (uint32_t i = threadIdx.x; i < 1024; i += THREADS) s_lut[i] = lut_entry(i);
  if (LOOKUP == SDB_LOOKUP_BINARY)
    for (uint32_t i = threadIdx.x; i < A.sample_n; i += THREADS) s_sample[i] = A.sample[i];
  if (SMEM)
    for (uint32_t i = threadIdx.x; i < A.P; i += THREADS) {
      s_cnt[i] = 0;
      if (SUM) s_sum[i] = 0;
    }
  __syncthreads();

  const int lane = threadIdx.x & 31;
  const uint64_t ngroups = (A.n + 3) >> 2;
  const uint64_t warp = ((uint64_t)blockIdx.x * THREADS + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * THREADS) >> 5;
  const uint32_t gmask = (A.B >= 32) ? 0u : ~((1u << A.B) - 1u);

  for (uint64_t gb = warp * 32; gb < ngroups; gb += nwarps * 32) {
    const uint64_t g = gb + lane;
    uint32_t xs[4], ys[4];
    int32_t as[4];
    bool ok[4];
    const uint64_t e0 = g * 4;
    if (A.vec && e0 + 3 < A.n) {
      uint4 xv = __ldcs(reinterpret_cast<const uint4*>(A.x) + g);
      uint4 yv = __ldcs(reinterpret_cast<const uint4*>(A.y) + g);
      xs[0] = xv.x; xs[1] = xv.y; xs[2] = xv.z; xs[3] = xv.w;
      ys[0] = yv.x; ys[1] = yv.y; ys[2] = yv.z; ys[3] = yv.w;
      if (SUM) {
        int4 av = __ldcs(reinterpret_cast<const int4*>(A.attr) + g);
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
    uint64_t h[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      ok[q] = ok[q] && !((xs[q] | ys[q]) & gmask);
      h[q] = ok[q] ? encode_cell(xs[q] >> A.k, ys[q] >> A.k, A.nsteps, A.st0, s_lut) : 0ull;
    }
    uint32_t r[4];
    if (LOOKUP == SDB_LOOKUP_BINARY)
      find_bs<4>(h, r, s_sample, A);
    else
      find_learned<4>(h, r, A);
    uint32_t pay[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) pay[q] = ok[q] ? __ldg(A.pay + r[q]) : NONE;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const bool multi = pay[q] != NONE && (pay[q] & 0x80000000u);
      agg_warp<SMEM, SUM>(multi ? NONE : pay[q], SUM ? as[q] : 0, s_cnt, s_sum, A);
      if (__any_sync(FULL, multi)) {
        uint32_t lo = 0, n = 0;
        if (multi) {
          uint32_t rr = pay[q] & 0x7fffffffu;
          lo = __ldg(A.list_off + rr);
          n = __ldg(A.list_off + rr + 1) - lo;
        }
        for (uint32_t t = 0; __any_sync(FULL, t < n); ++t)
          agg_warp<SMEM, SUM>(t < n ? __ldg(A.list_ids + lo + t) : NONE, SUM ? as[q] : 0, s_cnt,
                              s_sum, A);
      }
    }
  }

  if (SMEM) {
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < A.P; i += THREADS) {
      if (s_cnt[i]) {
        atomicAdd(&A.count[i], (unsigned long long)s_cnt[i]);
        if (SUM) atomicAdd(&A.sum[i], s_sum[i]);
      }
    }
  }
}

template <int LOOKUP, bool SMEM, bool SUM>
sdb_status launch_t(const JoinArgs& A, cudaStream_t s) {
  size_t smem = 2048;  // table
  if (SMEM) smem += (size_t)A.P * (SUM ? 12 : 4);
  if (LOOKUP == SDB_LOOKUP_BINARY) smem += (size_t)A.sample_n * 8;
  auto kern = join_kernel<LOOKUP, SMEM, SUM>;
  if (smem > 48 * 1024)
    SDB_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  SDB_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, smem));
  if (per_sm < 1) per_sm = 1;
  uint64_t blocks = (uint64_t)num_sms() * per_sm;
  // shared counters are 32-bit: keep each block under 2^31 points
  uint64_t min_blocks = A.n / (1ull << 31) + 1;
  if (blocks < min_blocks) blocks = min_blocks;
  uint64_t need = (A.n + 4 * THREADS - 1) / (4 * THREADS);
  if (blocks > need && need >= min_blocks) blocks = need > 0 ? need : 1;
  kern<<<(unsigned)blocks, THREADS, smem, s>>>(A);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  return SDB_OK;
}

}  // namespace

sdb_status launch_join(const uint32_t* x, const uint32_t* y, const int32_t* attr, uint64_t n,
                       const sdb_covering* cov, int lookup, uint64_t* count, int64_t* sum,
                       cudaStream_t s, bool zero) {
  if (zero) {
    SDB_TRY_CUDA(cudaMemsetAsync(count, 0, (size_t)cov->P * 8, s));
    if (sum) SDB_TRY_CUDA(cudaMemsetAsync(sum, 0, (size_t)cov->P * 8, s));
    if (lookup == SDB_LOOKUP_LEARNED)
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
  A.nsteps = (cov->F + 3) / 4;
  uint32_t pad = 4 * A.nsteps - cov->F;
  A.st0 = (pad & 1u) ? 2u : 0u;  // swap bit set when the padding is odd
  A.P = cov->P;
  A.leaves = cov->leaves;
  A.root_a = cov->root_a;
  A.root_b = cov->root_b;
  A.nleaves = cov->leaf_bits ? (1u << cov->leaf_bits) : 0u;
  A.fallbacks = cov->fallbacks;
  const bool smem = cov->P <= SMEM_POLYS;
  const bool has_sum = sum != nullptr;
  if (lookup == SDB_LOOKUP_BINARY) {
    if (smem) return has_sum ? launch_t<0, true, true>(A, s) : launch_t<0, true, false>(A, s);
    return has_sum ? launch_t<0, false, true>(A, s) : launch_t<0, false, false>(A, s);
  }
  if (smem) return has_sum ? launch_t<1, true, true>(A, s) : launch_t<1, true, false>(A, s);
  return has_sum ? launch_t<1, false, true>(A, s) : launch_t<1, false, false>(A, s);
}

}  // namespace sdb
