// Learned range index over the covering's sorted range starts (Sec. 3, "Point
// Indexing": learning the position of a key in the sorted array to speed up the
// search; RadixSpline is the paper's model, a two-level piecewise-linear model
// is used here).
//
//   root:  leaf(h) = clamp(floor(knot_j + (knot_{j+1} - knot_j) * frac), 0, L-1)  (FP32)
//          with j = h >> wshift, frac = (h - (j << wshift)) / 2^wshift and
//          knot_j = L * #{i : start_i < j << wshift} / R  (2^K uniform knots,
//          K = 12 by default; K = 0 is a single root line over [0, 4^F))
//   leaf:  pred(h) = first + floor(fma(a, float(h - base), b))         (FP32)
//
// Both maps are monotone in h.  The root is the piecewise-linear interpolant of
// the range starts' cumulative distribution, so leaves receive roughly equal
// numbers of ranges even where ranges crowd along polygon boundaries (a single
// line through (start_i, i) routes most ranges to a few leaves: the covering's
// id -> index map is a staircase at every scale).  Leaf l receives exactly the ids h in
// [base_l, base_{l+1}), where base_l is the smallest id the root sends to a
// leaf >= l; it is found by binary search on the root function itself, with the
// same instructions the lookup uses, so routing at fit time and lookup time
// agree bit for bit.  By monotonicity start_i < base_l exactly when the root
// sends start_i to a leaf below l, so one pass over the ranges counts the
// starts below every leaf's base, which fixes each leaf's first and last range.  The leaf line is a least-squares fit of the range index
// (relative to the leaf's first range) on the leaf-relative id.  Its error
// window covers, for every range i the leaf can see, every id of
// [start_i, start_{i+1}) that the leaf receives: by monotonicity it is enough to
// evaluate the prediction at the two ends of each such interval.  Lookups are
// verified anyway and fall back to binary search.
#include "sdb_internal.cuh"

namespace sdb {

namespace {

constexpr unsigned FULL = 0xffffffffu;
// knot j: L * (number of range starts below j << wshift) / R
__global__ void knots_kernel(const uint64_t* __restrict__ start, uint64_t R, uint32_t K,
                             uint32_t wshift, uint32_t L, float* __restrict__ knot) {
  uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j > K) return;
  const uint64_t key = (uint64_t)j << wshift;
  uint64_t lo = 0, len = R;  // first i with start[i] >= key
  while (len > 0) {
    uint64_t half = len >> 1;
    if (start[lo + half] < key) {
      lo += half + 1;
      len -= half + 1;
    } else {
      len = half;
    }
  }
  knot[j] = (float)((double)L * (double)lo / (double)R);
}

// base of every leaf l in [0, L]: smallest h in [0, top] with leaf(h) >= l
__global__ void leaf_base_kernel(const float* __restrict__ knot, uint32_t wshift, float inv_w,
                                 uint32_t L, uint64_t top, uint64_t* __restrict__ base) {
  uint32_t l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l > L) return;
  if (l == 0) {
    base[0] = 0;
    return;
  }
  if (l == L) {
    base[L] = top;
    return;
  }
  uint64_t lo = 0, hi = top;
  while (lo < hi) {
    uint64_t mid = lo + ((hi - lo) >> 1);
    if (root_leaf(knot, wshift, inv_w, L, mid) >= l)
      hi = mid;
    else
      lo = mid + 1;
  }
  base[l] = lo;
}

// fence j: the range start of index j << FENCE_SHIFT (j <= R >> FENCE_SHIFT)
__global__ void fence_kernel(const uint64_t* __restrict__ start, uint64_t nf,
                             uint64_t* __restrict__ fence) {
  const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < nf) fence[j] = start[j << FENCE_SHIFT];
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

__device__ __forceinline__ long long warp_max(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    long long t = __shfl_xor_sync(FULL, v, o);
    v = t > v ? t : v;
  }
  return v;
}

// below[l] = #{i < R : start_i < base_l} for l in [0, L].  Range i's start
// goes to leaf lam_i; the leaves lam_{i-1} < l <= lam_i have exactly i starts
// below their base (lam_{-1} = -1, and start_R = 4^F stands for leaf L).
__global__ void leaf_below_kernel(const uint64_t* __restrict__ start, uint64_t R,
                                  const float* __restrict__ knot, uint32_t wshift, float inv_w,
                                  uint32_t L, uint32_t* __restrict__ below) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > R) return;
  const uint32_t lam = i < R ? root_leaf(knot, wshift, inv_w, L, start[i]) : L;
  const uint32_t from = i == 0 ? 0u : root_leaf(knot, wshift, inv_w, L, start[i - 1]) + 1u;
  for (uint32_t l = from; l <= lam; ++l) below[l] = (uint32_t)i;
}

// one warp per leaf: centred least squares (FP32), error window
__global__ void leaf_fit_kernel(const uint64_t* __restrict__ start, uint64_t R,
                                const uint64_t* __restrict__ base,
                                const uint32_t* __restrict__ below, uint32_t L,
                                LeafRec* __restrict__ leaves) {
  uint32_t l = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (l >= L) return;
  const uint64_t b0 = base[l], b1 = base[l + 1];
  // range holding b0: the last start <= b0 (b0 < 4^F = start[R] for l < L)
  const uint32_t c0 = below[l];
  uint64_t first = (c0 < R && start[c0] == b0) ? c0 : (uint64_t)c0 - 1;
  first = first < R ? first : R - 1;
  LeafRec lr;
  lr.base = b0;
  lr.a = 0.f;
  lr.b = 0.f;
  lr.errlo = 0;
  lr.errhi = 0;
  if (b0 >= b1) {  // no id is routed here
    lr.first = lr.last = (uint32_t)first;
    if (lane == 0) leaves[l] = lr;
    return;
  }
  uint64_t last = (uint64_t)below[l + 1] - 1;  // range holding b1 - 1
  last = last < first ? first : (last < R ? last : R - 1);
  lr.first = (uint32_t)first;
  lr.last = (uint32_t)last;
  const uint64_t n = last - first + 1;
  // pass 1: means; pass 2: centred moments (FP32: the fit only shapes the
  // windows, which come from the lookup's own arithmetic in pass 3)
  float sx = 0.f, sy = 0.f;
  for (uint64_t i = first + lane; i <= last; i += 32) {
    const uint64_t s = start[i] > b0 ? start[i] : b0;
    sx += __ull2float_rn(s - b0);
    sy += (float)(i - first);
  }
  const float inv_n = 1.0f / (float)n;
  const float mx = warp_sum(sx) * inv_n, my = warp_sum(sy) * inv_n;
  float sxx = 0.f, sxy = 0.f;
  for (uint64_t i = first + lane; i <= last; i += 32) {
    const uint64_t s = start[i] > b0 ? start[i] : b0;
    const float dx = __ull2float_rn(s - b0) - mx, dy = (float)(i - first) - my;
    sxx = fmaf(dx, dx, sxx);
    sxy = fmaf(dx, dy, sxy);
  }
  sxx = warp_sum(sxx);
  sxy = warp_sum(sxy);
  const float slope = (sxx > 0.f && sxy > 0.f) ? sxy / sxx : 0.f;
  lr.a = slope;
  lr.b = my - slope * mx;
  // pass 3: error window with the lookup's own FP32 arithmetic
  long long ehi = 0, elo = 0;
  for (uint64_t i = first + lane; i <= last; i += 32) {
    uint64_t lo_h = start[i] > b0 ? start[i] : b0;
    uint64_t hi_h = (start[i + 1] < b1 ? start[i + 1] : b1) - 1;
    long long plo = (long long)leaf_predict(lr, lo_h);
    long long phi = (long long)leaf_predict(lr, hi_h);
    long long up = (long long)i - plo, dn = phi - (long long)i;
    ehi = up > ehi ? up : ehi;
    elo = dn > elo ? dn : elo;
  }
  ehi = warp_max(ehi);
  elo = warp_max(elo);
  const long long CAP = 1ll << 30;
  lr.errhi = (int32_t)(ehi > CAP ? CAP : ehi);
  lr.errlo = (int32_t)(elo > CAP ? CAP : elo);
  if (lane == 0) leaves[l] = lr;
}

}  // namespace

sdb_status build_learned_index(sdb_covering* cov, uint32_t leaf_bits, uint32_t root_bits,
                               cudaStream_t s) {
  TraceScope tr("index.build", s);
  const uint32_t L = 1u << leaf_bits;
  const uint64_t R = cov->R;
  const uint64_t top = 1ull << (2 * cov->F);
  const uint32_t kbits = 2 * cov->F < root_bits ? 2 * cov->F : root_bits;
  const uint32_t K = 1u << kbits;
  const uint32_t wshift = 2 * cov->F - kbits;
  const float inv_w = 1.0f / (float)(1ull << wshift);  // exact: a power of two
  Scratch sc(s);
  if (cov->leaves) dfree(cov->leaves, s);
  if (cov->knots) dfree(cov->knots, s);
  if (cov->fence) dfree(cov->fence, s);
  cov->leaves = nullptr;
  cov->knots = nullptr;
  cov->fence = nullptr;
  const uint64_t nf = (R >> FENCE_SHIFT) + 1;
  SDB_TRY(dalloc_n(&cov->fence, nf, s));
  fence_kernel<<<grid_for(nf, 256), 256, 0, s>>>(cov->start, nf, cov->fence);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  SDB_TRY(dalloc_n(&cov->leaves, L, s));
  if (reinterpret_cast<uintptr_t>(cov->leaves) & 31u) {  // the lookup reads 32 bytes at once
    set_error("learned index: leaf records not 32-byte aligned");
    return SDB_ECUDA;
  }
  SDB_TRY(dalloc_n(&cov->knots, (size_t)K + 1, s));
  if (!cov->fallbacks) {
    SDB_TRY(dalloc_n(&cov->fallbacks, 1, s));
    SDB_TRY_CUDA(cudaMemsetAsync(cov->fallbacks, 0, sizeof(unsigned long long), s));
  }
  knots_kernel<<<grid_for((size_t)K + 1, 256), 256, 0, s>>>(cov->start, R, K, wshift, L, cov->knots);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  uint64_t* base;
  uint32_t* below;
  SDB_TRY(sc.get(&base, (size_t)L + 1));
  SDB_TRY(sc.get(&below, (size_t)L + 1));
  leaf_base_kernel<<<grid_for((size_t)L + 1, 256), 256, 0, s>>>(cov->knots, wshift, inv_w, L, top,
                                                                 base);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  leaf_below_kernel<<<grid_for((size_t)R + 1, 256), 256, 0, s>>>(cov->start, R, cov->knots, wshift,
                                                                   inv_w, L, below);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  leaf_fit_kernel<<<grid_for((size_t)L * 32, 256), 256, 0, s>>>(cov->start, R, base, below, L,
                                                                  cov->leaves);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  SDB_TRY_CUDA(cudaStreamSynchronize(s));
  cov->leaf_bits = leaf_bits;
  cov->knot_bits = kbits;
  cov->knot_wshift = wshift;
  return SDB_OK;
}

}  // namespace sdb
