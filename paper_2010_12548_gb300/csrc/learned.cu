// Learned range index over the covering's sorted range starts (Sec. 3, "Point
// Indexing": learning the position of a key in the sorted array to speed up the
// search; RadixSpline is the paper's model, a two-level piecewise-linear model
// is used here).
//
//   root:  leaf(h) = clamp(floor(fma(ra, float(h), rb)), 0, L-1)       (FP32)
//   leaf:  pred(h) = first + floor(fma(a, float(h - base), b))         (FP32)
//
// Both maps are monotone in h.  The root is a least-squares line through
// (start_i, i * L / R).  Leaf l receives exactly the ids h in
// [base_l, base_{l+1}), where base_l is the smallest id the root sends to a
// leaf >= l; it is found by binary search on the root function itself, with the
// same instructions the lookup uses, so routing at fit time and lookup time
// agree bit for bit.  The leaf line is a least-squares fit of the range index
// (relative to the leaf's first range) on the leaf-relative id.  Its error
// window covers, for every range i the leaf can see, every id of
// [start_i, start_{i+1}) that the leaf receives: by monotonicity it is enough to
// evaluate the prediction at the two ends of each such interval.  Lookups are
// verified anyway and fall back to binary search.
#include "sdb_internal.cuh"

namespace sdb {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int RB = 256;  // root reduction block

__global__ __launch_bounds__(RB) void root_partial_kernel(const uint64_t* __restrict__ start,
                                                          uint64_t R, double inv_top, double inv_R,
                                                          double* __restrict__ part) {
  __shared__ double sh[4][RB];
  double sx = 0, sy = 0, sxx = 0, sxy = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * RB + threadIdx.x; i < R; i += (uint64_t)gridDim.x * RB) {
    double x = (double)start[i] * inv_top, y = (double)i * inv_R;
    sx += x;
    sy += y;
    sxx += x * x;
    sxy += x * y;
  }
  sh[0][threadIdx.x] = sx;
  sh[1][threadIdx.x] = sy;
  sh[2][threadIdx.x] = sxx;
  sh[3][threadIdx.x] = sxy;
  __syncthreads();
  for (int o = RB / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int c = 0; c < 4; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 4) part[blockIdx.x * 4 + threadIdx.x] = sh[threadIdx.x][0];
}

__device__ __forceinline__ uint64_t upper_bound_idx(const uint64_t* __restrict__ start, uint64_t R,
                                                    uint64_t h) {
  // last r in [0, R) with start[r] <= h (start[0] = 0 <= h < start[R])
  uint64_t lo = 0, len = R + 1;
  while (len > 1) {
    uint64_t half = len >> 1;
    if (start[lo + half] <= h) lo += half;
    len -= half;
  }
  return lo;
}

// base of every leaf l in [0, L]: smallest h in [0, top] with leaf(h) >= l
__global__ void leaf_base_kernel(float ra, float rb, uint32_t L, uint64_t top,
                                 uint64_t* __restrict__ base) {
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
    if (root_leaf(ra, rb, L, mid) >= l)
      hi = mid;
    else
      lo = mid + 1;
  }
  base[l] = lo;
}

__device__ __forceinline__ double warp_sum(double v) {
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

// one warp per leaf: range span, centred least squares, error window
__global__ void leaf_fit_kernel(const uint64_t* __restrict__ start, uint64_t R,
                                const uint64_t* __restrict__ base, uint32_t L,
                                LeafRec* __restrict__ leaves) {
  uint32_t l = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (l >= L) return;
  const uint64_t b0 = base[l], b1 = base[l + 1];
  LeafRec lr;
  lr.base = b0;
  lr.a = 0.f;
  lr.b = 0.f;
  lr.errlo = 0;
  lr.errhi = 0;
  if (b0 >= b1) {  // no id is routed here
    uint64_t f = b0 < start[R] ? upper_bound_idx(start, R, b0) : R - 1;
    lr.first = lr.last = (uint32_t)f;
    if (lane == 0) leaves[l] = lr;
    return;
  }
  const uint64_t first = upper_bound_idx(start, R, b0);
  const uint64_t last = upper_bound_idx(start, R, b1 - 1);
  lr.first = (uint32_t)first;
  lr.last = (uint32_t)last;
  const uint64_t n = last - first + 1;
  // pass 1: means
  double sx = 0, sy = 0;
  for (uint64_t i = first + lane; i <= last; i += 32) {
    uint64_t s = start[i] > b0 ? start[i] : b0;
    sx += (double)(s - b0);
    sy += (double)(i - first);
  }
  sx = warp_sum(sx);
  sy = warp_sum(sy);
  const double mx = sx / (double)n, my = sy / (double)n;
  // pass 2: centred moments
  double sxx = 0, sxy = 0;
  for (uint64_t i = first + lane; i <= last; i += 32) {
    uint64_t s = start[i] > b0 ? start[i] : b0;
    double dx = (double)(s - b0) - mx, dy = (double)(i - first) - my;
    sxx += dx * dx;
    sxy += dx * dy;
  }
  sxx = warp_sum(sxx);
  sxy = warp_sum(sxy);
  double slope = (sxx > 0 && sxy > 0) ? sxy / sxx : 0.0;
  lr.a = (float)slope;
  lr.b = (float)(my - slope * mx);
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

sdb_status build_learned_index(sdb_covering* cov, uint32_t leaf_bits, cudaStream_t s) {
  const uint32_t L = 1u << leaf_bits;
  const uint64_t R = cov->R;
  const uint64_t top = 1ull << (2 * cov->F);
  Scratch sc(s);
  // root: least squares of i*L/R on start_i (both scaled to [0, 1))
  const int nb = 256;
  double* part;
  SDB_TRY(sc.get(&part, (size_t)nb * 4));
  root_partial_kernel<<<nb, RB, 0, s>>>(cov->start, R, 1.0 / (double)top, 1.0 / (double)R, part);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  double hp[nb * 4];
  SDB_TRY_CUDA(cudaMemcpyAsync(hp, part, sizeof(hp), cudaMemcpyDeviceToHost, s));
  SDB_TRY_CUDA(cudaStreamSynchronize(s));
  double sx = 0, sy = 0, sxx = 0, sxy = 0;
  for (int b = 0; b < nb; ++b) {
    sx += hp[4 * b];
    sy += hp[4 * b + 1];
    sxx += hp[4 * b + 2];
    sxy += hp[4 * b + 3];
  }
  const double n = (double)R;
  double den = n * sxx - sx * sx, slope = den > 0 ? (n * sxy - sx * sy) / den : 1.0;
  if (!(slope > 0)) slope = 1.0;
  double icpt = (sy - slope * sx) / n;
  // leaf = L * (slope * h / top + icpt)
  cov->root_a = (float)((double)L * slope / (double)top);
  cov->root_b = (float)((double)L * icpt);
  if (!(cov->root_a > 0.f)) cov->root_a = (float)((double)L / (double)top);

  if (cov->leaves) dfree(cov->leaves, s);
  cov->leaves = nullptr;
  SDB_TRY(dalloc_n(&cov->leaves, L, s));
  if (!cov->fallbacks) {
    SDB_TRY(dalloc_n(&cov->fallbacks, 1, s));
    SDB_TRY_CUDA(cudaMemsetAsync(cov->fallbacks, 0, sizeof(unsigned long long), s));
  }
  uint64_t* base;
  SDB_TRY(sc.get(&base, (size_t)L + 1));
  leaf_base_kernel<<<grid_for((size_t)L + 1, 256), 256, 0, s>>>(cov->root_a, cov->root_b, L, top,
                                                                 base);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  leaf_fit_kernel<<<grid_for((size_t)L * 32, 256), 256, 0, s>>>(cov->start, R, base, L,
                                                                  cov->leaves);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  SDB_TRY_CUDA(cudaStreamSynchronize(s));
  cov->leaf_bits = leaf_bits;
  return SDB_OK;
}

}  // namespace sdb
