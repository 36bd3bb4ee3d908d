// Cell table: a direct-mapped first level over the covering's finest cell ids
// (Sec. 3, "Polygon Indexing": ACT is a radix tree over the cell ids in which
// large cells are met near the root; here one flat array holds the level
// L0 = T / 2 of that tree).
//
// The ids [0, 4^F) split into 2^T buckets of 2^shift consecutive ids
// (T even, shift = 2F - T): bucket b covers [b << shift, (b + 1) << shift),
// the descendants of the cell of level L0 whose id is b (the curve's prefix
// property).  The table is stored in row-major order of those cells, so a
// point finds its entry from its coordinates alone, (y >> (B - L0)) << L0 |
// (x >> (B - L0)), with no curve encoding.  With r0 and r1 the ranges holding
// the bucket's first and last id:
//   r0 == r1: entry = pay[r0]               (the range's payload, as stored)
//   r0 <  r1: entry = TAB_MIXED | m, win[m] = (r0, r1), m = rank of the cell
//             among the mixed cells in row-major order
// A payload is 0xFFFFFFFF (no polygon), < 2^31 (one polygon), or 2^31 | r with
// r < R; with R < 2^30 - 1 the values TAB_MIXED | m (m < 2^30 - 1) are disjoint
// from all of them.  For a mixed cell the range of a point's finest id h is the
// last r in [r0, r1] with start[r] <= h.
#include <algorithm>

#include "hilbert.cuh"
#include "sdb_internal.cuh"

namespace sdb {

namespace {

// last r in [0, R] with start[r] <= h (start[0] = 0 <= h)
__device__ __forceinline__ uint32_t last_le(const uint64_t* __restrict__ start, uint64_t R,
                                            uint64_t h) {
  uint64_t lo = 0, len = R + 1;
  while (len > 1) {
    const uint64_t half = len >> 1;
    if (__ldg(start + lo + half) <= h) lo += half;
    len -= half;
  }
  return (uint32_t)lo;
}

// the Hilbert id at level L0 of the cell at row-major position c
__device__ __forceinline__ uint64_t cell_bucket(uint64_t c, uint32_t L0, uint32_t nsteps,
                                                uint32_t st0, const uint32_t* s_tab) {
  const uint32_t cx = (uint32_t)(c & ((1ull << L0) - 1)), cy = (uint32_t)(c >> L0);
  return hilbert3_encode(cx, cy, nsteps, st0, s_tab);
}

__global__ void table_class_kernel(const uint64_t* __restrict__ start, uint64_t R,
                                   const uint32_t* __restrict__ pay, uint32_t shift, uint32_t L0,
                                   uint32_t nsteps, uint32_t st0, uint64_t nb,
                                   uint32_t* __restrict__ tab, uint32_t* __restrict__ mixed) {
  __shared__ uint32_t s_tab[HILBERT3_SMEM_WORDS];
  hilbert3_fill(s_tab);
  __syncthreads();
  for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c < nb;
       c += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t b = cell_bucket(c, L0, nsteps, st0, s_tab);
    const uint64_t lo = b << shift, hi = lo + ((1ull << shift) - 1);
    const uint32_t r0 = last_le(start, R, lo);
    // the bucket meets several ranges iff the next range starts inside it
    const bool mix = start[r0 + 1] <= hi;
    mixed[c] = mix ? 1u : 0u;
    if (!mix) tab[c] = pay[r0];
  }
}

__global__ void table_mixed_kernel(const uint64_t* __restrict__ start, uint64_t R,
                                   uint32_t shift, uint32_t L0, uint32_t nsteps, uint32_t st0,
                                   uint64_t nb, const uint32_t* __restrict__ mixed,
                                   const uint32_t* __restrict__ rank, uint32_t* __restrict__ tab,
                                   uint2* __restrict__ win) {
  __shared__ uint32_t s_tab[HILBERT3_SMEM_WORDS];
  hilbert3_fill(s_tab);
  __syncthreads();
  for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c < nb;
       c += (uint64_t)gridDim.x * blockDim.x) {
    if (!mixed[c]) continue;
    const uint64_t b = cell_bucket(c, L0, nsteps, st0, s_tab);
    const uint64_t lo = b << shift, hi = lo + ((1ull << shift) - 1);
    const uint32_t m = rank[c];
    tab[c] = TAB_MIXED | m;
    win[m] = make_uint2(last_le(start, R, lo), last_le(start, R, hi));
  }
}

}  // namespace

sdb_status build_cell_table(sdb_covering* cov, uint32_t table_bits, cudaStream_t s) {
  TraceScope tr("table.build", s);
  if (cov->R >= (uint64_t)TAB_MIXED_MAX) {
    set_error("cell table: %llu ranges, at most %u supported", (unsigned long long)cov->R,
              TAB_MIXED_MAX - 1);
    return SDB_EINVAL;
  }
  // whole quadtree levels: a bucket is a cell of level T / 2
  const uint32_t T = (table_bits & ~1u) < 2 * cov->F ? (table_bits & ~1u) : 2 * cov->F;
  const uint32_t shift = 2 * cov->F - T;
  const uint64_t nb = 1ull << T;
  if (cov->tab) dfree(cov->tab, s);
  if (cov->win) dfree(cov->win, s);
  cov->tab = nullptr;
  cov->win = nullptr;
  cov->tab_bits = 0;
  cov->tab_mixed = 0;
  Scratch sc(s);
  uint32_t *mixed, *rank, *dtot;
  SDB_TRY(dalloc_n(&cov->tab, nb, s));
  SDB_TRY(sc.get(&mixed, nb));
  SDB_TRY(sc.get(&rank, nb));
  SDB_TRY(sc.get(&dtot, 1));
  uint32_t nsteps, st0;
  hilbert3_params(T / 2, &nsteps, &st0);
  // a few blocks per SM (each fills the curve table in shared memory once)
  const unsigned grid = (unsigned)std::min<uint64_t>(grid_for(nb, 256), (uint64_t)num_sms() * 8);
  table_class_kernel<<<grid, 256, 0, s>>>(cov->start, cov->R, cov->pay, shift, T / 2,
                                                        nsteps, st0, nb, cov->tab, mixed);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  SDB_TRY(exclusive_scan<uint32_t>(mixed, rank, nb, dtot, s));
  uint32_t M = 0;
  SDB_TRY_CUDA(cudaMemcpyAsync(&M, dtot, 4, cudaMemcpyDeviceToHost, s));
  SDB_TRY_CUDA(cudaStreamSynchronize(s));
  if (M > 0) {
    SDB_TRY(dalloc_n(&cov->win, M, s));
    table_mixed_kernel<<<grid, 256, 0, s>>>(cov->start, cov->R, shift, T / 2, nsteps,
                                                          st0, nb, mixed, rank, cov->tab, cov->win);
    note_launch();
    SDB_TRY_CUDA(cudaGetLastError());
  }
  SDB_TRY_CUDA(cudaStreamSynchronize(s));
  cov->tab_bits = T;
  cov->tab_shift = shift;
  cov->tab_mixed = M;
  return SDB_OK;
}

}  // namespace sdb
