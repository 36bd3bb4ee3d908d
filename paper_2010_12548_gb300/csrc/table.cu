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
//   r0 <  r1: entry = TAB_MIXED | m, win[m] = (r0, r1), m = rank of the bucket
//             among the mixed buckets
// r0 for every bucket comes from one pass over the ranges (each range marks the
// first bucket starting inside it) and a prefix maximum over the buckets in
// curve order; the entries are then written at the cells' row-major places.
// A payload is 0xFFFFFFFF (no polygon), < 2^31 (one polygon), or 2^31 | r with
// r < R; with R < 2^30 - 1 the values TAB_MIXED | m (m < 2^30 - 1) are disjoint
// from all of them.  For a mixed cell the range of a point's finest id h is the
// last r in [r0, r1] with start[r] <= h.
//
// A second level (the next levels of the same tree) splits each mixed bucket
// into up to 8 x 8 sub-cells, stored row-major per bucket with the same entry
// encoding (TAB_MIXED | m2 indexing win2), so a point in a mixed bucket makes
// one more read and searches only when its sub-cell meets several ranges.
#include "sdb_internal.cuh"

#include <algorithm>
#include <vector>

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

// the row-major position of the cell of level L0 whose curve id is b: the
// digits from the top (plain orientation there) give the transformed quadrant
// (xt, yt) = (d >> 1, (d >> 1) ^ (d & 1)), undone by the orientation (sw, cm);
// yt = 0 transposes, and also complements when xt = 1
__device__ __forceinline__ uint64_t bucket_cell(uint64_t b, uint32_t L0) {
  uint32_t sw = 0, cm = 0, cx = 0, cy = 0;
  for (int lev = (int)L0 - 1; lev >= 0; --lev) {
    const uint32_t d = (uint32_t)(b >> (2 * lev)) & 3u;
    const uint32_t xt = d >> 1, yt = xt ^ (d & 1u);
    const uint32_t u = xt ^ cm, v = yt ^ cm;
    cx = (cx << 1) | (sw ? v : u);
    cy = (cy << 1) | (sw ? u : v);
    if (!yt) {
      sw ^= 1u;
      cm ^= xt;
    }
  }
  return ((uint64_t)cy << L0) | cx;
}

// mark[b] = the last range r with first bucket fb(r) = b, where fb(r) is the
// first bucket whose first id is >= start[r] (ranges are sorted: r is the last
// one when fb(r + 1) differs, so each mark has one writer)
__global__ void table_marks_kernel(const uint64_t* __restrict__ start, uint64_t R, uint32_t shift,
                                   uint64_t nb, uint32_t* __restrict__ mark) {
  const uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  const uint64_t round = (1ull << shift) - 1;
  const uint64_t b = (start[r] + round) >> shift;
  const uint64_t bn = r + 1 < R ? (start[r + 1] + round) >> shift : nb;
  if (b < nb && bn != b) mark[b] = (uint32_t)r;
}

// r0(b) = max(mark[0..b]): the range holding bucket b's first id.  A tile of
// TT buckets per block: tile maxima, their exclusive max-scan, then the scan
// within each tile.
constexpr int TT = 2048, TB = 256;

__device__ __forceinline__ uint32_t warp_incl_max(uint32_t v) {
  const uint32_t lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= (uint32_t)o) v = max(v, t);
  }
  return v;
}

__global__ __launch_bounds__(TB) void tile_max_kernel(const uint32_t* __restrict__ mark, uint64_t nb,
                                                      uint32_t* __restrict__ tmax) {
  __shared__ uint32_t s[TB / 32];
  const uint64_t b0 = (uint64_t)blockIdx.x * TT;
  uint32_t m = 0;
  for (uint32_t i = threadIdx.x; i < TT && b0 + i < nb; i += TB) m = max(m, mark[b0 + i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < TB / 32; ++w) m = max(m, s[w]);
    tmax[blockIdx.x] = m;
  }
}

// exclusive max-scan of the tile maxima, one block of 1024 threads
__global__ __launch_bounds__(1024) void tile_prefix_kernel(uint32_t* __restrict__ tmax, uint32_t nt) {
  __shared__ uint32_t s[32];
  __shared__ uint32_t carry;
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t base = 0; base < nt; base += 1024) {
    const uint32_t i = base + threadIdx.x;
    const uint32_t v = i < nt ? tmax[i] : 0u;
    const uint32_t inc = warp_incl_max(v);
    if (lane == 31) s[w] = inc;
    __syncthreads();
    if (w == 0) s[lane] = warp_incl_max(s[lane]);
    __syncthreads();
    const uint32_t wpre = w ? s[w - 1] : 0u;  // maximum over earlier warps
    uint32_t prev = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane == 0) prev = 0;                  // maximum over earlier lanes
    const uint32_t c = carry;
    __syncthreads();
    if (i < nt) tmax[i] = max(c, max(wpre, prev));
    if (threadIdx.x == 1023) carry = max(c, max(wpre, inc));
    __syncthreads();
  }
}

// per bucket (curve order): r0 = max-scan of the marks; a bucket inside one
// range stores that range's payload at its cell's row-major position, a
// bucket that meets several ranges is flagged
__global__ __launch_bounds__(TB) void table_fill_kernel(
    const uint32_t* __restrict__ mark, const uint32_t* __restrict__ tpre, uint64_t nb,
    const uint64_t* __restrict__ start, const uint32_t* __restrict__ pay, uint32_t shift,
    uint32_t L0, uint32_t* __restrict__ tab, uint32_t* __restrict__ mixed) {
  __shared__ uint32_t s[TB / 32];
  __shared__ uint32_t carry;
  const uint64_t b0 = (uint64_t)blockIdx.x * TT;
  if (threadIdx.x == 0) carry = tpre[blockIdx.x];
  __syncthreads();
  for (uint32_t base = 0; base < TT && b0 + base < nb; base += TB) {
    const uint64_t b = b0 + base + threadIdx.x;
    const uint32_t v = b < nb ? mark[b] : 0u;
    const uint32_t inc = warp_incl_max(v);
    if ((threadIdx.x & 31) == 31) s[threadIdx.x >> 5] = inc;
    __syncthreads();
    uint32_t wpre = 0;
    for (uint32_t w = 0; w < (threadIdx.x >> 5); ++w) wpre = max(wpre, s[w]);
    const uint32_t c = carry;
    const uint32_t r0 = max(c, max(wpre, inc));
    if (b < nb) {
      const uint64_t lo = b << shift, hi = lo + ((1ull << shift) - 1);
      // the bucket meets several ranges iff the next range starts inside it
      const bool mix = start[r0 + 1] <= hi;
      mixed[b] = mix ? 1u : 0u;
      if (!mix) tab[bucket_cell(b, L0)] = pay[r0];
    }
    __syncthreads();
    if (threadIdx.x == TB - 1) carry = r0;
    __syncthreads();
  }
}

__global__ void table_mixed_kernel(const uint64_t* __restrict__ start, uint64_t R,
                                   uint32_t shift, uint32_t L0, uint64_t nb,
                                   const uint32_t* __restrict__ mixed,
                                   const uint32_t* __restrict__ rank, uint32_t* __restrict__ tab,
                                   uint2* __restrict__ win, uint32_t* __restrict__ mpos) {
  for (uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; b < nb;
       b += (uint64_t)gridDim.x * blockDim.x) {
    if (!mixed[b]) continue;
    const uint64_t lo = b << shift, hi = lo + ((1ull << shift) - 1);
    const uint32_t m = rank[b];
    const uint64_t pos = bucket_cell(b, L0);
    tab[pos] = TAB_MIXED | m;
    win[m] = make_uint2(last_le(start, R, lo), last_le(start, R, hi));
    mpos[m] = (uint32_t)pos;
  }
}

// last r in [a, b] with start[r] <= h (start[a] <= h)
__device__ __forceinline__ uint32_t last_le_in(const uint64_t* __restrict__ start, uint32_t a,
                                               uint32_t b, uint64_t h) {
  uint32_t lo = a, len = b - a + 1;
  while (len > 1) {
    const uint32_t half = len >> 1;
    if (__ldg(start + lo + half) <= h) lo += half;
    len -= half;
  }
  return lo;
}

// The second level.  Mixed bucket m (row-major cell pos = mpos[m] of level L0)
// splits into S x S sub-cells of level L1 = L0 + s2 (S = 2^s2), stored
// row-major within the bucket at sub[m * S^2 + (sy << s2 | sx)].  A sub-cell is
// again a quadtree cell, so its finest ids are one contiguous block
// [hs << 2 (F - L1), (hs + 1) << 2 (F - L1)), hs its curve id at level L1; the
// ranges holding the block's first and last id lie in the bucket's window.
// Pass 1 (write = false) flags the sub-cells that meet several ranges and
// stores the payload of the others; pass 2 writes TAB_MIXED | m2 and the
// window of the m2-th flagged sub-cell.
__global__ void table_sub_kernel(const uint64_t* __restrict__ start, const uint32_t* __restrict__ pay,
                                 const uint2* __restrict__ win, const uint32_t* __restrict__ mpos,
                                 uint64_t M, uint32_t L0, uint32_t s2, uint32_t F,
                                 uint32_t* __restrict__ sub, uint32_t* __restrict__ flag,
                                 const uint32_t* __restrict__ rank2, uint2* __restrict__ win2,
                                 bool write) {
  const uint64_t per = 1ull << (2 * s2);
  const uint32_t L1 = L0 + s2, sh = 2 * (F - L1);
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < M * per;
       t += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t m = t >> (2 * s2);
    const uint32_t j = (uint32_t)(t & (per - 1));
    if (write && !flag[t]) continue;
    const uint32_t pos = mpos[m];
    const uint32_t cx = pos & ((1u << L0) - 1u), cy = pos >> L0;
    const uint32_t sx = j & ((1u << s2) - 1u), sy = j >> s2;
    const uint64_t hs = hilbert_id((cx << s2) | sx, (cy << s2) | sy, L1);
    const uint64_t lo = hs << sh, hi = lo + ((1ull << sh) - 1);
    const uint2 w = win[m];
    const uint32_t r0 = last_le_in(start, w.x, w.y, lo), r1 = last_le_in(start, r0, w.y, hi);
    if (!write) {
      flag[t] = r0 != r1 ? 1u : 0u;
      if (r0 == r1) sub[t] = pay[r0];
    } else {
      const uint32_t m2 = rank2[t];
      sub[t] = TAB_MIXED | m2;
      win2[m2] = make_uint2(r0, r1);
    }
  }
}

// The top level: cell (tx, ty) of level Lt covers the 2^d x 2^d cells of the
// table's level L0 = Lt + d below it.  When all of them hold the same
// single-polygon payload p (no mixed cell, no list, no boundary flag) the whole
// cell lies in one range -- its ids are contiguous and the canonical covering
// merges equal neighbours, so cells with equal payloads side by side belong to
// one range -- and the cell's word is p; all empty gives TOP_WORD_NONE;
// anything else TOP_WORD_ASK (the table decides).  The words then become one
// byte each through a palette of the most frequent payloads.
constexpr uint32_t TOP_WORD_ASK = 0xFFFFFFFEu, TOP_WORD_NONE = 0xFFFFFFFFu;

__global__ void table_top_kernel(const uint32_t* __restrict__ tab, uint32_t L0, uint32_t Lt,
                                 uint32_t* __restrict__ word) {
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= (1u << (2 * Lt))) return;
  const uint32_t d = L0 - Lt, tx = c & ((1u << Lt) - 1u), ty = c >> Lt;
  const uint32_t first = tab[((size_t)(ty << d) << L0) | (tx << d)];
  bool same = true;
  for (uint32_t j = 0; j < (1u << d) && same; ++j)
    for (uint32_t i = 0; i < (1u << d); ++i)
      if (tab[((size_t)((ty << d) + j) << L0) | ((tx << d) + i)] != first) {
        same = false;
        break;
      }
  uint32_t v = TOP_WORD_ASK;
  if (same) {
    if (first == 0xFFFFFFFFu)
      v = TOP_WORD_NONE;
    else if (first < 0x40000000u)  // one polygon (its slot), no boundary flag
      v = first;
  }
  word[c] = v;
}

// occurrences of each single-polygon payload among the top level's cells
__global__ void top_count_kernel(const uint32_t* __restrict__ word, uint32_t nt,
                                 uint32_t* __restrict__ count) {
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < nt && word[c] < TOP_WORD_ASK) atomicAdd(&count[word[c]], 1u);
}

// the byte of each cell: its payload's palette index (map), or TOP_NONE / TOP_ASK
__global__ void top_byte_kernel(const uint32_t* __restrict__ word, uint32_t nt,
                                const uint8_t* __restrict__ map, uint8_t* __restrict__ top) {
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nt) return;
  const uint32_t v = word[c];
  top[c] = v == TOP_WORD_NONE ? TOP_NONE : (v == TOP_WORD_ASK ? TOP_ASK : map[v]);
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
  if (cov->sub) dfree(cov->sub, s);
  if (cov->win2) dfree(cov->win2, s);
  if (cov->top) dfree(cov->top, s);
  if (cov->top_pal) dfree(cov->top_pal, s);
  cov->top_pal = nullptr;
  cov->tab = nullptr;
  cov->win = nullptr;
  cov->sub = nullptr;
  cov->win2 = nullptr;
  cov->top = nullptr;
  cov->top_level = 0;
  cov->tab_bits = 0;
  cov->tab_mixed = 0;
  cov->sub_bits = 0;
  cov->sub_mixed = 0;
  Scratch sc(s);
  uint32_t *mixed, *rank, *dtot, *mark, *tpre;
  const uint64_t nt = (nb + TT - 1) / TT;
  SDB_TRY(dalloc_n(&cov->tab, nb, s));
  SDB_TRY(sc.get(&mixed, nb));
  SDB_TRY(sc.get(&rank, nb));
  SDB_TRY(sc.get(&mark, nb));
  SDB_TRY(sc.get(&tpre, nt));
  SDB_TRY(sc.get(&dtot, 1));
  SDB_TRY_CUDA(cudaMemsetAsync(mark, 0, nb * 4, s));
  table_marks_kernel<<<grid_for(cov->R, 256), 256, 0, s>>>(cov->start, cov->R, shift, nb, mark);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  tile_max_kernel<<<(unsigned)nt, TB, 0, s>>>(mark, nb, tpre);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  tile_prefix_kernel<<<1, 1024, 0, s>>>(tpre, (uint32_t)nt);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  table_fill_kernel<<<(unsigned)nt, TB, 0, s>>>(mark, tpre, nb, cov->start, cov->pay, shift, T / 2,
                                                cov->tab, mixed);
  note_launch();
  SDB_TRY_CUDA(cudaGetLastError());
  const unsigned grid = grid_for(nb, 256);
  SDB_TRY(exclusive_scan<uint32_t>(mixed, rank, nb, dtot, s));
  uint32_t M = 0;
  SDB_TRY_CUDA(cudaMemcpyAsync(&M, dtot, 4, cudaMemcpyDeviceToHost, s));
  SDB_TRY_CUDA(cudaStreamSynchronize(s));
  // second level: sub-cells of 2^s2 x 2^s2 per mixed bucket, s2 <= 3 whole
  // levels above the finest, while the sub-cell count keeps indices in range
  const uint32_t L0 = T / 2;
  uint32_t s2 = cov->F - L0 < 3 ? cov->F - L0 : 3;
  while (s2 > 0 && (uint64_t)M << (2 * s2) >= (uint64_t)TAB_MIXED_MAX) --s2;
  uint64_t M2 = 0;
  if (M > 0) {
    uint32_t* mpos;
    SDB_TRY(sc.get(&mpos, M));
    SDB_TRY(dalloc_n(&cov->win, M, s));
    table_mixed_kernel<<<grid, 256, 0, s>>>(cov->start, cov->R, shift, L0, nb, mixed, rank,
                                            cov->tab, cov->win, mpos);
    note_launch();
    SDB_TRY_CUDA(cudaGetLastError());
    if (s2 > 0) {
      const uint64_t ns = M << (2 * s2);
      uint32_t *flag2, *rank2;
      SDB_TRY(dalloc_n(&cov->sub, ns, s));
      SDB_TRY(sc.get(&flag2, ns));
      SDB_TRY(sc.get(&rank2, ns));
      const unsigned g2 = grid_for(ns, 256);
      table_sub_kernel<<<g2, 256, 0, s>>>(cov->start, cov->pay, cov->win, mpos, M, L0, s2,
                                          cov->F, cov->sub, flag2, nullptr, nullptr, false);
      note_launch();
      SDB_TRY_CUDA(cudaGetLastError());
      SDB_TRY(exclusive_scan<uint32_t>(flag2, rank2, ns, dtot, s));
      uint32_t m2 = 0;
      SDB_TRY_CUDA(cudaMemcpyAsync(&m2, dtot, 4, cudaMemcpyDeviceToHost, s));
      SDB_TRY_CUDA(cudaStreamSynchronize(s));
      M2 = m2;
      if (M2 > 0) {
        SDB_TRY(dalloc_n(&cov->win2, M2, s));
        table_sub_kernel<<<g2, 256, 0, s>>>(cov->start, cov->pay, cov->win, mpos, M, L0, s2,
                                            cov->F, cov->sub, flag2, rank2, cov->win2, true);
        note_launch();
        SDB_TRY_CUDA(cudaGetLastError());
      }
    }
  }
  // the top level for shared memory (levels 4 .. TOP_MAX_LEVEL): the cells'
  // words on the device, the palette and the byte per cell on the host
  if (L0 >= 4) {
    const uint32_t Lt = L0 < TOP_MAX_LEVEL ? L0 : TOP_MAX_LEVEL;
    const uint32_t nt = 1u << (2 * Lt);
    uint32_t* word;
    SDB_TRY(sc.get(&word, nt));
    table_top_kernel<<<(nt + 255) / 256, 256, 0, s>>>(cov->tab, L0, Lt, word);
    note_launch();
    SDB_TRY_CUDA(cudaGetLastError());
    // payloads are polygon slots (< P): count them on the device, pick the
    // palette on the host from P counts, map the cells on the device
    const uint32_t P = cov->P;
    uint32_t* cnt;
    uint8_t* dmap;
    SDB_TRY(sc.get(&cnt, P));
    SDB_TRY(sc.get(&dmap, P));
    SDB_TRY_CUDA(cudaMemsetAsync(cnt, 0, (size_t)P * 4, s));
    top_count_kernel<<<(nt + 255) / 256, 256, 0, s>>>(word, nt, cnt);
    note_launch();
    SDB_TRY_CUDA(cudaGetLastError());
    std::vector<uint32_t> hc(P);
    SDB_TRY_CUDA(cudaMemcpyAsync(hc.data(), cnt, (size_t)P * 4, cudaMemcpyDeviceToHost, s));
    SDB_TRY_CUDA(cudaStreamSynchronize(s));
    // the most frequent payloads (ties by slot) take the palette's slots
    std::vector<uint32_t> order;
    for (uint32_t j = 0; j < P; ++j)
      if (hc[j]) order.push_back(j);
    const size_t keep = std::min<size_t>(order.size(), TOP_PALETTE);
    auto more = [&](uint32_t a, uint32_t b) { return hc[a] != hc[b] ? hc[a] > hc[b] : a < b; };
    std::partial_sort(order.begin(), order.begin() + keep, order.end(), more);
    std::vector<uint32_t> pal(TOP_PALETTE, 0xFFFFFFFFu);
    std::vector<uint8_t> map(P, TOP_ASK);
    for (size_t i = 0; i < keep; ++i) {
      pal[i] = order[i];
      map[order[i]] = (uint8_t)i;
    }
    SDB_TRY(dalloc_n(&cov->top, nt, s));
    SDB_TRY(dalloc_n(&cov->top_pal, TOP_PALETTE, s));
    SDB_TRY_CUDA(cudaMemcpyAsync(dmap, map.data(), P, cudaMemcpyHostToDevice, s));
    SDB_TRY_CUDA(cudaMemcpyAsync(cov->top_pal, pal.data(), TOP_PALETTE * 4,
                                 cudaMemcpyHostToDevice, s));
    top_byte_kernel<<<(nt + 255) / 256, 256, 0, s>>>(word, nt, dmap, cov->top);
    note_launch();
    SDB_TRY_CUDA(cudaGetLastError());
    cov->top_level = Lt;
  }
  SDB_TRY_CUDA(cudaStreamSynchronize(s));
  cov->tab_bits = T;
  cov->tab_shift = shift;
  cov->tab_mixed = M;
  cov->sub_bits = cov->sub ? s2 : 0;
  cov->sub_mixed = M2;
  return SDB_OK;
}

}  // namespace sdb
