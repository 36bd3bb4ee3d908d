// Finest-level Hilbert cell ids on the GPU, three levels per table step
// (Sec. 3: a point is mapped to its cell on the finest grid level, and cells
// are numbered along the Hilbert curve).
//
// The curve is the quadrant-digit variant of hilbert_id(): at every level the
// current orientation is a pair (sw, cm) (transpose, complement), the digit of
// the transformed quadrant (xt, yt) is (xt << 1) | (xt ^ yt), and a quadrant
// with yt = 0 toggles sw and, when xt = 1, also cm.
//
// One table entry maps (sw, cm, 3 bits of x, 3 bits of y) to the 6 id bits of
// those levels and the orientation after them, in one byte (256 entries).  In
// shared memory the 64 words of the table are stored once per bank, word w of
// lane l at [w * 32 + l], so a warp's 32 lookups never conflict (8 KB); kernels
// in which few points encode keep one unreplicated copy (256 bytes).
// A level count F that is not a multiple of 3 is padded with zero levels on
// top; each zero level transposes, so the walk starts with sw set when the
// padding is odd and reaches the real top level in the plain orientation.
#pragma once
#include <cstdint>

namespace sdb {

constexpr int HILBERT3_WORDS = 64;
constexpr int HILBERT3_SMEM_WORDS = HILBERT3_WORDS * 32;
constexpr int HILBERT3_SMEM_BYTES = HILBERT3_SMEM_WORDS * 4;

// idx = sw << 7 | cm << 6 | x3 << 3 | y3 -> id bits (low 6) | orientation << 6
__host__ __device__ __forceinline__ uint32_t hilbert3_entry(uint32_t idx) {
  uint32_t sw = (idx >> 7) & 1u, cm = (idx >> 6) & 1u;
  const uint32_t xn = (idx >> 3) & 7u, yn = idx & 7u;
  uint32_t out = 0;
#pragma unroll
  for (int lev = 2; lev >= 0; --lev) {
    const uint32_t xb = (xn >> lev) & 1u, yb = (yn >> lev) & 1u;
    const uint32_t xt = (sw ? yb : xb) ^ cm, yt = (sw ? xb : yb) ^ cm;
    out = (out << 2) | (xt << 1) | (xt ^ yt);
    if (!yt) {
      sw ^= 1u;
      cm ^= xt;
    }
  }
  return out | (((sw << 1) | cm) << 6);
}

// fills the replicated table; the caller synchronises the block afterwards
__device__ __forceinline__ void hilbert3_fill(uint32_t* tab) {
  for (int i = threadIdx.x; i < HILBERT3_SMEM_WORDS; i += blockDim.x) {
    const uint32_t w = (uint32_t)i >> 5;
    tab[i] = hilbert3_entry(4 * w) | (hilbert3_entry(4 * w + 1) << 8) |
             (hilbert3_entry(4 * w + 2) << 16) | (hilbert3_entry(4 * w + 3) << 24);
  }
}

// table steps and starting orientation for F levels
__host__ __device__ inline void hilbert3_params(uint32_t F, uint32_t* nsteps, uint32_t* st0) {
  *nsteps = (F + 2) / 3;
  *st0 = ((3 * *nsteps - F) & 1u) ? 2u : 0u;
}

// One table step: the 3 top bits of xs and ys (coordinates shifted to the top
// of the word) with the orientation st (already shifted left by 6) select a
// table byte: 6 id bits and the next orientation.
__device__ __forceinline__ uint32_t hilbert3_step(uint32_t& xs, uint32_t& ys, uint32_t& st,
                                                  const uint32_t* row) {
  const uint32_t idx = st | ((xs >> 26) & 0x38u) | (ys >> 29);
  xs <<= 3;
  ys <<= 3;
  // the byte idx & 3 of the table word, upper bytes zero
  const uint32_t e = __byte_perm(row[(idx >> 2) << 5], 0u, 0x4440u | (idx & 3u));
  st = e & 0xc0u;
  return e & 63u;
}

// The same table once, unreplicated (64 words, 256 bytes): for kernels in which
// only a few points encode their cell id, so bank conflicts are rare and the
// shared memory is better left to the L1 cache.
constexpr int HILBERT3_COMPACT_BYTES = HILBERT3_WORDS * 4;

__device__ __forceinline__ void hilbert3_fill_compact(uint32_t* tab) {
  for (int w = threadIdx.x; w < HILBERT3_WORDS; w += blockDim.x)
    tab[w] = hilbert3_entry(4 * w) | (hilbert3_entry(4 * w + 1) << 8) |
             (hilbert3_entry(4 * w + 2) << 16) | (hilbert3_entry(4 * w + 3) << 24);
}

// id of cell (cx, cy) at the level the parameters were made for (cx, cy < 2^F),
// from the unreplicated table
__device__ __forceinline__ uint64_t hilbert3_encode_compact(uint32_t cx, uint32_t cy,
                                                            uint32_t nsteps, uint32_t st0,
                                                            const uint32_t* tab) {
  if (nsteps == 0) return 0;
  const uint32_t sh = 32 - 3 * nsteps;
  uint32_t xs = cx << sh, ys = cy << sh, st = st0 << 6;
  uint64_t h = 0;
  for (uint32_t s = 0; s < nsteps; ++s) {
    const uint32_t idx = st | ((xs >> 26) & 0x38u) | (ys >> 29);
    xs <<= 3;
    ys <<= 3;
    const uint32_t e = __byte_perm(tab[idx >> 2], 0u, 0x4440u | (idx & 3u));
    st = e & 0xc0u;
    h = (h << 6) | (e & 63u);
  }
  return h;
}

// id of cell (cx, cy) at the level the parameters were made for (cx, cy < 2^F)
__device__ __forceinline__ uint64_t hilbert3_encode(uint32_t cx, uint32_t cy, uint32_t nsteps,
                                                    uint32_t st0, const uint32_t* tab) {
  if (nsteps == 0) return 0;
  const uint32_t* row = tab + (threadIdx.x & 31u);
  const uint32_t sh = 32 - 3 * nsteps;  // nsteps <= 10: the 3 * nsteps bits at the top
  uint32_t xs = cx << sh, ys = cy << sh, st = st0 << 6;
  uint64_t h = 0;
  for (uint32_t s = 0; s < nsteps; ++s) h = (h << 6) | hilbert3_step(xs, ys, st, row);
  return h;
}

}  // namespace sdb
