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
// lane l at [w * 32 + l], so a warp's 32 lookups never conflict (8 KB).
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

// id of cell (cx, cy) at the level the parameters were made for (cx, cy < 2^F)
__device__ __forceinline__ uint64_t hilbert3_encode(uint32_t cx, uint32_t cy, uint32_t nsteps,
                                                    uint32_t st0, const uint32_t* tab) {
  const uint32_t lane = threadIdx.x & 31u;
  uint64_t h = 0;
  uint32_t st = st0;
  for (int s = (int)nsteps - 1; s >= 0; --s) {
    const uint32_t idx = (st << 6) | (((cx >> (3 * s)) & 7u) << 3) | ((cy >> (3 * s)) & 7u);
    const uint32_t e = (tab[(idx >> 2) * 32 + lane] >> (8 * (idx & 3u))) & 255u;
    h = (h << 6) | (e & 63u);
    st = e >> 6;
  }
  return h;
}

}  // namespace sdb
