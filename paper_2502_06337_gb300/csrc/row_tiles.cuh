// Row-pair difference tiles shared by the curve vote's row bands and the eps-band vote.
//
// A band of rows [R0, R1) of the G x G accumulator is held in shared memory as (R1 - R0)/2 row
// pairs of RS >= G 32-bit words: word (i, j) carries rows R0 + 2i (low 16 bits) and R0 + 2i + 1
// (high 16 bits) at column j; words j >= G of a pair are padding (RS a multiple of 4). A run of
// cells [a, b] of one row is entered as a difference: +inc at column a and -inc (modulo 2^32)
// at column b + 1 (in the padding when b = G - 1, if RS > G), inc = 1 for the pair's first row
// and 2^16 for its second. Prefix sums along each row pair then turn the differences into
// counts.
//
// The words are summed modulo 2^32. The prefix sum at any column equals c_lo + 2^16 c_hi for the
// two rows' true counts there, and every count of a slice is at most its 65535 circles, so
// that sum lies below 2^32 and splits into the exact pair of 16-bit counts.
#pragma once

#include <stdint.h>

namespace sprot {

// Turns the tile's differences into counts (one warp per row pair) and writes the band's rows
// into a slice's partial accumulator out_slice (G rows x G/2 words, columns 2k and 2k + 1 of a
// row in word k). Every thread of the block must call it; the tile is rewritten in place.
__device__ __forceinline__ void flush_row_pair_tile(uint32_t* tile, int G, int RS, int R0, int R1,
                                                    uint32_t* out_slice) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int W2 = G >> 1;
  for (int rp = warp; rp < ((R1 - R0) >> 1); rp += nwarps) {
    uint32_t* row = tile + rp * RS;
    uint32_t carry = 0;
    for (int c0 = 0; c0 < G; c0 += 32) {
      const int c = c0 + lane;
      uint32_t v = c < G ? row[c] : 0u;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
      }
      v += carry;
      if (c < G) row[c] = v;
      carry = __shfl_sync(0xffffffffu, v, 31);
    }
  }
  __syncthreads();
  uint4* out4 = reinterpret_cast<uint4*>(out_slice);
  for (int g = threadIdx.x; g < (((R1 - R0) * W2) >> 2); g += blockDim.x) {
    const int rr = (4 * g) / W2, c2 = 4 * g - rr * W2;
    const uint4* rw = reinterpret_cast<const uint4*>(tile + (rr >> 1) * RS + 2 * c2);
    const uint4 ra = rw[0], rb = rw[1];
    const int sh = (rr & 1) ? 16 : 0;
    auto pk = [sh](uint32_t x, uint32_t y) { return ((x >> sh) & 0xffffu) | (((y >> sh) & 0xffffu) << 16); };
    out4[((R0 + rr) * W2 + c2) >> 2] = make_uint4(pk(ra.x, ra.y), pk(ra.z, ra.w), pk(rb.x, rb.y), pk(rb.z, rb.w));
  }
}

}  // namespace sprot
