// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) and the Box-Muller transform of the
// sketch stream: key = (lo32(seed), stream id), counter = (lo32(e/2), hi32(e/2), replica,
// hi32(seed)); two 53-bit uniforms u = ((w0 >> 5) 2^26 + (w1 >> 6) + 1/2) 2^-53 per call,
// and element e takes z_{e mod 2} of z0 = sqrt(-2 ln u1) cos(2 pi u2),
// z1 = sqrt(-2 ln u1) sin(2 pi u2).  Shared by the stored sketches and the operand packer
// that generates a sketch in place, so both give the same values.
#pragma once

#include <stdint.h>

namespace tatrg {

__device__ __forceinline__ void philox_round(uint32_t& c0, uint32_t& c1, uint32_t& c2,
                                             uint32_t& c3, uint32_t k0, uint32_t k1) {
  const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
  uint32_t hi0 = __umulhi(m0, c0), lo0 = m0 * c0;
  uint32_t hi1 = __umulhi(m1, c2), lo1 = m1 * c2;
  uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
  c0 = n0;
  c1 = lo1;
  c2 = n2;
  c3 = lo0;
}

// the four 32-bit words of counter block p
__device__ __forceinline__ void philox4x32_10(uint64_t seed, uint32_t sid, uint32_t replica,
                                              int64_t p, uint32_t (&w)[4]) {
  uint32_t c0 = uint32_t(p), c1 = uint32_t(uint64_t(p) >> 32), c2 = replica, c3 = uint32_t(seed >> 32);
  uint32_t k0 = uint32_t(seed), k1 = sid;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    philox_round(c0, c1, c2, c3, k0, k1);
  }
  w[0] = c0;
  w[1] = c1;
  w[2] = c2;
  w[3] = c3;
}

__device__ __forceinline__ double u53(uint32_t a, uint32_t b) {
  return (double(a >> 5) * 67108864.0 + double(b >> 6) + 0.5) * (1.0 / 9007199254740992.0);
}

// The pair (z0, z1) of counter block p with Box-Muller evaluated in float arithmetic
// (relative error ~1e-7): for sketches that feed split-precision contractions, whose
// operands are rounded to two tensor-core numbers (~2^-22 relative) anyway.  The uniforms
// are the 53-bit values rounded to float (never zero: the smallest is 2^-54).
__device__ __forceinline__ void gauss_pair_f32(uint64_t seed, uint32_t sid, uint32_t replica,
                                               int64_t p, float& z0, float& z1) {
  uint32_t w[4];
  philox4x32_10(seed, sid, replica, p, w);
  const float u1 = float(u53(w[0], w[1])), u2 = float(u53(w[2], w[3]));
  const float rad = sqrtf(-2.0f * logf(u1));
  float sn, cs;
  sincospif(2.0f * u2, &sn, &cs);  // angle 2 pi u2, reduced exactly in units of pi
  z0 = rad * cs;
  z1 = rad * sn;
}

}  // namespace tatrg
