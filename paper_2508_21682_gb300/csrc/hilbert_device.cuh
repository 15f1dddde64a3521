// Device-side Hilbert key helpers (Skilling's transposed index), shared by the
// key, sort fix-up and search kernels.
//
// Paper, Section 2: points are ordered along a Hilbert curve; the curve itself
// is not specified there, and this library uses Skilling's transposed-index
// construction (AIP Conf. Proc. 707, 2004) as its convention.
//
// A point's permuted, reflected coordinates Y[0..d) (each `L` bits wide) live
// in a caller-provided byte array (shared or local memory); the transform runs
// in place. The top L bit levels of a b-bit key equal the L-bit key of the
// coordinates' top L bits: the level-q step of the transform changes only bits
// below q, and the final correction word t is built the same way, so a key
// prefix that covers only the top L levels needs only those bits.
#pragma once

#include <stdint.h>

// Bit (c & 31) of word c >> 5 of plane `lvl` of point `p`.
__device__ __forceinline__ uint32_t hf_plane_bit(const uint32_t* __restrict__ planes, int64_t n,
                                                 int W32, int lvl, int64_t p, int c) {
  return (__ldg(planes + ((size_t)lvl * n + p) * W32 + (c >> 5)) >> (c & 31)) & 1u;
}

// Y[i] = top `L` bits of code[pi[i]] of point p, reflected when bit i of the
// tree's reflection mask is set.
__device__ __forceinline__ void hf_load_coords_planes(const uint32_t* __restrict__ planes,
                                                      int64_t n, int d, int W32, int L,
                                                      const int32_t* __restrict__ pi,
                                                      const uint32_t* __restrict__ rbits,
                                                      int64_t p, uint8_t* Y) {
  const uint32_t full = (1u << L) - 1u;
  for (int i = 0; i < d; ++i) {
    const int c = pi ? pi[i] : i;
    uint32_t v = 0;
    for (int l = 0; l < L; ++l) v = (v << 1) | hf_plane_bit(planes, n, W32, l, p, c);
    if (rbits && ((rbits[i >> 5] >> (i & 31)) & 1u)) v ^= full;
    Y[i] = (uint8_t)v;
  }
}

// Same from byte codes (bits wide), keeping the top L bits.
__device__ __forceinline__ void hf_load_coords_codes(const uint8_t* __restrict__ codes, int d,
                                                     int bits, int L,
                                                     const int32_t* __restrict__ pi,
                                                     const uint32_t* __restrict__ rbits,
                                                     uint8_t* Y) {
  const uint32_t full = (1u << L) - 1u;
  for (int i = 0; i < d; ++i) {
    const int c = pi ? pi[i] : i;
    uint32_t v = (uint32_t)codes[c] >> (bits - L);
    if (rbits && ((rbits[i >> 5] >> (i & 31)) & 1u)) v ^= full;
    Y[i] = (uint8_t)v;
  }
}

// Skilling's axes-to-transpose map on Y[0..d), L bits per coordinate.
__device__ __forceinline__ void hf_skilling(uint8_t* Y, int d, int L) {
  uint32_t x0 = Y[0];
  for (int q = L - 1; q >= 1; --q) {
    const uint32_t P = (1u << q) - 1u;
    // i = 0: inverts X[0] when its bit q is set; the exchange with itself is a no-op
    if ((x0 >> q) & 1u) x0 ^= P;
    for (int i = 1; i < d; ++i) {
      const uint32_t xi = Y[i];
      if ((xi >> q) & 1u) {
        x0 ^= P;
      } else {
        const uint32_t t = (x0 ^ xi) & P;
        x0 ^= t;
        Y[i] = (uint8_t)(xi ^ t);
      }
    }
  }
  Y[0] = (uint8_t)x0;
  uint32_t prev = x0;
  for (int i = 1; i < d; ++i) {
    prev ^= Y[i];
    Y[i] = (uint8_t)prev;
  }
  uint32_t t = 0;
  for (int q = L - 1; q >= 1; --q)
    if ((prev >> q) & 1u) t ^= (1u << q) - 1u;
  if (t)
    for (int i = 0; i < d; ++i) Y[i] ^= (uint8_t)t;
}

// Key word `wi` of the transformed Y (L levels): bit g = 64*wi + j of the key
// (from the top) is bit (L-1-g/d) of Y[g % d]; bits at or beyond d*L are 0.
__device__ __forceinline__ uint64_t hf_pack_word(const uint8_t* Y, int d, int L, int wi) {
  uint64_t v = 0;
  const int64_t total = (int64_t)d * L;
  int64_t g = (int64_t)wi * 64;
  int l = (int)(g / d);
  int i = (int)(g - (int64_t)l * d);
  for (int j = 0; j < 64; ++j, ++g) {
    uint64_t bit = 0;
    if (g < total) {
      bit = (Y[i] >> (L - 1 - l)) & 1u;
      if (++i == d) {
        i = 0;
        ++l;
      }
    }
    v = (v << 1) | bit;
  }
  return v;
}
