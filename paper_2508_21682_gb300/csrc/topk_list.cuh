// Per-point top-k list kept in registers, shared by the window and Gram
// kernels.
#pragma once

#include <math.h>
#include <stdint.h>

// (distance, index) order: distance first, then index (as unsigned).
__device__ __forceinline__ bool lessp(float da, uint32_t ia, float db, uint32_t ib) {
  return da < db || (da == db && ia < ib);
}

// A point's list in registers: KP slots, ascending by (distance, index).
// The graph keeps the top KP >= k per point (KP = 16, 32 or 64) so that every
// slot index is a compile-time constant and the list stays in registers; the
// top k of the top KP is the top k, so the caller keeps the first k columns.
template <int KP>
struct ListK {
  float d[KP];
  uint32_t i[KP];

  // gd, gi: the point's KP slots (16-byte aligned: KP is a multiple of 4)
  __device__ __forceinline__ void load(const float* gd, const uint32_t* gi) {
#pragma unroll
    for (int j = 0; j < KP; j += 4) {
      const float4 a = *reinterpret_cast<const float4*>(gd + j);
      const uint4 b = *reinterpret_cast<const uint4*>(gi + j);
      d[j] = a.x;
      d[j + 1] = a.y;
      d[j + 2] = a.z;
      d[j + 3] = a.w;
      i[j] = b.x;
      i[j + 1] = b.y;
      i[j + 2] = b.z;
      i[j + 3] = b.w;
    }
  }
  __device__ __forceinline__ void store(float* gd, uint32_t* gi) const {
#pragma unroll
    for (int j = 0; j < KP; j += 4) {
      *reinterpret_cast<float4*>(gd + j) = make_float4(d[j], d[j + 1], d[j + 2], d[j + 3]);
      *reinterpret_cast<uint4*>(gi + j) = make_uint4(i[j], i[j + 1], i[j + 2], i[j + 3]);
    }
  }
  // Every slot empty: (+inf, 0xffffffff).
  __device__ __forceinline__ void clear() {
#pragma unroll
    for (int j = 0; j < KP; ++j) {
      d[j] = INFINITY;
      i[j] = 0xffffffffu;
    }
  }
  // Inserts (cd, ci) unless it is no better than the last slot or listed.
  __device__ __forceinline__ void offer(float cd, uint32_t ci) {
    if (!lessp(cd, ci, d[KP - 1], i[KP - 1])) return;
    // a listed candidate (the common case once lists have settled: the same
    // neighbour comes back in later trees) leaves before the insertion work
    uint32_t dupm[KP];
#pragma unroll
    for (int j = 0; j < KP; ++j) dupm[j] = i[j] == ci ? 1u : 0u;
#pragma unroll
    for (int w = 1; w < KP; w <<= 1)
#pragma unroll
      for (int j = 0; j + w < KP; j += 2 * w) dupm[j] |= dupm[j + w];
    if (dupm[0]) return;
    // insert position: the number of entries below the candidate (balanced
    // tree of bits: short dependency chains)
    uint32_t lowm[KP];
#pragma unroll
    for (int j = 0; j < KP; ++j) lowm[j] = lessp(d[j], i[j], cd, ci) ? 1u : 0u;
#pragma unroll
    for (int w = 1; w < KP; w <<= 1)
#pragma unroll
      for (int j = 0; j + w < KP; j += 2 * w) lowm[j] += lowm[j + w];
    // entries below the candidate form a prefix; each slot then takes its new
    // value from the old list independently
    const uint32_t below = lowm[0];
#pragma unroll
    for (int j = KP - 1; j >= 0; --j) {
      const bool shift = (uint32_t)j > below;
      const bool here = (uint32_t)j == below;
      const float pd = j > 0 ? d[j - 1] : cd;
      const uint32_t pi = j > 0 ? i[j - 1] : ci;
      d[j] = shift ? pd : (here ? cd : d[j]);
      i[j] = shift ? pi : (here ? ci : i[j]);
    }
  }
};
