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

  __device__ __forceinline__ void load(const float* gd, const uint32_t* gi) {
#pragma unroll
    for (int j = 0; j < KP; ++j) {
      d[j] = gd[j];
      i[j] = gi[j];
    }
  }
  __device__ __forceinline__ void store(float* gd, uint32_t* gi) const {
#pragma unroll
    for (int j = 0; j < KP; ++j) {
      gd[j] = d[j];
      gi[j] = i[j];
    }
  }
  // Inserts (cd, ci) unless it is no better than the last slot or listed.
  __device__ __forceinline__ void offer(float cd, uint32_t ci) {
    if (!lessp(cd, ci, d[KP - 1], i[KP - 1])) return;
    bool dup = false;
#pragma unroll
    for (int j = 0; j < KP; ++j) dup |= (i[j] == ci);
    if (dup) return;
    // position = number of entries below the candidate (they form a prefix);
    // every slot then takes its new value from the old list independently
    uint32_t below = 0;
#pragma unroll
    for (int j = 0; j < KP; ++j) below += lessp(d[j], i[j], cd, ci) ? 1u : 0u;
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
