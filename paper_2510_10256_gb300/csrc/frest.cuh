// frest.cuh -- filter membership (Sec. 3.2).  Shells: a candidate is
// filtered iff its stencil is in the rest-filter table built at scene
// creation.  Rods: through the per-edge arc-length windows (below).
#pragma once
#include <cstdint>

#include "common.cuh"

// The table's keys are also held in an open-addressing hash set (built with
// the row offsets, at most half full; an empty slot holds FREST_EMPTY, which
// no key equals: its type bits would be 3), probed linearly from a mixed
// hash of the key -- one or two dependent loads per lookup instead of a
// binary search's chain.  The mixer is the SplitMix64 finalizer (Vigna).
constexpr uint64_t FREST_EMPTY = ~0ull;

__host__ __device__ __forceinline__ uint64_t frest_hash(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ bool frest_contains(const uint64_t* __restrict__ tab, uint64_t mask, uint64_t key) {
  uint64_t h = frest_hash(key) & mask;
  for (uint64_t probe = 0; probe <= mask; ++probe) {
    const uint64_t v = tab[h];
    if (v == key) return true;
    if (v == FREST_EMPTY) return false;
    h = (h + 1) & mask;
  }
  return false;
}

// Rods: edges ki < kj of one polyline are filtered when kj is within the
// forward window of ki (kj <= win[ki]) or, on a closed loop, within its
// backward window (kj >= wst[ki] >= 0: the gap the other way round is below
// the activation).  loops: the member has closed loops (else wst is not read).
__device__ __forceinline__ bool rod_filtered(const int32_t* __restrict__ win, const int32_t* __restrict__ wst,
                                             bool loops, uint32_t ki, uint32_t kj) {
  if ((int)kj <= win[ki]) return true;
  if (!loops) return false;
  const int w = wst[ki];
  return w >= 0 && (int)kj >= w;
}

// Rods: the index gap of edges ki < kj of one polyline (Kaldor culling);
// on a closed loop of m edges the shorter way round
__device__ __forceinline__ int rod_gap(const int32_t* __restrict__ rloop, uint32_t ki, uint32_t kj) {
  const int g = (int)(kj - ki), m = rloop[ki];
  return m > 0 ? min(g, m - g) : g;
}
