// prims.cuh -- device-wide primitives: exclusive scan, order-preserving
// compaction, and a stable LSD radix sort (8-bit digits, shared-memory local
// ranking, coalesced scatter).  Written for the pass's own buffers; sizes are
// passed from the host.
#pragma once
#include "common.cuh"

namespace cbp {

constexpr int SCAN_T = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_T * SCAN_ITEMS;

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Block-wide exclusive scan of one value per thread (blockDim.x == SCAN_T).
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T* total) {
  __shared__ T warp_tot[SCAN_T / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T inc = warp_incl_scan(v);
  if (lane == 31) warp_tot[w] = inc;
  __syncthreads();
  if (w == 0) {
    T t = (lane < SCAN_T / 32) ? warp_tot[lane] : T(0);
    T ti = warp_incl_scan(t);
    if (lane < SCAN_T / 32) warp_tot[lane] = ti - t;
    if (lane == SCAN_T / 32 - 1) *total = ti;
  }
  __syncthreads();
  T r = warp_tot[w] + inc - v;
  __syncthreads();
  return r;
}

template <typename TIn, typename TOut>
__global__ void k_scan_reduce(const TIn* in, int64_t n, TOut* block_sums) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  TOut s = 0;
#pragma unroll
  for (int r = 0; r < SCAN_ITEMS; ++r) {
    int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + r;
    if (i < n) s += (TOut)in[i];
  }
  __shared__ TOut tot;
  block_excl_scan<TOut>(s, &tot);
  if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

// single block: exclusive scan of block sums in place; writes the grand total
template <typename TOut>
__global__ void k_scan_block_sums(TOut* sums, int64_t nb, TOut* total) {
  __shared__ TOut carry_s;
  __shared__ TOut tot;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  for (int64_t base = 0; base < nb; base += SCAN_T) {
    int64_t i = base + threadIdx.x;
    TOut v = (i < nb) ? sums[i] : TOut(0);
    TOut ex = block_excl_scan<TOut>(v, &tot);
    TOut carry = carry_s;
    if (i < nb) sums[i] = ex + carry;
    __syncthreads();
    if (threadIdx.x == 0) carry_s = carry + tot;
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = carry_s;
}

template <typename TIn, typename TOut>
__global__ void k_scan_apply(const TIn* in, int64_t n, const TOut* block_sums, TOut* out) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  TOut v[SCAN_ITEMS];
  TOut s = 0;
#pragma unroll
  for (int r = 0; r < SCAN_ITEMS; ++r) {
    int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + r;
    v[r] = (i < n) ? (TOut)in[i] : TOut(0);
    s += v[r];
  }
  __shared__ TOut tot;
  TOut ex = block_excl_scan<TOut>(s, &tot) + block_sums[blockIdx.x];
#pragma unroll
  for (int r = 0; r < SCAN_ITEMS; ++r) {
    int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + r;
    if (i < n) out[i] = ex;
    ex += v[r];
  }
}

// Small inputs: one block walks the tiles in order with a running carry (one
// launch instead of three; the tiles are few, so the serial walk is short).
template <typename TIn, typename TOut>
__global__ void __launch_bounds__(SCAN_T) k_scan_single(const TIn* in, int64_t n, TOut* out, TOut* total) {
  __shared__ TOut tot;
  TOut carry = 0;
  for (int64_t base = 0; base < n; base += SCAN_TILE) {
    TOut v[SCAN_ITEMS];
    TOut s = 0;
#pragma unroll
    for (int r = 0; r < SCAN_ITEMS; ++r) {
      const int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + r;
      v[r] = (i < n) ? (TOut)in[i] : TOut(0);
      s += v[r];
    }
    TOut ex = block_excl_scan<TOut>(s, &tot) + carry;
#pragma unroll
    for (int r = 0; r < SCAN_ITEMS; ++r) {
      const int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + r;
      if (i < n) out[i] = ex;
      ex += v[r];
    }
    carry += tot;  // tot is final: block_excl_scan ends with a barrier
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

// Inputs of at most this many tiles take the single-block scan.
constexpr int64_t SCAN_SINGLE_TILES = 8;

// Exclusive scan out[i] = sum_{k<i} in[k]; *total_dev = sum of all (device).
// tmp must hold scan_tmp_elems(n) elements of TOut.  in and out may alias.
inline int64_t scan_tmp_elems(int64_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE + 1; }

template <typename TIn, typename TOut>
void exclusive_scan(const TIn* in, TOut* out, int64_t n, TOut* tmp, TOut* total_dev, cudaStream_t st) {
  int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (nb < 1) nb = 1;
  if (nb <= SCAN_SINGLE_TILES) {
    k_scan_single<TIn, TOut><<<1, SCAN_T, 0, cb_count(st)>>>(in, n, out, total_dev);
    return;
  }
  k_scan_reduce<TIn, TOut><<<(int)nb, SCAN_T, 0, cb_count(st)>>>(in, n, tmp);
  k_scan_block_sums<TOut><<<1, SCAN_T, 0, cb_count(st)>>>(tmp, nb, total_dev);
  k_scan_apply<TIn, TOut><<<(int)nb, SCAN_T, 0, cb_count(st)>>>(in, n, tmp, out);
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort, 8-bit digit per pass.
// ---------------------------------------------------------------------------
constexpr int RS_T = 256;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_T * RS_ITEMS;
constexpr int RS_WARPS = RS_T / 32;

template <typename K>
__global__ void k_radix_hist(const K* __restrict__ keys, int64_t n, int shift, uint32_t* hist, int nblocks) {
  __shared__ uint32_t sh[256];
  sh[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll
  for (int r = 0; r < RS_ITEMS; ++r) {
    int64_t i = base + (int64_t)r * RS_T + threadIdx.x;
    if (i < n) atomicAdd(&sh[(uint32_t)(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = sh[threadIdx.x];
}

// Scatter of one digit pass.  offs holds the global start of (digit, block)
// at [digit * nblocks + block]; with FOLD the kernel reads the per-block
// histograms instead (hist[digit * nblocks + block]) and forms its own starts
// (few blocks: each thread sums one digit's row), which saves the scan.
template <typename K, typename V, bool HAS_V, bool FOLD = false>
__global__ void __launch_bounds__(RS_T) k_radix_scatter(const K* __restrict__ kin, const V* __restrict__ vin,
                                                        K* __restrict__ kout, V* __restrict__ vout, int64_t n,
                                                        int shift, const uint32_t* __restrict__ offs, int nblocks) {
  __shared__ uint32_t gstart[FOLD ? 256 : 1];
  if constexpr (FOLD) {
    const uint32_t* row = offs + (int64_t)threadIdx.x * nblocks;
    uint32_t before = 0, all = 0;
    for (int b = 0; b < nblocks; ++b) {
      const uint32_t c = row[b];
      before += b < (int)blockIdx.x ? c : 0u;
      all += c;
    }
    __shared__ uint32_t tot_f;
    gstart[threadIdx.x] = block_excl_scan<uint32_t>(all, &tot_f) + before;
  }
  __shared__ K sk[RS_TILE];
  __shared__ V sv[HAS_V ? RS_TILE : 1];
  __shared__ uint32_t wcnt[RS_WARPS][256];
  __shared__ uint32_t woff[RS_WARPS][256];
  __shared__ uint32_t run[256];
  __shared__ uint32_t dstart[256];
  __shared__ uint32_t tot_dummy;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int q = 0; q < RS_WARPS; ++q) wcnt[q][tid] = 0;
  run[tid] = 0;
  K key[RS_ITEMS];
  V val[RS_ITEMS];
  uint32_t dig[RS_ITEMS], rank[RS_ITEMS];
#pragma unroll
  for (int r = 0; r < RS_ITEMS; ++r) {
    int64_t i = base + (int64_t)r * RS_T + tid;
    bool ok = i < n;
    key[r] = ok ? kin[i] : K(0);
    if (HAS_V) val[r] = ok ? vin[i] : V(0);
    dig[r] = ok ? ((uint32_t)(key[r] >> shift) & 255u) : 256u;
  }
  __syncthreads();
  const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < RS_ITEMS; ++r) {
    uint32_t peers = __match_any_sync(0xffffffffu, dig[r]);
    uint32_t rw = __popc(peers & lt);
    if (rw == 0 && dig[r] < 256u) wcnt[w][dig[r]] = __popc(peers);
    __syncthreads();
    {
      uint32_t s = run[tid];
#pragma unroll
      for (int q = 0; q < RS_WARPS; ++q) {
        uint32_t c = wcnt[q][tid];
        wcnt[q][tid] = 0;
        woff[q][tid] = s;
        s += c;
      }
      run[tid] = s;
    }
    __syncthreads();
    rank[r] = (dig[r] < 256u) ? woff[w][dig[r]] + rw : 0u;
  }
  // tile-local start of each digit
  uint32_t ex = block_excl_scan<uint32_t>(run[tid], &tot_dummy);
  dstart[tid] = ex;
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RS_ITEMS; ++r) {
    if (dig[r] < 256u) {
      uint32_t lp = dstart[dig[r]] + rank[r];
      sk[lp] = key[r];
      if (HAS_V) sv[lp] = val[r];
    }
  }
  __syncthreads();
  const int64_t cnt = (n - base) < RS_TILE ? (n - base) : RS_TILE;
  for (int i = tid; i < cnt; i += RS_T) {
    K k = sk[i];
    uint32_t d = (uint32_t)(k >> shift) & 255u;
    const int64_t g0 = FOLD ? (int64_t)gstart[d] : (int64_t)offs[(int64_t)d * nblocks + blockIdx.x];
    int64_t pos = g0 + (i - dstart[d]);
    kout[pos] = k;
    if (HAS_V) vout[pos] = sv[i];
  }
}

inline int64_t radix_hist_elems(int64_t n) { return 256 * ((n + RS_TILE - 1) / RS_TILE + 1); }

// Sorts of at most this many tiles form the digit starts inside the scatter.
constexpr int RS_FOLD_BLOCKS = 32;

// Sort keys (and values) on bits [lo_bit, hi_bit).  Buffers ping-pong between
// (k0, v0) and (k1, v1); returns 0 if the result is in k0/v0, 1 if in k1/v1.
// hist: radix_hist_elems(n) uint32; scan_tmp: scan_tmp_elems(hist elems) uint32.
// need: the key bits that may be set; a digit with none of them is the same
// (zero) in every key, so its pass would not move anything and is skipped.
template <typename K, typename V, bool HAS_V>
int radix_sort(K* k0, V* v0, K* k1, V* v1, int64_t n, int lo_bit, int hi_bit, uint32_t* hist,
               uint32_t* scan_tmp, cudaStream_t st, uint64_t need = ~0ull) {
  if (n <= 1) return 0;
  int nb = (int)((n + RS_TILE - 1) / RS_TILE);
  int cur = 0;
  for (int sh = lo_bit; sh < hi_bit; sh += 8) {
    if (((need >> sh) & 0xffull) == 0) continue;
    const K* ki = cur ? k1 : k0;
    const V* vi = cur ? v1 : v0;
    K* ko = cur ? k0 : k1;
    V* vo = cur ? v0 : v1;
    k_radix_hist<K><<<nb, RS_T, 0, cb_count(st)>>>(ki, n, sh, hist, nb);
    if (nb <= RS_FOLD_BLOCKS) {
      k_radix_scatter<K, V, HAS_V, true><<<nb, RS_T, 0, cb_count(st)>>>(ki, vi, ko, vo, n, sh, hist, nb);
    } else {
      exclusive_scan<uint32_t, uint32_t>(hist, hist, (int64_t)256 * nb, scan_tmp, (uint32_t*)nullptr, st);
      k_radix_scatter<K, V, HAS_V><<<nb, RS_T, 0, cb_count(st)>>>(ki, vi, ko, vo, n, sh, hist, nb);
    }
    cur ^= 1;
  }
  return cur;
}

// ---------------------------------------------------------------------------
// order-preserving compaction helpers
// ---------------------------------------------------------------------------
template <typename T, typename F>
__global__ void k_compact(const T* __restrict__ in, const F* __restrict__ flags, const uint32_t* __restrict__ pos,
                          int64_t n, T* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && flags[i]) out[pos[i]] = in[i];
}

}  // namespace cbp
