// common.cuh -- shared device/host helpers of the contact library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "../../include/contact.h"

#define CB_THREADS 256

// Pair keys: bits 63..62 type, 61..31 first index, 30..0 second index.
#define CB_KEY_ROD_EE 0u
#define CB_KEY_PT 1u
#define CB_KEY_EE 2u

__host__ __device__ __forceinline__ uint64_t cb_key(uint32_t type, uint32_t i, uint32_t j) {
  return ((uint64_t)type << 62) | ((uint64_t)i << 31) | (uint64_t)j;
}
__host__ __device__ __forceinline__ uint32_t cb_key_type(uint64_t k) { return (uint32_t)(k >> 62); }
__host__ __device__ __forceinline__ uint32_t cb_key_i(uint64_t k) { return (uint32_t)((k >> 31) & 0x7FFFFFFFu); }
__host__ __device__ __forceinline__ uint32_t cb_key_j(uint64_t k) { return (uint32_t)(k & 0x7FFFFFFFu); }

// Device status bits (OR-ed into the scene's status word by kernels).
#define CB_DEV_CAPACITY 1u
#define CB_DEV_PENETRATION 2u
#define CB_DEV_ITER_LIMIT 4u

// FP64 arithmetic (x = exact-rounding helpers) with the rounding written in the source: no contraction into
// fused multiply-adds, so predicates decided here are reproducible bit for bit
// by any IEEE-754 implementation evaluating the same expression.
__device__ __forceinline__ double xmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double xadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double xsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double xdiv(double a, double b) { return __ddiv_rn(a, b); }

struct d3 {
  double x, y, z;
};
__device__ __forceinline__ d3 mk3(double x, double y, double z) { return d3{x, y, z}; }
__device__ __forceinline__ d3 sub3(d3 a, d3 b) { return d3{xsub(a.x, b.x), xsub(a.y, b.y), xsub(a.z, b.z)}; }
__device__ __forceinline__ double dot3(d3 a, d3 b) { return xadd(xadd(xmul(a.x, b.x), xmul(a.y, b.y)), xmul(a.z, b.z)); }
__device__ __forceinline__ d3 cross3(d3 a, d3 b) {
  return d3{xsub(xmul(a.y, b.z), xmul(a.z, b.y)), xsub(xmul(a.z, b.x), xmul(a.x, b.z)),
            xsub(xmul(a.x, b.y), xmul(a.y, b.x))};
}

// Process-wide count of kernels this library has launched: every launch passes
// its stream through cb_count().
long long cb_launch_counter_add();
static inline cudaStream_t cb_count(cudaStream_t st) {
  cb_launch_counter_add();
  return st;
}

static inline int cb_grid(int64_t n, int per_block = CB_THREADS) {
  int64_t g = (n + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > 2147483647LL) g = 2147483647LL;
  return (int)g;
}

#define CB_CUDA(call)                                                  \
  do {                                                                 \
    cudaError_t e_ = (call);                                           \
    if (e_ != cudaSuccess) {                                           \
      fprintf(stderr, "contact: CUDA error %s at %s:%d\n",             \
              cudaGetErrorString(e_), __FILE__, __LINE__);             \
      return CB_ERR_CUDA;                                              \
    }                                                                  \
  } while (0)

#define CB_TRY(call)                 \
  do {                               \
    cb_status s_ = (call);           \
    if (s_ != CB_OK) return s_;      \
  } while (0)
