// spmv.cu -- y = (H + shift I) v for the scene's BSR Hessian (the product a
// Newton driver's conjugate-gradient solve needs; the paper minimises with
// projected Newton, App. A).  One thread per block row: the row's 3x3 blocks
// times the three components of v at their columns; vectors are [3][n] SoA.
#include "scene.cuh"

namespace {

__global__ void k_bsr_spmv(int n, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                           const double* __restrict__ val, const double* __restrict__ v, double shift,
                           double* __restrict__ y) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double y0 = shift * v[r], y1 = shift * v[(size_t)n + r], y2 = shift * v[2 * (size_t)n + r];
  for (int k = row_ptr[r]; k < row_ptr[r + 1]; ++k) {
    const int c = col[k];
    const double* b = val + 9 * (size_t)k;
    const double v0 = v[c], v1 = v[(size_t)n + c], v2 = v[2 * (size_t)n + c];
    y0 += b[0] * v0 + b[1] * v1 + b[2] * v2;
    y1 += b[3] * v0 + b[4] * v1 + b[5] * v2;
    y2 += b[6] * v0 + b[7] * v1 + b[8] * v2;
  }
  y[r] = y0;
  y[(size_t)n + r] = y1;
  y[2 * (size_t)n + r] = y2;
}

}  // namespace

extern "C" cb_status cb_bsr_spmv(cb_scene* s, const double* v, double* y, double shift, void* stream) {
  if (!s || !v || !y || v == y) return CB_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  s->last_stream = st;
  if (s->n == 0) return CB_OK;
  if (!s->bsr_row.p) return CB_ERR_ARG;  // no barrier_eval / barrier_energy yet
  // an empty matrix (no active pair) still has row_ptr: zeros
  k_bsr_spmv<<<cb_grid(s->n), CB_THREADS, 0, cb_count(st)>>>(s->n, (const int32_t*)s->bsr_row.p,
                                                              (const int32_t*)s->bsr_col.p,
                                                              (const double*)s->bsr_val.p, v, shift, y);
  CB_CUDA(cudaGetLastError());
  return CB_OK;
}
