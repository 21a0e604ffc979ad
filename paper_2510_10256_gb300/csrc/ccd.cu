// ccd.cu -- stage (e): conservative step bound for the line search (Sec. 3.3).
//
// Candidates: pairs whose swept boxes (x and x + p) inflated by xi/2 overlap.
// Class of a pair at x: F if filtered (Sec. 3.2), C if unfiltered and already
// within the offset (Sec. 3.4), U otherwise.  Offset: U -> xi (0 in the
// single-phase mode), F and C -> 0 (the filtered pairs are single-phase, Eq. 4).
// Each pair is bounded by additive CCD (C-IPC): in the pair's local frame with
// the mean displacement removed, l_p bounds the relative speed of the closest
// points; the first step (1-s) g0 / l_p and every later step c (d - offset)/l_p
// cannot close the gap, and the iteration stops before the gap would drop
// below s g0.  alpha = min(1, min_p t_p).
#include <cmath>

#include "geometry.cuh"
#include "prims.cuh"
#include "scene.cuh"

namespace {

constexpr double ACCD_S = 0.1;
constexpr double ACCD_C = 0.9;
constexpr int ACCD_MAX_ITER = 10000;

struct CcdArgs {
  int64_t np;
  const uint64_t* __restrict__ keys;
  const int32_t* __restrict__ ev0;
  const int32_t* __restrict__ ev1;
  const int32_t* __restrict__ tv;
  const int32_t* __restrict__ comp;
  const int32_t* __restrict__ win;
  const uint64_t* __restrict__ frest;
  int64_t nf;
  int T, n, kind;
  int filter_off, single, core_temp;
  double xi;
  const double* __restrict__ x;
  const double* __restrict__ p;
  double* __restrict__ t_out;
  uint8_t* __restrict__ cls_out;
  unsigned long long* __restrict__ alpha_bits;
  unsigned long long* __restrict__ status;
  unsigned long long* __restrict__ max_iters;
};

__device__ __forceinline__ d3 ld(const double* __restrict__ a, int n, int v) {
  return mk3(a[v], a[(size_t)n + v], a[2 * (size_t)n + v]);
}
__device__ __forceinline__ double norm3(d3 a) { return __dsqrt_rn(dot3(a, a)); }
__device__ __forceinline__ d3 axpy3(d3 x, double t, d3 p) {
  return mk3(xadd(x.x, xmul(t, p.x)), xadd(x.y, xmul(t, p.y)), xadd(x.z, xmul(t, p.z)));
}

__global__ void __launch_bounds__(128) k_accd(CcdArgs A) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= A.np) return;
  const uint64_t key = A.keys[q];
  const uint32_t ty = cb_key_type(key), ki = cb_key_i(key), kj = cb_key_j(key);
  int v[4];
  bool ee;
  if (ty == CB_KEY_PT) {
    v[0] = (int)ki;
    v[1] = A.tv[kj];
    v[2] = A.tv[A.T + kj];
    v[3] = A.tv[2 * A.T + kj];
    ee = false;
  } else {
    v[0] = A.ev0[ki];
    v[1] = A.ev1[ki];
    v[2] = A.ev0[kj];
    v[3] = A.ev1[kj];
    ee = true;
  }
  // class at x
  bool filt = false;
  if (!A.filter_off) {
    if (A.kind == CB_ROD) {
      filt = A.comp[A.ev0[ki]] == A.comp[A.ev0[kj]] && (int)kj <= A.win[ki];
    } else if (A.nf > 0) {
      int64_t lo = 0, hi = A.nf;
      while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (A.frest[mid] < key) lo = mid + 1;
        else hi = mid;
      }
      filt = lo < A.nf && A.frest[lo] == key;
    }
  }
  d3 X0 = ld(A.x, A.n, v[0]), X1 = ld(A.x, A.n, v[1]), X2 = ld(A.x, A.n, v[2]), X3 = ld(A.x, A.n, v[3]);
  d3 P0 = ld(A.p, A.n, v[0]), P1 = ld(A.p, A.n, v[1]), P2 = ld(A.p, A.n, v[2]), P3 = ld(A.p, A.n, v[3]);
  double d;
  cbg::stencil_distance(ee, X0, X1, X2, X3, d);
  int cls = filt ? 1 : 0;
  if (!filt && A.core_temp && !A.single && d <= A.xi) cls = 2;
  const double off = (cls == 0 && !A.single) ? A.xi : 0.0;
  // local frame; displacements minus their mean
  const d3 pb = mk3(xmul(xadd(xadd(xadd(P0.x, P1.x), P2.x), P3.x), 0.25),
                    xmul(xadd(xadd(xadd(P0.y, P1.y), P2.y), P3.y), 0.25),
                    xmul(xadd(xadd(xadd(P0.z, P1.z), P2.z), P3.z), 0.25));
  d3 Y0 = sub3(X0, X0), Y1 = sub3(X1, X0), Y2 = sub3(X2, X0), Y3 = sub3(X3, X0);
  const d3 Q0 = sub3(P0, pb), Q1 = sub3(P1, pb), Q2 = sub3(P2, pb), Q3 = sub3(P3, pb);
  const double n0 = norm3(Q0), n1 = norm3(Q1), n2 = norm3(Q2), n3 = norm3(Q3);
  const double lp = ee ? xadd(fmax(n0, n1), fmax(n2, n3)) : xadd(n0, fmax(fmax(n1, n2), n3));
  double t;
  int it = 0;
  const double t_c = 1.0;
  if (lp == 0.0) {
    t = t_c;
  } else {
    cbg::stencil_distance(ee, Y0, Y1, Y2, Y3, d);
    const double g0 = xsub(d, off);
    if (g0 <= 0.0) {
      t = 0.0;
      atomicOr(A.status, (unsigned long long)CB_DEV_PENETRATION);
    } else {
      const double g = xmul(ACCD_S, g0);
      t = 0.0;
      double tl = xdiv(xmul(xsub(1.0, ACCD_S), g0), lp);
      bool done = false;
      for (it = 0; it < ACCD_MAX_ITER; ++it) {
        Y0 = axpy3(Y0, tl, Q0);
        Y1 = axpy3(Y1, tl, Q1);
        Y2 = axpy3(Y2, tl, Q2);
        Y3 = axpy3(Y3, tl, Q3);
        cbg::stencil_distance(ee, Y0, Y1, Y2, Y3, d);
        if (t > 0.0 && xsub(d, off) < g) break;
        t = xadd(t, tl);
        if (t > t_c) {
          t = t_c;
          done = true;
          ++it;
          break;
        }
        tl = xdiv(xmul(ACCD_C, xsub(d, off)), lp);
      }
      if (!done) {
        if (it == ACCD_MAX_ITER) atomicOr(A.status, (unsigned long long)CB_DEV_ITER_LIMIT);
        else ++it;
      }
    }
  }
  A.t_out[q] = t;
  A.cls_out[q] = (uint8_t)cls;
  atomicMin(A.alpha_bits, (unsigned long long)__double_as_longlong(t));
  atomicMax(A.max_iters, (unsigned long long)it);
}

__global__ void k_alpha_final(const unsigned long long* bits, double* out) { *out = __longlong_as_double(*bits); }
__global__ void k_set(unsigned long long* p, unsigned long long v) { *p = v; }

}  // namespace

cb_status ccd_run(cb_scene* s, const double* x, const double* p, double* alpha, cudaStream_t st) {
  CB_TRY(broad_phase(s, s->bwc, x, p, 0.5 * s->xi, s->ccd_keys, &s->n_ccd, st));
  uint64_t* sc = scalars(s);
  unsigned long long* ab = (unsigned long long*)(sc + SC_ALPHA_BITS);
  unsigned long long* mi = (unsigned long long*)(sc + SC_ITERS);
  k_set<<<1, 1, 0, cb_count(st)>>>(ab, (unsigned long long)0x3ff0000000000000ull);  // 1.0
  k_set<<<1, 1, 0, cb_count(st)>>>(mi, 0ull);
  const int64_t np = s->n_ccd;
  if (np > 0) {
    CB_TRY(buf_ensure(s->ccd_t, sizeof(double) * (size_t)np, st));
    CB_TRY(buf_ensure(s->ccd_cls, (size_t)np, st));
    CcdArgs A;
    A.np = np;
    A.keys = bp<uint64_t>(s->ccd_keys);
    A.ev0 = bp<int32_t>(s->ev0);
    A.ev1 = bp<int32_t>(s->ev1);
    A.tv = bp<int32_t>(s->tv);
    A.comp = bp<int32_t>(s->comp);
    A.win = bp<int32_t>(s->win);
    A.frest = bp<uint64_t>(s->frest);
    A.nf = s->n_frest;
    A.T = s->T;
    A.n = s->n;
    A.kind = s->kind;
    A.filter_off = s->filter == CB_FILTER_OFF;
    A.single = s->filter == CB_FILTER_SINGLE;
    A.core_temp = s->core_temp;
    A.xi = s->xi;
    A.x = x;
    A.p = p;
    A.t_out = bp<double>(s->ccd_t);
    A.cls_out = bp<uint8_t>(s->ccd_cls);
    A.alpha_bits = ab;
    A.status = (unsigned long long*)(sc + SC_STATUS);
    A.max_iters = mi;
    k_accd<<<cb_grid(np, 128), 128, 0, cb_count(st)>>>(A);
  }
  if (alpha) k_alpha_final<<<1, 1, 0, cb_count(st)>>>(ab, alpha);
  CB_CUDA(cudaGetLastError());
  return CB_OK;
}
