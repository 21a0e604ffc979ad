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
//
// Only the minimum is needed, so the step bound is computed exactly without
// iterating every pair: the additive CCD result is never below its first step,
// t_p >= min(1, (1-s) g0 / l_p) =: lb_p.  Pass 1 computes lb_p for every pair
// (one distance each; pairs whose first step already passes t = 1, or that do
// not move, are resolved exactly here).  Pass 2 runs the full iteration on the
// unresolved pairs with lb_p in a band (lo, hi]; once the minimum m found so
// far is <= hi, every pair left has t_p >= lb_p > hi >= m and
// alpha = min(1, m) exactly; otherwise the next band is evaluated.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "geometry.cuh"
#include "prims.cuh"
#include "scene.cuh"

namespace {

constexpr double ACCD_S = 0.1;
constexpr double ACCD_C = 0.9;
constexpr int ACCD_MAX_ITER = 10000;
constexpr uint8_t EXACT = 0x80;   // class byte flag: t_p is exact (else a lower bound)

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
  unsigned long long* __restrict__ alpha_bits;  // min over exact t_p
  unsigned long long* __restrict__ lb_bits;     // min over lower bounds of unresolved pairs
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

// Everything additive CCD needs before its first step.
struct AccdStart {
  bool ee;
  int cls;
  double off, lp, g0;
  d3 Y0, Y1, Y2, Y3, Q0, Q1, Q2, Q3;
};

__device__ __forceinline__ AccdStart accd_start(const CcdArgs& A, int64_t q) {
  AccdStart S;
  const uint64_t key = A.keys[q];
  const uint32_t ty = cb_key_type(key), ki = cb_key_i(key), kj = cb_key_j(key);
  int v[4];
  if (ty == CB_KEY_PT) {
    v[0] = (int)ki;
    v[1] = A.tv[kj];
    v[2] = A.tv[A.T + kj];
    v[3] = A.tv[2 * A.T + kj];
    S.ee = false;
  } else {
    v[0] = A.ev0[ki];
    v[1] = A.ev1[ki];
    v[2] = A.ev0[kj];
    v[3] = A.ev1[kj];
    S.ee = true;
  }
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
  const d3 X0 = ld(A.x, A.n, v[0]), X1 = ld(A.x, A.n, v[1]), X2 = ld(A.x, A.n, v[2]), X3 = ld(A.x, A.n, v[3]);
  const d3 P0 = ld(A.p, A.n, v[0]), P1 = ld(A.p, A.n, v[1]), P2 = ld(A.p, A.n, v[2]), P3 = ld(A.p, A.n, v[3]);
  double d;
  cbg::stencil_distance(S.ee, X0, X1, X2, X3, d);
  S.cls = filt ? 1 : 0;
  if (!filt && A.core_temp && !A.single && d <= A.xi) S.cls = 2;
  S.off = (S.cls == 0 && !A.single) ? A.xi : 0.0;
  const d3 pb = mk3(xmul(xadd(xadd(xadd(P0.x, P1.x), P2.x), P3.x), 0.25),
                    xmul(xadd(xadd(xadd(P0.y, P1.y), P2.y), P3.y), 0.25),
                    xmul(xadd(xadd(xadd(P0.z, P1.z), P2.z), P3.z), 0.25));
  S.Y0 = sub3(X0, X0);
  S.Y1 = sub3(X1, X0);
  S.Y2 = sub3(X2, X0);
  S.Y3 = sub3(X3, X0);
  S.Q0 = sub3(P0, pb);
  S.Q1 = sub3(P1, pb);
  S.Q2 = sub3(P2, pb);
  S.Q3 = sub3(P3, pb);
  const double n0 = norm3(S.Q0), n1 = norm3(S.Q1), n2 = norm3(S.Q2), n3 = norm3(S.Q3);
  S.lp = S.ee ? xadd(fmax(n0, n1), fmax(n2, n3)) : xadd(n0, fmax(fmax(n1, n2), n3));
  // The distance of the local-frame copy Y (Y0 = 0) equals d bit for bit: the
  // distance routine itself works relative to the first vertex, and
  // (x_i - x_0) - 0 = x_i - x_0 exactly.
  S.g0 = (S.lp != 0.0) ? xsub(d, S.off) : 0.0;
  return S;
}

// pass 1: lower bound (or exact value) of every pair's t_p
__global__ void __launch_bounds__(128) k_ccd_bound(CcdArgs A, double* __restrict__ lb_out) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= A.np) return;
  const AccdStart S = accd_start(A, q);
  double t;
  bool exact = true;
  if (S.lp == 0.0) {
    t = 1.0;
  } else if (S.g0 <= 0.0) {
    t = 0.0;
    atomicOr(A.status, (unsigned long long)CB_DEV_PENETRATION);
  } else {
    const double tl = xdiv(xmul(xsub(1.0, ACCD_S), S.g0), S.lp);
    if (tl > 1.0) {
      t = 1.0;  // the first step already passes t_c = 1: no contact within the step
    } else {
      t = tl;
      exact = false;
    }
  }
  A.t_out[q] = t;
  lb_out[q] = exact ? 2.0 : t;  // 2: resolved (never selected again)
  A.cls_out[q] = (uint8_t)S.cls | (exact ? EXACT : 0);
  if (exact) atomicMin(A.alpha_bits, (unsigned long long)__double_as_longlong(t));
  else atomicMin(A.lb_bits, (unsigned long long)__double_as_longlong(t));
}

// select unresolved pairs with lo < lb <= hi
__global__ void k_ccd_select(int64_t np, const double* __restrict__ lb, double lo, double hi,
                             uint32_t* __restrict__ flag) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < np) flag[q] = (lb[q] > lo && lb[q] <= hi) ? 1u : 0u;
}

__global__ void k_list(int64_t np, const uint32_t* __restrict__ flag, const uint32_t* __restrict__ pos,
                       uint32_t* __restrict__ list) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < np && flag[q]) list[pos[q]] = (uint32_t)q;
}

// pass 2: full additive CCD of the selected pairs
__global__ void __launch_bounds__(128) k_ccd_exact(CcdArgs A, int64_t m, const uint32_t* __restrict__ list) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= m) return;
  const int64_t q = list[w];
  AccdStart S = accd_start(A, q);
  const double g = xmul(ACCD_S, S.g0);
  double t = 0.0, d;
  double tl = xdiv(xmul(xsub(1.0, ACCD_S), S.g0), S.lp);
  int it;
  bool capped = true;
  for (it = 0; it < ACCD_MAX_ITER; ++it) {
    S.Y0 = axpy3(S.Y0, tl, S.Q0);
    S.Y1 = axpy3(S.Y1, tl, S.Q1);
    S.Y2 = axpy3(S.Y2, tl, S.Q2);
    S.Y3 = axpy3(S.Y3, tl, S.Q3);
    cbg::stencil_distance(S.ee, S.Y0, S.Y1, S.Y2, S.Y3, d);
    if (t > 0.0 && xsub(d, S.off) < g) {
      capped = false;
      break;
    }
    t = xadd(t, tl);
    if (t > 1.0) {
      t = 1.0;
      capped = false;
      break;
    }
    tl = xdiv(xmul(ACCD_C, xsub(d, S.off)), S.lp);
  }
  if (capped) atomicOr(A.status, (unsigned long long)CB_DEV_ITER_LIMIT);
  A.t_out[q] = t;
  A.cls_out[q] = (uint8_t)S.cls | EXACT;
  atomicMin(A.alpha_bits, (unsigned long long)__double_as_longlong(t));
  atomicMax(A.max_iters, (unsigned long long)(it + 1));
}

__global__ void k_alpha_final(const unsigned long long* bits, double* out) { *out = __longlong_as_double(*bits); }
__global__ void k_set(unsigned long long* p, unsigned long long v) { *p = v; }

}  // namespace

cb_status ccd_run(cb_scene* s, const double* x, const double* p, double* alpha, cudaStream_t st) {
  CB_TRY(broad_phase(s, s->bwc, x, p, 0.5 * s->xi, s->ccd_keys, &s->n_ccd, st));
  uint64_t* sc = scalars(s);
  unsigned long long* ab = (unsigned long long*)(sc + SC_ALPHA_BITS);
  unsigned long long* lbm = (unsigned long long*)(sc + SC_COUNT0);
  unsigned long long* mi = (unsigned long long*)(sc + SC_ITERS);
  k_set<<<1, 1, 0, cb_count(st)>>>(ab, 0x3ff0000000000000ull);   // 1.0
  k_set<<<1, 1, 0, cb_count(st)>>>(lbm, 0x4000000000000000ull);  // 2.0: nothing unresolved
  k_set<<<1, 1, 0, cb_count(st)>>>(mi, 0ull);
  const int64_t np = s->n_ccd;
  if (np > 0) {
    CB_TRY(buf_ensure(s->ccd_t, sizeof(double) * (size_t)np, st));
    CB_TRY(buf_ensure(s->ccd_cls, (size_t)np, st));
    CB_TRY(buf_ensure(s->ccd_lb, sizeof(double) * (size_t)np, st));
    CB_TRY(buf_ensure(s->ccd_flag, sizeof(uint32_t) * (size_t)np, st));
    CB_TRY(buf_ensure(s->ccd_pos, sizeof(uint32_t) * ((size_t)np + 1), st));
    CB_TRY(buf_ensure(s->ccd_list, sizeof(uint32_t) * (size_t)np, st));
    CB_TRY(buf_ensure(s->scan_tmp, sizeof(uint64_t) * (size_t)(cbp::scan_tmp_elems(np) + 8), st));
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
    A.lb_bits = lbm;
    A.status = (unsigned long long*)(sc + SC_STATUS);
    A.max_iters = mi;
    k_ccd_bound<<<cb_grid(np, 128), 128, 0, cb_count(st)>>>(A, bp<double>(s->ccd_lb));
    CB_CUDA(cudaGetLastError());
    uint64_t h[2];
    CB_TRY(read_scalars(s, SC_COUNT0, 1, &h[0], st));
    CB_TRY(read_scalars(s, SC_ALPHA_BITS, 1, &h[1], st));
    double L, m;
    memcpy(&L, &h[0], 8);
    memcpy(&m, &h[1], 8);
    // bands (lo, hi] of lower bounds, grown until the exact minimum found so
    // far is not above the band's upper end (L > 1: every pair resolved)
    double lo = -1.0, hi = std::min(1.0, 2.0 * L);
    while (L <= 1.0 && m > L) {
      k_ccd_select<<<cb_grid(np), CB_THREADS, 0, cb_count(st)>>>(np, bp<double>(s->ccd_lb), lo, hi,
                                                                  bp<uint32_t>(s->ccd_flag));
      uint32_t* tot = (uint32_t*)(sc + SC_COUNT1);
      cbp::exclusive_scan<uint32_t, uint32_t>(bp<uint32_t>(s->ccd_flag), bp<uint32_t>(s->ccd_pos), np,
                                              bp<uint32_t>(s->scan_tmp), tot, st);
      k_list<<<cb_grid(np), CB_THREADS, 0, cb_count(st)>>>(np, bp<uint32_t>(s->ccd_flag), bp<uint32_t>(s->ccd_pos),
                                                           bp<uint32_t>(s->ccd_list));
      uint64_t hm;
      CB_TRY(read_scalars(s, SC_COUNT1, 1, &hm, st));
      const int64_t msel = (int64_t)(uint32_t)hm;
      if (msel > 0)
        k_ccd_exact<<<cb_grid(msel, 128), 128, 0, cb_count(st)>>>(A, msel, bp<uint32_t>(s->ccd_list));
      CB_CUDA(cudaGetLastError());
      CB_TRY(read_scalars(s, SC_ALPHA_BITS, 1, &h[1], st));
      memcpy(&m, &h[1], 8);
      if (m <= hi || hi >= 1.0) break;  // every pair left has t_p >= lb_p > hi >= m
      lo = hi;
      double nh = 4.0 * hi;
      if (!(nh > hi)) nh = 1.0;  // hi == 0 (underflowed first steps): take the rest at once
      hi = std::min(1.0, nh);
    }
  }
  if (alpha) k_alpha_final<<<1, 1, 0, cb_count(st)>>>(ab, alpha);
  CB_CUDA(cudaGetLastError());
  return CB_OK;
}
