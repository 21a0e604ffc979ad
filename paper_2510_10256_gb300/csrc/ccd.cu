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
// alpha = min(1, m) exactly; otherwise the band (hi, m] is evaluated, after
// which the same holds.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "bound32.cuh"
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
  const float* __restrict__ xf;   // FP32 (x - centre)
  const float* __restrict__ pf;   // FP32 p
  float X;                        // max |x - centre|
  double thrC;                    // U pairs with a distance bound above this are surely not class C
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

__device__ __forceinline__ cbb::f3 ldf(const float* __restrict__ a, int n, int v) {
  return cbb::f3{a[v], a[(size_t)n + v], a[2 * (size_t)n + v]};
}

// Minimum of non-negative doubles over the warp (compared as bit patterns),
// one atomicMin per warp; 2.0 marks "no value".
__device__ __forceinline__ void warp_min_atomic(double v, unsigned long long* __restrict__ dst) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long u = __shfl_xor_sync(0xffffffffu, b, o);
    b = u < b ? u : b;
  }
  if ((threadIdx.x & 31) == 0 && b < 0x4000000000000000ull) atomicMin(dst, b);
}

__device__ __forceinline__ void warp_append(bool flag, uint32_t value, uint32_t* __restrict__ list,
                                            unsigned int* __restrict__ count) {
  const unsigned m = __ballot_sync(0xffffffffu, flag);
  if (!m) return;
  const unsigned lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  unsigned base = 0;
  if ((int)lane == leader) base = atomicAdd(count, (unsigned)__popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (flag) list[base + __popc(m & ((1u << lane) - 1u))] = value;
}

// pass 1a: an FP32 lower bound of the distance and an FP32 upper bound of
// l_p give a lower bound of the first step.  A pair whose class is certain and
// whose bound exceeds 1 is resolved (t_p = 1); a smaller bound is kept as its
// lower bound.  Pairs the FP32 bounds cannot settle are queued for pass 1b.
__global__ void __launch_bounds__(128) k_ccd_screen(CcdArgs A, double* __restrict__ lb_out,
                                                    uint32_t* __restrict__ list, unsigned int* __restrict__ nlist) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool need = false;
  double m_exact = 2.0, m_lb = 2.0;  // this lane's contributions to the two minima
  if (q < A.np) {
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
    need = true;
    const float lb = cbb::lower_bound(ee, ldf(A.xf, A.n, v[0]), ldf(A.xf, A.n, v[1]), ldf(A.xf, A.n, v[2]),
                                      ldf(A.xf, A.n, v[3]), A.X);
    if (filt || (double)lb >= A.thrC) {
      const int cls = filt ? 1 : 0;
      const double off = (cls == 0 && !A.single) ? A.xi : 0.0;
      const cbb::f3 p0 = ldf(A.pf, A.n, v[0]), p1 = ldf(A.pf, A.n, v[1]), p2 = ldf(A.pf, A.n, v[2]),
                    p3 = ldf(A.pf, A.n, v[3]);
      const cbb::f3 pm = cbb::fscale3(cbb::fadd3(cbb::fadd3(p0, p1), cbb::fadd3(p2, p3)), 0.25f);
      const float n0 = sqrtf(cbb::fdot3(cbb::fsub3(p0, pm), cbb::fsub3(p0, pm)));
      const float n1 = sqrtf(cbb::fdot3(cbb::fsub3(p1, pm), cbb::fsub3(p1, pm)));
      const float n2 = sqrtf(cbb::fdot3(cbb::fsub3(p2, pm), cbb::fsub3(p2, pm)));
      const float n3 = sqrtf(cbb::fdot3(cbb::fsub3(p3, pm), cbb::fsub3(p3, pm)));
      const float lp32 = ee ? fmaxf(n0, n1) + fmaxf(n2, n3) : n0 + fmaxf(fmaxf(n1, n2), n3);
      const float Pm = fmaxf(fmaxf(cbb::fmaxabs3(p0), cbb::fmaxabs3(p1)), fmaxf(cbb::fmaxabs3(p2), cbb::fmaxabs3(p3)));
      const float u = 5.9604645e-8f;
      const double lp_ub = (double)lp32 * (1.0 + 64.0 * u) + 64.0 * u * (double)Pm;
      const double g_lb = (double)lb - off - 1e-12 * (1.0 + (double)A.X);
      if (lp32 > 1e-30f && g_lb > 0.0) {
        const double tl_lb = (1.0 - ACCD_S) * g_lb / lp_ub * (1.0 - 1e-9);
        const bool exact = tl_lb > 1.0 + 1e-9;
        const double t = exact ? 1.0 : tl_lb;
        A.t_out[q] = t;
        lb_out[q] = exact ? 2.0 : t;
        A.cls_out[q] = (uint8_t)cls | (exact ? EXACT : 0);
        if (exact) m_exact = t;
        else m_lb = t;
        need = false;
      }
    }
  }
  warp_min_atomic(m_exact, A.alpha_bits);
  warp_min_atomic(m_lb, A.lb_bits);
  warp_append(need, (uint32_t)q, list, nlist);
}

// pass 1b: exact FP64 first step of the queued pairs
__global__ void __launch_bounds__(128) k_ccd_bound(CcdArgs A, double* __restrict__ lb_out,
                                                   const uint32_t* __restrict__ list,
                                                   const unsigned int* __restrict__ nlist) {
  const unsigned m = *nlist;
  double m_exact = 2.0, m_lb = 2.0;
  for (unsigned w = blockIdx.x * blockDim.x + threadIdx.x; w < m; w += gridDim.x * blockDim.x) {
    const int64_t q = list[w];
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
    if (exact) m_exact = fmin(m_exact, t);
    else m_lb = fmin(m_lb, t);
  }
  warp_min_atomic(m_exact, A.alpha_bits);
  warp_min_atomic(m_lb, A.lb_bits);
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
  if (S.lp == 0.0 || S.g0 <= 0.0) {  // only reachable through an FP32 bound below 1
    const double t0 = S.lp == 0.0 ? 1.0 : 0.0;
    if (S.lp != 0.0) atomicOr(A.status, (unsigned long long)CB_DEV_PENETRATION);
    A.t_out[q] = t0;
    A.cls_out[q] = (uint8_t)S.cls | EXACT;
    atomicMin(A.alpha_bits, (unsigned long long)__double_as_longlong(t0));
    return;
  }
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
    CB_TRY(to_f32(s, x, s->bwc.ctr, s->xf, st));
    CB_TRY(to_f32(s, p, nullptr, s->pf, st));
    A.xf = bp<float>(s->xf);
    A.pf = bp<float>(s->pf);
    A.X = (float)s->bwc.X;
    A.thrC = s->xi * (1.0 + 1e-9) + 1e-9;
    CB_TRY(buf_ensure(s->dlist, sizeof(uint32_t) * (size_t)np, st));
    unsigned int* nl = (unsigned int*)(sc + SC_NLIST);
    k_set<<<1, 1, 0, cb_count(st)>>>((unsigned long long*)(sc + SC_NLIST), 0ull);
    k_ccd_screen<<<cb_grid(np, 128), 128, 0, cb_count(st)>>>(A, bp<double>(s->ccd_lb), bp<uint32_t>(s->dlist), nl);
    k_ccd_bound<<<std::min<int64_t>(cb_grid(np, 128), 152 * 16), 128, 0, cb_count(st)>>>(
        A, bp<double>(s->ccd_lb), bp<uint32_t>(s->dlist), nl);
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
      // only pairs with lb_p <= m can still lower the minimum: one more band
      // (hi, m] makes it exact
      lo = hi;
      hi = std::min(1.0, m);
    }
  }
  if (alpha) k_alpha_final<<<1, 1, 0, cb_count(st)>>>(ab, alpha);
  CB_CUDA(cudaGetLastError());
  return CB_OK;
}
