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
// iterating every pair to its end: the additive CCD iterate t only grows, and
// t_p >= min(1, (1-s) g0 / l_p) =: lb_p.  Pass 1 computes lb_p for every pair
// (one distance each; pairs whose first step already passes t = 1, or that do
// not move, are resolved exactly here).  Pass 2 works in rounds with a ceiling
// h per member, starting at 4 L (L the smallest lb_p) and growing 4x: each
// round iterates the pairs with lb_p <= h, stopping a pair when it finishes
// (exact t_p) or when its iterate reaches h or the member's current minimum;
// a stopped pair keeps its iterate as its new lb_p.  After a round every
// unfinished pair has t_p >= lb_p >= min(h, m) with m the smallest exact t_p
// found, so once m <= h (or h = 1) alpha = min(1, m) exactly.  A pair's
// iteration always restarts from t = 0, so an exact t_p is the same number
// as a single uninterrupted run.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "bound32.cuh"
#include "geometry.cuh"
#include "frest.cuh"
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
  const int32_t* __restrict__ wst;
  const int32_t* __restrict__ rloop;
  const uint32_t* __restrict__ frest_j;  // partner index j of the sorted rest-filtered keys
  const uint32_t* __restrict__ frow_pt;  // ... their row offsets by vertex and by edge (frest.cuh)
  const uint32_t* __restrict__ frow_ee;
  int64_t nf;
  int T, n, kind;
  const int32_t* __restrict__ vsc;           // member of each vertex
  const MemberParams* __restrict__ mp;
  const double* __restrict__ cx;             // per member: centre[3], X
  const double* __restrict__ x;
  const double* __restrict__ p;
  double* __restrict__ t_out;
  uint8_t* __restrict__ cls_out;
  unsigned long long* __restrict__ macc;     // per member: alpha bits, lb bits, status, band lo/hi
  unsigned long long* __restrict__ status;
  unsigned long long* __restrict__ max_iters;
  const float4* __restrict__ xf;  // FP32 (x - member centre), one float4 per vertex
  const float4* __restrict__ pf;  // FP32 p, one float4 per vertex
  uint32_t* __restrict__ ulist;   // pairs left unresolved by the first step (lb < 1)
  unsigned int* __restrict__ nu;
};

__device__ __forceinline__ unsigned long long* macc_of(const CcdArgs& A, int m, int slot) {
  return &A.macc[(size_t)m * MACC_STRIDE + slot];
}

__device__ __forceinline__ d3 ld(const double* __restrict__ a, int n, int v) {
  return mk3(a[v], a[(size_t)n + v], a[2 * (size_t)n + v]);
}
__device__ __forceinline__ double norm3(d3 a) { return __dsqrt_rn(dot3(a, a)); }
__device__ __forceinline__ d3 axpy3(d3 x, double t, d3 p) {
  return mk3(xadd(x.x, xmul(t, p.x)), xadd(x.y, xmul(t, p.y)), xadd(x.z, xmul(t, p.z)));
}

// filtered class of a pair (Sec. 3.2 tables built at scene creation)
__device__ __forceinline__ bool is_filtered(const CcdArgs& A, const MemberParams& M, uint64_t key, uint32_t ki,
                                            uint32_t kj) {
  if (M.filter_off) return false;
  if (A.kind == CB_ROD) return A.comp[A.ev0[ki]] == A.comp[A.ev0[kj]] && rod_filtered(A.win, A.wst, M.loops != 0, ki, kj);
  if (A.nf <= 0) return false;
  return frest_contains(A.frest_j, A.frow_pt, A.frow_ee, key);
}

// Everything additive CCD needs before its first step.
struct AccdStart {
  bool ee;
  int cls, mem;
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
  S.mem = A.vsc[v[0]];
  const MemberParams& M = A.mp[S.mem];
  const bool filt = is_filtered(A, M, key, ki, kj);
  const d3 X0 = ld(A.x, A.n, v[0]), X1 = ld(A.x, A.n, v[1]), X2 = ld(A.x, A.n, v[2]), X3 = ld(A.x, A.n, v[3]);
  const d3 P0 = ld(A.p, A.n, v[0]), P1 = ld(A.p, A.n, v[1]), P2 = ld(A.p, A.n, v[2]), P3 = ld(A.p, A.n, v[3]);
  double d;
  cbg::stencil_distance(S.ee, X0, X1, X2, X3, d);
  S.cls = filt ? 1 : 0;
  if (!filt && M.core_temp && !M.single && d <= M.xi) S.cls = 2;
  S.off = (S.cls == 0 && !M.single) ? M.xi : 0.0;
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

__device__ __forceinline__ cbb::f3 ldf(const float4* __restrict__ a, int n, int v) {
  const float4 q = a[v];
  return cbb::f3{q.x, q.y, q.z};
}

// Minimum of non-negative doubles per member (compared as bit patterns): one
// atomicMin per warp when the warp holds one member, per lane otherwise;
// 2.0 marks "no value".
__device__ __forceinline__ void member_min_atomic(const CcdArgs& A, double v, int mem, int slot) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int m0 = __shfl_sync(0xffffffffu, mem, 0);
  if (__all_sync(0xffffffffu, mem == m0 || mem < 0)) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long u = __shfl_xor_sync(0xffffffffu, b, o);
      b = u < b ? u : b;
    }
    if ((threadIdx.x & 31) == 0 && m0 >= 0 && b < 0x4000000000000000ull) atomicMin(macc_of(A, m0, slot), b);
  } else if (mem >= 0 && b < 0x4000000000000000ull) {
    atomicMin(macc_of(A, mem, slot), b);
  }
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
// The bound is formed in FP32 with every operation rounded towards the safe
// side (__f*_rd for lower bounds, __f*_ru for upper ones) and a final factor
// 1 - 2^-23, so it stays below the first step as FP64 evaluates it; the
// thresholds are the members' FP32 copies rounded up.  (FP64 would put ~25
// operations per candidate on the FP64 pipe, which issues 1/64 as fast.)
__global__ void __launch_bounds__(128) k_ccd_screen(CcdArgs A, double* __restrict__ lb_out,
                                                    uint32_t* __restrict__ list, unsigned int* __restrict__ nlist) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool need = false, unres = false;
  double m_exact = 2.0, m_lb = 2.0;  // this lane's contributions to the two minima
  int mem = -1;
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
    mem = A.vsc[v[0]];
    const MemberParams& M = A.mp[mem];
    const bool filt = is_filtered(A, M, key, ki, kj);
    need = true;
    // Kaldor culling (rods: edges numbered along each polyline): the pair
    // does not constrain the step
    const bool culled = M.cull_radius > 0 && A.comp[A.ev0[ki]] == A.comp[A.ev0[kj]] &&
                        rod_gap(A.rloop, ki, kj) <= M.cull_radius;
    if (culled) {
      A.t_out[q] = 1.0;
      A.cls_out[q] = (uint8_t)3 | EXACT;
      m_exact = 1.0;
      need = false;
    } else {
      const double Xd = A.cx[4 * mem + 3];
      const float lb = cbb::lower_bound(ee, ldf(A.xf, A.n, v[0]), ldf(A.xf, A.n, v[1]), ldf(A.xf, A.n, v[2]),
                                        ldf(A.xf, A.n, v[3]), (float)Xd);
      if (filt || lb >= M.thrC32) {  // surely not class C at or above thrC32
        const int cls = filt ? 1 : 0;
        const float off = (cls == 0 && !M.single) ? M.xi32 : 0.f;
        const cbb::f3 p0 = ldf(A.pf, A.n, v[0]), p1 = ldf(A.pf, A.n, v[1]), p2 = ldf(A.pf, A.n, v[2]),
                      p3 = ldf(A.pf, A.n, v[3]);
        const cbb::f3 pm = cbb::fscale3(cbb::fadd3(cbb::fadd3(p0, p1), cbb::fadd3(p2, p3)), 0.25f);
        const float n0 = sqrtf(cbb::fdot3(cbb::fsub3(p0, pm), cbb::fsub3(p0, pm)));
        const float n1 = sqrtf(cbb::fdot3(cbb::fsub3(p1, pm), cbb::fsub3(p1, pm)));
        const float n2 = sqrtf(cbb::fdot3(cbb::fsub3(p2, pm), cbb::fsub3(p2, pm)));
        const float n3 = sqrtf(cbb::fdot3(cbb::fsub3(p3, pm), cbb::fsub3(p3, pm)));
        const float lp32 = ee ? fmaxf(n0, n1) + fmaxf(n2, n3) : n0 + fmaxf(fmaxf(n1, n2), n3);
        const float Pm = fmaxf(fmaxf(cbb::fmaxabs3(p0), cbb::fmaxabs3(p1)), fmaxf(cbb::fmaxabs3(p2), cbb::fmaxabs3(p3)));
        const float u64 = 3.8146973e-6f;  // 64 u, u = 2^-24: exact
        const float lp_ub = __fadd_ru(__fmul_ru(lp32, 1.f + u64), __fmul_ru(u64, Pm));
        const float slack = __fmul_ru(1e-12f, __fadd_ru(1.f, __double2float_ru(Xd)));
        const float g_lb = __fsub_rd(__fsub_rd(lb, off), slack);
        if (lp32 > 1e-30f && g_lb > 0.f) {
          // (1 - s) g / l_p; 0.9f rounds below 0.9 = 1 - s
          const float tl_lb = __fmul_rd(__fdiv_rd(__fmul_rd(0.9f, g_lb), lp_ub), 0.99999988f);
          const bool exact = tl_lb > 1.f;
          const double t = exact ? 1.0 : (double)tl_lb;
          A.t_out[q] = t;
          if (!exact) lb_out[q] = t;
          A.cls_out[q] = (uint8_t)cls | (exact ? EXACT : 0);
          if (exact) m_exact = t;
          else m_lb = t;
          unres = !exact;
          need = false;
        }
      }
    }
  }
  member_min_atomic(A, m_exact, mem, MACC_ALPHA);
  member_min_atomic(A, m_lb, mem, MACC_LB);
  warp_append(need, (uint32_t)q, list, nlist);
  warp_append(unres, (uint32_t)q, A.ulist, A.nu);
}

// pass 1b: exact FP64 first step of the queued pairs
__global__ void __launch_bounds__(128) k_ccd_bound(CcdArgs A, double* __restrict__ lb_out,
                                                   const uint32_t* __restrict__ list,
                                                   const unsigned int* __restrict__ nlist) {
  const unsigned m = *nlist;
  // uniform trip count per block so that every lane reaches the warp minima
  for (unsigned w0 = blockIdx.x * blockDim.x; w0 < m; w0 += gridDim.x * blockDim.x) {
    const unsigned w = w0 + threadIdx.x;
    double m_exact = 2.0, m_lb = 2.0;
    int mem = -1;
    bool unres = false;
    uint32_t qq = 0;
    if (w < m) {
      const int64_t q = list[w];
      const AccdStart S = accd_start(A, q);
      mem = S.mem;
      double t;
      bool exact = true;
      if (S.lp == 0.0) {
        t = 1.0;
      } else if (S.g0 <= 0.0) {
        t = 0.0;
        atomicOr(A.status, (unsigned long long)CB_DEV_PENETRATION);
        atomicOr(macc_of(A, mem, MACC_STATUS), (unsigned long long)CB_DEV_PENETRATION);
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
      if (!exact) lb_out[q] = t;
      A.cls_out[q] = (uint8_t)S.cls | (exact ? EXACT : 0);
      if (exact) m_exact = t;
      else m_lb = t;
      unres = !exact;
      qq = (uint32_t)q;
    }
    member_min_atomic(A, m_exact, mem, MACC_ALPHA);
    member_min_atomic(A, m_lb, mem, MACC_LB);
    warp_append(unres, qq, A.ulist, A.nu);
  }
}

// select the listed pairs with lb <= hi of their member: flag[w] for pair
// ulist[w], counted by kind (point-triangle in the low 32 bits, edge-edge in
// the high ones) so that the list puts each kind together: the distance
// routine branches on the kind, and a warp that mixes them runs both
__global__ void k_ccd_select_u(int64_t nu, const uint32_t* __restrict__ ulist, const uint64_t* __restrict__ keys,
                               const int32_t* __restrict__ ev0, const int32_t* __restrict__ vsc,
                               const double* __restrict__ lb, const unsigned long long* __restrict__ macc,
                               unsigned long long* __restrict__ flag) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nu) return;
  const uint32_t q = ulist[w];
  const uint64_t key = keys[q];
  const bool pt = cb_key_type(key) == CB_KEY_PT;
  const int v0 = pt ? (int)cb_key_i(key) : ev0[cb_key_i(key)];
  const int mem = vsc[v0];
  const double hi = __longlong_as_double(macc[(size_t)mem * MACC_STRIDE + MACC_HI]);
  flag[w] = lb[q] <= hi ? (pt ? 1ull : 1ull << 32) : 0ull;
}

// the selected pairs, point-triangle ones first (npt of them, the low half of
// the scan's total), each kind in list order
__global__ void k_list_u(int64_t nu, const uint32_t* __restrict__ ulist, const unsigned long long* __restrict__ flag,
                         const unsigned long long* __restrict__ pos, const unsigned long long* __restrict__ total,
                         uint32_t* __restrict__ list) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nu || !flag[w]) return;
  const unsigned long long p = pos[w];
  const uint64_t at = (flag[w] & 0xffffffffull) ? (p & 0xffffffffull) : (*total & 0xffffffffull) + (p >> 32);
  if (at < (uint64_t)nu) list[at] = ulist[w];  // always: at most nu pairs are selected
}

// pass 2: additive CCD of the selected pairs, each up to its member's ceiling.
// Pairs need very different numbers of steps, and an FP64 warp instruction
// costs a warp the same whether one lane or 32 use it, so the warps are
// persistent and hand idle lanes new pairs -- but only once EXACT_REFILL of
// them are idle (or all are): the set-up of a pair (its first distance) then
// runs once for a group of lanes instead of once per lane that finishes.
// A pair's arithmetic is the same whichever lane runs it.
constexpr int EXACT_REFILL = 8;

struct ExactLane {
  AccdStart S;
  int64_t q;
  double t, tl, g, hi, cap;
  int it;
};

// finish a pair: exact t_p (lower-bound flag clear) or a lower bound
__device__ __forceinline__ void exact_finish(const CcdArgs& A, const ExactLane& L, double* __restrict__ lb_out,
                                             bool stopped, double t) {
  A.t_out[L.q] = t;
  if (stopped) {
    A.cls_out[L.q] = (uint8_t)L.S.cls;
    lb_out[L.q] = t;
    return;
  }
  A.cls_out[L.q] = (uint8_t)L.S.cls | EXACT;
  lb_out[L.q] = 2.0;
  atomicMin(macc_of(A, L.S.mem, MACC_ALPHA), (unsigned long long)__double_as_longlong(t));
}

// fetch: a zeroed counter of the pairs handed out
__global__ void __launch_bounds__(128) k_ccd_exact(CcdArgs A, int64_t m, const uint32_t* __restrict__ list,
                                                   double* __restrict__ lb_out,
                                                   unsigned long long* __restrict__ fetch) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned below = (1u << lane) - 1u;
  ExactLane L;
  bool have = false, drained = false;
  int max_it = 0;
  for (;;) {
    const unsigned idle = __ballot_sync(0xffffffffu, !have);
    const int nidle = __popc(idle);
    if (!drained && (nidle >= EXACT_REFILL || nidle == 32)) {
      // the group of idle lanes takes the next pairs of the list
      unsigned long long b = 0;
      if (lane == 0) b = atomicAdd(fetch, (unsigned long long)nidle);
      b = __shfl_sync(0xffffffffu, b, 0);
      if ((int64_t)b + nidle >= m) drained = true;  // nothing left after this group
      const int64_t w = (int64_t)b + __popc(idle & below);
      if (!have && w < m) {
        L.q = list[w];
        L.S = accd_start(A, L.q);
        if (L.S.lp == 0.0 || L.S.g0 <= 0.0) {  // only reachable through an FP32 bound below 1
          if (L.S.lp != 0.0) {
            atomicOr(A.status, (unsigned long long)CB_DEV_PENETRATION);
            atomicOr(macc_of(A, L.S.mem, MACC_STATUS), (unsigned long long)CB_DEV_PENETRATION);
          }
          exact_finish(A, L, lb_out, false, L.S.lp == 0.0 ? 1.0 : 0.0);
        } else {
          // ceiling: the band's upper end, lowered to the member's minimum as it falls
          L.hi = __longlong_as_double(*macc_of(A, L.S.mem, MACC_HI));
          L.cap = fmin(L.hi, __longlong_as_double(*(volatile unsigned long long*)macc_of(A, L.S.mem, MACC_ALPHA)));
          L.g = xmul(ACCD_S, L.S.g0);
          L.t = 0.0;
          L.tl = xdiv(xmul(xsub(1.0, ACCD_S), L.S.g0), L.S.lp);
          L.it = 0;
          have = true;
        }
      }
    }
    if (!__any_sync(0xffffffffu, have)) {
      if (drained) break;
      continue;  // every pair of the group finished at its set-up: fetch again
    }
    if (have) {
      // one additive-CCD step
      AccdStart& S = L.S;
      S.Y0 = axpy3(S.Y0, L.tl, S.Q0);
      S.Y1 = axpy3(S.Y1, L.tl, S.Q1);
      S.Y2 = axpy3(S.Y2, L.tl, S.Q2);
      S.Y3 = axpy3(S.Y3, L.tl, S.Q3);
      double d;
      cbg::stencil_distance(S.ee, S.Y0, S.Y1, S.Y2, S.Y3, d);
      const int it = L.it++;
      if (L.t > 0.0 && xsub(d, S.off) < L.g) {
        exact_finish(A, L, lb_out, false, L.t);
        have = false;
      } else {
        L.t = xadd(L.t, L.tl);
        if (L.t > 1.0) {
          exact_finish(A, L, lb_out, false, 1.0);
          have = false;
        } else {
          if ((it & 7) == 7)
            L.cap = fmin(L.hi, __longlong_as_double(*(volatile unsigned long long*)macc_of(A, S.mem, MACC_ALPHA)));
          if (L.cap < 1.0 && L.t >= L.cap) {  // t_p >= t >= cap: this pair cannot lower the minimum now
            exact_finish(A, L, lb_out, true, L.t);
            have = false;
          } else if (it + 1 >= ACCD_MAX_ITER) {
            atomicOr(A.status, (unsigned long long)CB_DEV_ITER_LIMIT);
            exact_finish(A, L, lb_out, false, L.t);
            have = false;
          } else {
            L.tl = xdiv(xmul(ACCD_C, xsub(d, S.off)), S.lp);
          }
        }
      }
      if (!have) max_it = max(max_it, it + 1);
    }
  }
  const int wm = __reduce_max_sync(0xffffffffu, max_it);
  if (lane == 0 && wm > 0) atomicMax(A.max_iters, (unsigned long long)wm);
}

__global__ void k_alpha_final(int count, const unsigned long long* __restrict__ macc, double* __restrict__ out) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < count) out[m] = __longlong_as_double(macc[(size_t)m * MACC_STRIDE + MACC_ALPHA]);
}
__global__ void k_set(unsigned long long* p, unsigned long long v) { *p = v; }
__global__ void k_macc_set(int count, unsigned long long* __restrict__ macc, int slot, unsigned long long v) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < count) macc[(size_t)m * MACC_STRIDE + slot] = v;
}

}  // namespace

cb_status ccd_run(cb_scene* s, const double* x, const double* p, double* alpha, cudaStream_t st) {
  CB_TRY(broad_phase(s, s->bwc, x, p, true, false, s->ccd_keys, &s->n_ccd, st));
  uint64_t* sc = scalars(s);
  const int M = s->count;
  unsigned long long* macc = bp<unsigned long long>(s->macc);
  unsigned long long* mi = (unsigned long long*)(sc + SC_ITERS);
  k_macc_set<<<cb_grid(M), CB_THREADS, 0, cb_count(st)>>>(M, macc, MACC_ALPHA, 0x3ff0000000000000ull);  // 1.0
  k_macc_set<<<cb_grid(M), CB_THREADS, 0, cb_count(st)>>>(M, macc, MACC_LB, 0x4000000000000000ull);     // 2.0
  k_macc_set<<<cb_grid(M), CB_THREADS, 0, cb_count(st)>>>(M, macc, MACC_STATUS, 0ull);
  k_set<<<1, 1, 0, cb_count(st)>>>(mi, 0ull);
  const int64_t np = s->n_ccd;
  if (np > 0) {
    CB_TRY(buf_ensure(s->ccd_t, sizeof(double) * (size_t)np, st));
    CB_TRY(buf_ensure(s->ccd_cls, (size_t)np, st));
    CB_TRY(buf_ensure(s->ccd_lb, sizeof(double) * (size_t)np, st));
    CB_TRY(buf_ensure(s->ccd_flag, sizeof(unsigned long long) * (size_t)np, st));
    CB_TRY(buf_ensure(s->ccd_pos, sizeof(unsigned long long) * ((size_t)np + 1), st));
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
    A.wst = bp<int32_t>(s->wst);
    A.rloop = bp<int32_t>(s->rloop);
    A.frest_j = bp<uint32_t>(s->frest_j);
    A.frow_pt = bp<uint32_t>(s->frow_pt);
    A.frow_ee = bp<uint32_t>(s->frow_ee);
    A.nf = s->n_frest;
    A.T = s->T;
    A.n = s->n;
    A.kind = s->kind;
    A.vsc = bp<int32_t>(s->vsc);
    A.mp = bp<MemberParams>(s->mp);
    A.cx = bp<double>(s->bwc.cx);
    A.x = x;
    A.p = p;
    A.t_out = bp<double>(s->ccd_t);
    A.cls_out = bp<uint8_t>(s->ccd_cls);
    A.macc = macc;
    A.status = (unsigned long long*)(sc + SC_STATUS);
    A.max_iters = mi;
    CB_TRY(to_f32(s, x, bp<double>(s->bwc.cx), s->xf, st));
    CB_TRY(to_f32(s, p, nullptr, s->pf, st));
    A.xf = bp<float4>(s->xf);
    A.pf = bp<float4>(s->pf);
    CB_TRY(buf_ensure(s->dlist, sizeof(uint32_t) * (size_t)np, st));
    CB_TRY(buf_ensure(s->ccd_ulist, sizeof(uint32_t) * (size_t)np, st));
    unsigned int* nl = (unsigned int*)(sc + SC_NLIST);
    k_set<<<1, 1, 0, cb_count(st)>>>((unsigned long long*)(sc + SC_NLIST), 0ull);
    k_set<<<1, 1, 0, cb_count(st)>>>((unsigned long long*)(sc + SC_NU), 0ull);
    A.ulist = bp<uint32_t>(s->ccd_ulist);
    A.nu = (unsigned int*)(sc + SC_NU);
    k_ccd_screen<<<cb_grid(np, 128), 128, 0, cb_count(st)>>>(A, bp<double>(s->ccd_lb), bp<uint32_t>(s->dlist), nl);
    k_ccd_bound<<<std::min<int64_t>(cb_grid(np, 128), (int64_t)s->n_sms * 16), 128, 0, cb_count(st)>>>(
        A, bp<double>(s->ccd_lb), bp<uint32_t>(s->dlist), nl);
    CB_CUDA(cudaGetLastError());
    // Per member: the pairs left unresolved by pass 1 (lb < 1, listed by the
    // pass-1 kernels themselves) go through rounds with ceiling
    // h = 4 L, 16 L, ... (capped at 1) until the member's minimum is <= h.
    // Members whose minimum is already below every remaining bound are done
    // after pass 1.
    std::vector<unsigned long long> hm((size_t)M * MACC_STRIDE);
    auto read_macc = [&]() -> cb_status {
      CB_CUDA(cudaMemcpyAsync(s->hstage_host, macc, sizeof(unsigned long long) * MACC_STRIDE * M,
                              cudaMemcpyDeviceToHost, st));
      CB_CUDA(cudaStreamSynchronize(st));
      memcpy(hm.data(), s->hstage_host, sizeof(unsigned long long) * MACC_STRIDE * M);
      return CB_OK;
    };
    auto upload_band = [&](const std::vector<double>& lo, const std::vector<double>& hi) -> cb_status {
      // hm holds the device values read just before, and no kernel runs in between
      for (int m = 0; m < M; ++m) {
        memcpy(&hm[(size_t)m * MACC_STRIDE + MACC_LO], &lo[m], 8);
        memcpy(&hm[(size_t)m * MACC_STRIDE + MACC_HI], &hi[m], 8);
      }
      memcpy(s->hstage_host, hm.data(), sizeof(unsigned long long) * MACC_STRIDE * M);
      CB_CUDA(cudaMemcpyAsync(macc, s->hstage_host, sizeof(unsigned long long) * MACC_STRIDE * M,
                              cudaMemcpyHostToDevice, st));
      return CB_OK;
    };
    auto dbl = [](unsigned long long b) {
      double d;
      memcpy(&d, &b, 8);
      return d;
    };
    CB_TRY(read_macc());
    std::vector<double> lo(M, 3.0), hi(M, -1.0);
    std::vector<char> done(M, 1);
    bool any = false;
    for (int m = 0; m < M; ++m) {
      const double L = dbl(hm[(size_t)m * MACC_STRIDE + MACC_LB]);
      const double mm = dbl(hm[(size_t)m * MACC_STRIDE + MACC_ALPHA]);
      if (!(L > 1.0 || mm <= L)) {
        done[m] = 0;
        lo[m] = -1.0;
        hi[m] = 1.0;
        any = true;
      }
    }
    uint32_t* tot = (uint32_t*)(sc + SC_COUNT1);
    int64_t nu = 0;
    if (any) {
      uint64_t hn;
      CB_TRY(read_scalars(s, SC_NU, 1, &hn, st));
      nu = (int64_t)(uint32_t)hn;
      for (int m = 0; m < M; ++m)
        if (!done[m]) hi[m] = std::min(1.0, 4.0 * dbl(hm[(size_t)m * MACC_STRIDE + MACC_LB]));
      any = nu > 0;
    }
    while (any) {
      CB_TRY(upload_band(lo, hi));
      unsigned long long* flag64 = bp<unsigned long long>(s->ccd_flag);
      unsigned long long* pos64 = bp<unsigned long long>(s->ccd_pos);
      unsigned long long* tot64 = (unsigned long long*)tot;
      k_ccd_select_u<<<cb_grid(nu), CB_THREADS, 0, cb_count(st)>>>(
          nu, bp<uint32_t>(s->ccd_ulist), bp<uint64_t>(s->ccd_keys), bp<int32_t>(s->ev0), bp<int32_t>(s->vsc),
          bp<double>(s->ccd_lb), macc, flag64);
      cbp::exclusive_scan<unsigned long long, unsigned long long>(flag64, pos64, nu,
                                                                  bp<unsigned long long>(s->scan_tmp), tot64, st);
      k_list_u<<<cb_grid(nu), CB_THREADS, 0, cb_count(st)>>>(nu, bp<uint32_t>(s->ccd_ulist), flag64, pos64, tot64,
                                                             bp<uint32_t>(s->ccd_list));
      uint64_t hmsel;
      CB_TRY(read_scalars(s, SC_COUNT1, 1, &hmsel, st));
      const int64_t msel = (int64_t)(hmsel & 0xffffffffull) + (int64_t)(hmsel >> 32);
      if (msel > 0) {
        // persistent warps: at most three 128-thread blocks per SM (the
        // kernel's registers), fewer when the list is short
        unsigned long long* fetch = (unsigned long long*)(sc + SC_FETCH);
        CB_CUDA(cudaMemsetAsync(fetch, 0, sizeof(unsigned long long), st));
        const int64_t g = std::min<int64_t>(cb_grid(msel, 128), (int64_t)s->n_sms * 3);
        k_ccd_exact<<<(int)g, 128, 0, cb_count(st)>>>(A, msel, bp<uint32_t>(s->ccd_list), bp<double>(s->ccd_lb),
                                                      fetch);
      }
      CB_CUDA(cudaGetLastError());
      CB_TRY(read_macc());
      any = false;
      for (int m = 0; m < M; ++m) {
        if (done[m]) continue;
        const double mm = dbl(hm[(size_t)m * MACC_STRIDE + MACC_ALPHA]);
        if (mm <= hi[m] || hi[m] >= 1.0) {
          done[m] = 1;  // every unfinished pair has t_p >= lb_p >= min(h, m)
          hi[m] = -1.0;
        } else {
          hi[m] = std::min(1.0, 4.0 * hi[m]);
          any = true;
        }
      }
    }
  }
  if (alpha) k_alpha_final<<<cb_grid(M), CB_THREADS, 0, cb_count(st)>>>(M, macc, alpha);
  CB_CUDA(cudaGetLastError());
  return CB_OK;
}

// ---------------------------------------------------------------------------
// ccd_step_noalloc: the same additive-CCD step bound over a caller-given list
// of stencils, with no device allocation at all.
//
// Some callers cannot allocate device memory while they run the step bound: a
// solver that has handed a fixed budget of the device to a memory pool, or a
// time-critical loop where an allocation or a free could stall the device.
// For them every buffer this call needs is the one array below, allocated when
// the library's code is loaded onto a device.  The first call on each device
// looks up its address (and may make the CUDA runtime load this code onto that
// device), so it should come before any stream capture.  The array is shared
// by every call on a device: calls that overlap in time on one device (two
// streams, two host threads) race and give wrong results.
//
// Layout (64-bit words): NA_SLOTS accumulator words (alpha bits, smallest
// lower bound bits, condition flags), then one lower bound per stencil.

namespace {
constexpr int NA_SLOTS = 32;  // 256 bytes: keeps the per-stencil part 256-byte aligned
constexpr int NA_ALPHA = 0, NA_LB = 1, NA_FLAGS = 2;
constexpr unsigned long long NA_ONE = 0x3ff0000000000000ull;  // 1.0
constexpr unsigned long long NA_TWO = 0x4000000000000000ull;  // 2.0: "no value"
}  // namespace

static __device__ __align__(256) unsigned long long g_noalloc_scratch[NA_SLOTS + CB_NOALLOC_MAX_STENCILS];

namespace {

struct NaArgs {
  int64_t ns;
  int n;
  const int32_t* __restrict__ st;   // [ns][4] vertex ids
  const uint8_t* __restrict__ ee;   // [ns] 1 edge-edge, 0 point-triangle
  const double* __restrict__ off;   // [ns] offset
  const double* __restrict__ x;
  const double* __restrict__ p;
  unsigned long long* __restrict__ scr;
};

struct NaStart {
  bool ee;
  double off, lp, g0;
  d3 Y0, Y1, Y2, Y3, Q0, Q1, Q2, Q3;
};

// first-step data of stencil q (the same arithmetic as accd_start); false for
// a stencil with a vertex id outside [0, n), an offset that is negative or
// not finite, or positions / displacements that make its distance or motion
// bound non-finite (such a stencil is reported, never silently passed)
__device__ __forceinline__ bool na_start(const NaArgs& A, int64_t q, NaStart& S) {
  int v[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[k] = A.st[4 * q + k];
    if (v[k] < 0 || v[k] >= A.n) return false;
  }
  S.ee = A.ee[q] != 0;
  S.off = A.off[q];
  if (!(S.off >= 0.0) || !isfinite(S.off)) return false;
  const d3 X0 = ld(A.x, A.n, v[0]), X1 = ld(A.x, A.n, v[1]), X2 = ld(A.x, A.n, v[2]), X3 = ld(A.x, A.n, v[3]);
  const d3 P0 = ld(A.p, A.n, v[0]), P1 = ld(A.p, A.n, v[1]), P2 = ld(A.p, A.n, v[2]), P3 = ld(A.p, A.n, v[3]);
  double d;
  cbg::stencil_distance(S.ee, X0, X1, X2, X3, d);
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
  // fmax drops a NaN operand, so a non-finite displacement is caught from the norms themselves
  if (!isfinite(n0) || !isfinite(n1) || !isfinite(n2) || !isfinite(n3) || !isfinite(d)) return false;
  S.lp = S.ee ? xadd(fmax(n0, n1), fmax(n2, n3)) : xadd(n0, fmax(fmax(n1, n2), n3));
  S.g0 = (S.lp != 0.0) ? xsub(d, S.off) : 0.0;
  return isfinite(S.lp) && isfinite(S.g0);
}

// one atomicMin per warp of the lanes' non-negative values (2.0 = none)
__device__ __forceinline__ void na_warp_min(unsigned long long* slot, double v) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long u = __shfl_xor_sync(0xffffffffu, b, o);
    b = u < b ? u : b;
  }
  if ((threadIdx.x & 31) == 0 && b < NA_TWO) atomicMin(slot, b);
}

__global__ void k_na_init(unsigned long long* __restrict__ scr) {
  if (threadIdx.x == 0) {
    scr[NA_ALPHA] = NA_ONE;
    scr[NA_LB] = NA_TWO;
    scr[NA_FLAGS] = 0ull;
  }
}

// first step of every stencil: resolves t_p = 1 (no motion, or the first step
// already passes 1) and t_p = 0 (at or inside the offset); otherwise stores
// the lower bound (1-s) g0 / l_p of t_p
__global__ void __launch_bounds__(128) k_na_first(NaArgs A) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double m_exact = 2.0, m_lb = 2.0;
  if (q < A.ns) {
    NaStart S;
    double lbq = 2.0;
    if (!na_start(A, q, S)) {
      atomicOr(&A.scr[NA_FLAGS], (unsigned long long)CB_NOALLOC_BAD_STENCIL);
    } else if (S.lp == 0.0) {
      m_exact = 1.0;
    } else if (S.g0 <= 0.0) {
      m_exact = 0.0;
      atomicOr(&A.scr[NA_FLAGS], (unsigned long long)CB_DEV_PENETRATION);
    } else {
      const double tl = xdiv(xmul(xsub(1.0, ACCD_S), S.g0), S.lp);
      if (tl > 1.0) {
        m_exact = 1.0;
      } else {
        lbq = tl;
        m_lb = tl;
      }
    }
    A.scr[NA_SLOTS + q] = (unsigned long long)__double_as_longlong(lbq);
  }
  na_warp_min(&A.scr[NA_ALPHA], m_exact);
  na_warp_min(&A.scr[NA_LB], m_lb);
}

// full additive CCD of stencil q (the iteration of k_ccd_exact)
__device__ double na_iterate(const NaArgs& A, int64_t q) {
  NaStart S;
  if (!na_start(A, q, S)) return 2.0;
  if (S.lp == 0.0) return 1.0;
  if (S.g0 <= 0.0) return 0.0;
  const double g = xmul(ACCD_S, S.g0);
  double t = 0.0, d;
  double tl = xdiv(xmul(xsub(1.0, ACCD_S), S.g0), S.lp);
  for (int it = 0; it < ACCD_MAX_ITER; ++it) {
    S.Y0 = axpy3(S.Y0, tl, S.Q0);
    S.Y1 = axpy3(S.Y1, tl, S.Q1);
    S.Y2 = axpy3(S.Y2, tl, S.Q2);
    S.Y3 = axpy3(S.Y3, tl, S.Q3);
    cbg::stencil_distance(S.ee, S.Y0, S.Y1, S.Y2, S.Y3, d);
    if (t > 0.0 && xsub(d, S.off) < g) return t;
    t = xadd(t, tl);
    if (t > 1.0) return 1.0;
    tl = xdiv(xmul(ACCD_C, xsub(d, S.off)), S.lp);
  }
  atomicOr(&A.scr[NA_FLAGS], (unsigned long long)CB_DEV_ITER_LIMIT);
  return t;
}

// Bands of lower bounds, as in ccd_run but decided on the device: band 0 is
// (-1, min(1, 2L)] with L the smallest bound; band 1 is (hi0, min(1, m)] with
// m the minimum after band 0.  Every stencil left after band 1 has
// t_p >= lb_p > m, so alpha = min(1, m) exactly.  The minimum is read once per
// block: a smaller value seen later only narrows the band to stencils that
// still could lower it.
__global__ void __launch_bounds__(128) k_na_band(NaArgs A, int band) {
  __shared__ double s_lo, s_hi;
  if (threadIdx.x == 0) {
    const double L = __longlong_as_double(A.scr[NA_LB]);
    const double m = __longlong_as_double(A.scr[NA_ALPHA]);
    const double h0 = fmin(1.0, 2.0 * L);
    double lo = 3.0, hi = 3.0;  // empty band
    if (!(L > 1.0 || m <= L)) {
      if (band == 0) {
        lo = -1.0;
        hi = h0;
      } else if (!(m <= h0 || h0 >= 1.0)) {
        lo = h0;
        hi = fmin(1.0, m);
      }
    }
    s_lo = lo;
    s_hi = hi;
  }
  __syncthreads();
  const double lo = s_lo, hi = s_hi;
  if (lo >= 3.0) return;  // uniform over the block
  for (int64_t w0 = (int64_t)blockIdx.x * blockDim.x; w0 < A.ns; w0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = w0 + threadIdx.x;
    double t = 2.0;
    if (q < A.ns) {
      const double lbq = __longlong_as_double(A.scr[NA_SLOTS + q]);
      if (lbq > lo && lbq <= hi) t = na_iterate(A, q);
    }
    na_warp_min(&A.scr[NA_ALPHA], t);
  }
}

__global__ void k_na_final(const unsigned long long* __restrict__ scr, double* __restrict__ alpha,
                           uint32_t* __restrict__ flags) {
  if (threadIdx.x == 0) {
    *alpha = __longlong_as_double(scr[NA_ALPHA]);
    *flags = (uint32_t)scr[NA_FLAGS];
  }
}

constexpr int NA_MAX_DEVICES = 256;
std::mutex g_na_mutex;
unsigned long long* g_na_ptr[NA_MAX_DEVICES];
int g_na_sms[NA_MAX_DEVICES];

// address of the scratch array on the current device and the device's SM
// count, looked up once per device (valid until the device is reset)
cb_status na_scratch(int* dev_out, unsigned long long** out, int* sms) {
  int dev = -1;
  CB_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= NA_MAX_DEVICES) return CB_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
      fprintf(stderr, "contact: ccd_step_noalloc: scratch address lookup failed on device %d: %s\n", dev,
              cudaGetErrorString(e));
      return CB_ERR_CUDA;
    }
    int nsm = 0;
    CB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    g_na_sms[dev] = nsm > 0 ? nsm : 1;
    g_na_ptr[dev] = (unsigned long long*)ptr;
  }
  *dev_out = dev;
  *out = g_na_ptr[dev];
  *sms = g_na_sms[dev];
  return CB_OK;
}

// true if p is device memory of `dev` or managed memory; a host pointer or
// memory of another device is rejected before any kernel dereferences it
bool na_on_device(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free error of an unknown pointer
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

cb_status ccd_step_noalloc(const double* x_dev, const double* p_dev, int32_t n_verts, const int32_t* stencils_dev,
                           const uint8_t* is_ee_dev, const double* offset_dev, int64_t n_stencils,
                           double* alpha_dev, uint32_t* flags_dev, void* stream) {
  if (!alpha_dev || !flags_dev || n_verts < 0 || n_stencils < 0) return CB_ERR_ARG;
  if (n_stencils > CB_NOALLOC_MAX_STENCILS) {
    fprintf(stderr, "contact: ccd_step_noalloc: %lld stencils exceed the fixed maximum of %d per call\n",
            (long long)n_stencils, (int)CB_NOALLOC_MAX_STENCILS);
    return CB_ERR_TOO_LARGE;
  }
  if (n_stencils > 0 && (n_verts < 1 || !x_dev || !p_dev || !stencils_dev || !is_ee_dev || !offset_dev))
    return CB_ERR_ARG;
  unsigned long long* scr = nullptr;
  int dev = -1, nsm = 1;
  CB_TRY(na_scratch(&dev, &scr, &nsm));
  if (!na_on_device(alpha_dev, dev) || !na_on_device(flags_dev, dev)) return CB_ERR_ARG;
  if (n_stencils > 0 && (!na_on_device(x_dev, dev) || !na_on_device(p_dev, dev) ||
                         !na_on_device(stencils_dev, dev) || !na_on_device(is_ee_dev, dev) ||
                         !na_on_device(offset_dev, dev)))
    return CB_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  k_na_init<<<1, 32, 0, cb_count(st)>>>(scr);
  if (n_stencils > 0) {
    NaArgs A;
    A.ns = n_stencils;
    A.n = n_verts;
    A.st = stencils_dev;
    A.ee = is_ee_dev;
    A.off = offset_dev;
    A.x = x_dev;
    A.p = p_dev;
    A.scr = scr;
    k_na_first<<<cb_grid(n_stencils, 128), 128, 0, cb_count(st)>>>(A);
    // the band kernels stride over the list: up to 16 resident blocks of 128 threads per SM
    const int gb = (int)std::min<int64_t>(cb_grid(n_stencils, 128), (int64_t)nsm * 16);
    k_na_band<<<gb, 128, 0, cb_count(st)>>>(A, 0);
    k_na_band<<<gb, 128, 0, cb_count(st)>>>(A, 1);
  }
  k_na_final<<<1, 32, 0, cb_count(st)>>>(scr, alpha_dev, flags_dev);
  CB_CUDA(cudaGetLastError());
  return CB_OK;
}
