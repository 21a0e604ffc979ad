// narrow.cu -- stages (b), (c), (d): barrier filter, distances, barrier energy,
// gradient and PSD-projected Hessian, assembly into a global gradient and BSR.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "bound32.cuh"
#include "geometry.cuh"
#include "frest.cuh"
#include "pairs.cuh"
#include "prims.cuh"
#include "scene.cuh"

namespace {


// ------------------------------------------------------------------ (b) ----

// rods: arc length S at every vertex, summed sequentially along each polyline
__global__ void k_arclength(int n_rods, const int32_t* __restrict__ rod_ptr, const double* __restrict__ rest, int n,
                            double* __restrict__ S) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rods) return;
  const int s = rod_ptr[r], e = rod_ptr[r + 1];
  if (e <= s) return;
  S[s] = 0.0;
  for (int v = s + 1; v < e; ++v) {
    double dx = xsub(rest[v], rest[v - 1]);
    double dy = xsub(rest[(size_t)n + v], rest[(size_t)n + v - 1]);
    double dz = xsub(rest[2 * (size_t)n + v], rest[2 * (size_t)n + v - 1]);
    S[v] = xadd(S[v - 1], __dsqrt_rn(xadd(xadd(xmul(dx, dx), xmul(dy, dy)), xmul(dz, dz))));
  }
}

// rods: for edge k the last edge l of the same polyline with arc-length gap
// s0(l) - s1(k) < a (the reference distance between the edges; it grows with
// l), win[k]; on a closed loop also the first edge l past that window whose
// gap the other way round, (L - s1(l)) + s0(k), is below a (it shrinks as l
// grows), wst[k] (-1 if none).  An edge spans arc lengths s0 = S[v0] to s1 =
// S[v1], the closing edge of a loop from S at the last vertex to the loop
// length L.  The reference distance of a pair is the smaller gap; incident
// pairs (a shared vertex) are skipped.
__device__ __forceinline__ double edge_len(const double* __restrict__ rest, int n, int a, int b) {
  const double dx = xsub(rest[b], rest[a]);
  const double dy = xsub(rest[(size_t)n + b], rest[(size_t)n + a]);
  const double dz = xsub(rest[2 * (size_t)n + b], rest[2 * (size_t)n + a]);
  return __dsqrt_rn(xadd(xadd(xmul(dx, dx), xmul(dy, dy)), xmul(dz, dz)));
}

__global__ void k_rod_window(int E, const int32_t* __restrict__ ev0, const int32_t* __restrict__ ev1,
                             const int32_t* __restrict__ comp, const double* __restrict__ S,
                             const double* __restrict__ rest, int n, const int32_t* __restrict__ rlast, double a,
                             int32_t* __restrict__ win, int32_t* __restrict__ wst,
                             unsigned long long* __restrict__ dmin_bits, unsigned long long* __restrict__ nfilt,
                             unsigned long long* __restrict__ dmin_comp) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= E) return;
  const int k0 = ev0[k], k1 = ev1[k];
  const int rl = rlast[k];
  const double s0k = S[k0];
  const double s1k = k1 > k0 ? S[k1] : xadd(S[k0], edge_len(rest, n, k0, k1));
  // closed loop: its length, and the gap the other way round to edge l
  const bool loop = rl >= 0 && k < rl;
  const double L = loop ? xadd(S[ev0[rl]], edge_len(rest, n, ev0[rl], ev1[rl])) : 0.0;
  auto back_gap = [&](int l) {
    const double s1l = l == rl ? L : S[ev1[l]];
    return xadd(xsub(L, s1l), s0k);
  };
  auto incident = [&](int l) {
    const int l0 = ev0[l], l1 = ev1[l];
    return l0 == k0 || l0 == k1 || l1 == k0 || l1 == k1;
  };
  int last = k + 1;
  double mn = INFINITY;
  unsigned long long cnt = 0;
  for (int l = k + 1; l < E; ++l) {
    const int l0 = ev0[l];
    if (comp[l0] != comp[k1]) break;
    if (incident(l)) continue;
    const double dbar = xsub(S[l0], s1k);
    if (!(dbar < a)) break;
    last = l;
    mn = fmin(mn, loop ? fmin(dbar, back_gap(l)) : dbar);
    ++cnt;
  }
  win[k] = last;
  int first = -1;
  if (loop) {
    for (int l = rl; l > last && l > k; --l) {
      if (incident(l)) continue;
      const double g = back_gap(l);
      if (!(g < a)) break;
      first = l;
      mn = fmin(mn, g);
      ++cnt;
    }
  }
  wst[k] = first;
  if (cnt) {
    atomicMin(dmin_bits, (unsigned long long)__double_as_longlong(mn));
    atomicMin(&dmin_comp[comp[k1]], (unsigned long long)__double_as_longlong(mn));
    atomicAdd(nfilt, cnt);
  }
}

// shells: rest candidates of one component whose rest distance is below a
__global__ void k_rest_filter(int64_t nc, const uint64_t* __restrict__ keys, const int32_t* __restrict__ ev0,
                              const int32_t* __restrict__ ev1, const int32_t* __restrict__ tv, int T,
                              const int32_t* __restrict__ comp, const double* __restrict__ rest, int n, double a,
                              uint32_t* __restrict__ flag, double* __restrict__ dbar,
                              unsigned long long* __restrict__ dmin_bits,
                              unsigned long long* __restrict__ dmin_comp) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long mb = 0x7ff0000000000000ull;  // +inf: no filtered pair in this lane
  if (c < nc) {
    Stencil s = stencil_of(keys[c], ev0, ev1, tv, T);
    uint32_t f = 0;
    double d = 0.0;
    if (comp[s.v[0]] == comp[s.v[2]]) {
      cbg::stencil_distance(s.ee, load3(rest, n, s.v[0]), load3(rest, n, s.v[1]), load3(rest, n, s.v[2]),
                            load3(rest, n, s.v[3]), d);
      if (d < a) {
        f = 1;
        mb = (unsigned long long)__double_as_longlong(d);
        atomicMin(&dmin_comp[comp[s.v[0]]], mb);
      }
    }
    flag[c] = f;
    dbar[c] = d;
  }
  // one atomicMin per warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long u = __shfl_xor_sync(0xffffffffu, mb, o);
    mb = u < mb ? u : mb;
  }
  if ((threadIdx.x & 31) == 0 && mb != 0x7ff0000000000000ull) atomicMin(dmin_bits, mb);
}

// Per-stencil activation: whether the FP64 boxes of a pair's two primitives
// (uninflated boxes of the static broad phase), each inflated by half the
// pair's own width fw, overlap on all three axes (closed intervals).
__device__ __forceinline__ bool within_own_width(const double* __restrict__ box_raw, int64_t prim1, int64_t prim2,
                                                 double fw) {
  const double h = xmul(0.5, fw);
  const double* b1 = box_raw + prim1 * 6;
  const double* b2 = box_raw + prim2 * 6;
  bool ov = true;
#pragma unroll
  for (int k = 0; k < 3; ++k) ov = ov && xsub(b1[k], h) <= xadd(b2[3 + k], h) && xsub(b2[k], h) <= xadd(b1[3 + k], h);
  return ov;
}

// class-F width of a pair whose first stencil vertex is v0 (per member:
// dbar_min, or its component's with CB_DBAR_PER_COMPONENT)
__device__ __forceinline__ double member_f_width(const MemberParams& M, const unsigned long long* __restrict__ dbar_comp,
                                                 const int32_t* __restrict__ comp, int v0) {
  return M.per_comp ? __longlong_as_double((long long)dbar_comp[comp[v0]]) : M.dbar_min;
}

// class byte of a filtered candidate dropped by the per-stencil activation
constexpr uint8_t KL_DROPPED = 0xFE;

struct StencilArgs {
  const double* __restrict__ box_raw;            // null unless a member uses per-stencil activation
  const unsigned long long* __restrict__ dbar_comp;
  const int32_t* __restrict__ comp;
  unsigned long long* __restrict__ ndrop;
};

__global__ void k_filter_rod(int64_t nc, const uint64_t* __restrict__ cand, const int32_t* __restrict__ ev0,
                             const int32_t* __restrict__ comp, const int32_t* __restrict__ win,
                             const int32_t* __restrict__ wst, const int32_t* __restrict__ rloop,
                             const int32_t* __restrict__ vsc, const MemberParams* __restrict__ mp,
                             uint8_t* __restrict__ klass, unsigned long long* __restrict__ nfilt, StencilArgs SA) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t f = 0, dropped = 0;
  if (c < nc) {
    const uint64_t key = cand[c];
    const uint32_t k = cb_key_i(key), l = cb_key_j(key);
    const int v0 = ev0[k];
    const MemberParams& M = mp[vsc[v0]];
    const bool same = comp[v0] == comp[ev0[l]];
    f = (!M.filter_off && same && rod_filtered(win, wst, M.loops != 0, k, l)) ? 1u : 0u;
    // Kaldor culling: edges are numbered along each polyline, so the gap is
    // l - k (the shorter way round on a closed loop)
    uint8_t kl = (M.cull_radius > 0 && same && rod_gap(rloop, k, l) <= M.cull_radius) ? (uint8_t)3 : (uint8_t)f;
    if (kl == 1 && M.per_stencil &&
        !within_own_width(SA.box_raw, k, l, member_f_width(M, SA.dbar_comp, SA.comp, v0))) {
      kl = KL_DROPPED;
      f = 0;
      dropped = 1;
    }
    klass[c] = kl;
  }
  uint32_t b = __ballot_sync(0xffffffffu, f);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(nfilt, (unsigned long long)__popc(b));
  b = __ballot_sync(0xffffffffu, dropped);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(SA.ndrop, (unsigned long long)__popc(b));
}

__global__ void k_filter_shell(int64_t nc, const uint64_t* __restrict__ cand, const uint32_t* __restrict__ frest_j,
                               const uint32_t* __restrict__ row_pt, const uint32_t* __restrict__ row_ee, int64_t nf,
                               const int32_t* __restrict__ ev0, const int32_t* __restrict__ vsc,
                               const MemberParams* __restrict__ mp, uint8_t* __restrict__ klass,
                               unsigned long long* __restrict__ nfilt, int n, int T, StencilArgs SA) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t f = 0, dropped = 0;
  if (c < nc) {
    const uint64_t key = cand[c];
    const bool pt = cb_key_type(key) == CB_KEY_PT;
    const int v0 = pt ? (int)cb_key_i(key) : ev0[cb_key_i(key)];
    const MemberParams& M = mp[vsc[v0]];
    if (!M.filter_off && nf > 0) f = frest_contains(frest_j, row_pt, row_ee, key) ? 1u : 0u;
    uint8_t kl = (uint8_t)f;
    if (f && M.per_stencil) {
      // broad-phase primitive ids: vertices, then triangles, then edges
      const int64_t p1 = pt ? (int64_t)cb_key_i(key) : (int64_t)n + T + cb_key_i(key);
      const int64_t p2 = pt ? (int64_t)n + cb_key_j(key) : (int64_t)n + T + cb_key_j(key);
      if (!within_own_width(SA.box_raw, p1, p2, member_f_width(M, SA.dbar_comp, SA.comp, v0))) {
        kl = KL_DROPPED;
        f = 0;
        dropped = 1;
      }
    }
    klass[c] = kl;
  }
  uint32_t b = __ballot_sync(0xffffffffu, f);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(nfilt, (unsigned long long)__popc(b));
  b = __ballot_sync(0xffffffffu, dropped);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(SA.ndrop, (unsigned long long)__popc(b));
}

// per-stencil activation: keep flags of the candidates, then the kept ones
// (keys and classes) in their order
__global__ void k_keep_flag(int64_t nc, const uint8_t* __restrict__ klass, uint32_t* __restrict__ flag) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < nc) flag[c] = klass[c] != KL_DROPPED ? 1u : 0u;
}
__global__ void k_keep_write(int64_t nc, const uint64_t* __restrict__ cand, const uint8_t* __restrict__ klass,
                             const uint32_t* __restrict__ flag, const uint32_t* __restrict__ pos,
                             uint64_t* __restrict__ cand_out, uint8_t* __restrict__ klass_out) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < nc && flag[c]) {
    cand_out[pos[c]] = cand[c];
    klass_out[pos[c]] = klass[c];
  }
}

// ------------------------------------------------------------------ (c) ----

// Per-member sum of lane values: one atomic per warp when the warp holds one
// member (lanes without a value pass mem < 0), one per lane otherwise.  Every
// lane of the warp must call it.
__device__ __forceinline__ void member_energy_add(unsigned long long* __restrict__ macc, int mem, double e) {
  const int m0 = __shfl_sync(0xffffffffu, mem, 0);
  if (__all_sync(0xffffffffu, mem == m0 || mem < 0)) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0 && e != 0.0 && m0 >= 0)
      atomicAdd((double*)&macc[(size_t)m0 * MACC_STRIDE + MACC_E], e);
  } else if (mem >= 0 && e != 0.0) {
    atomicAdd((double*)&macc[(size_t)mem * MACC_STRIDE + MACC_E], e);
  }
}

// Warp-aggregated append of flagged lanes' values to a list.
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

// Warp-aggregated append from the end of a list of cap entries backwards.
__device__ __forceinline__ void warp_append_back(bool flag, uint32_t value, uint32_t* __restrict__ list,
                                                 int64_t cap, unsigned int* __restrict__ count) {
  const unsigned m = __ballot_sync(0xffffffffu, flag);
  if (!m) return;
  const unsigned lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  unsigned base = 0;
  if ((int)lane == leader) base = atomicAdd(count, (unsigned)__popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (flag) list[cap - 1 - (int64_t)(base + __popc(m & ((1u << lane) - 1u)))] = value;
}

// Per candidate, phase 1: an FP32 lower bound of the distance.  Candidates it
// places beyond every threshold of their class (U: a, which is above xi; F:
// dbar_min) are inactive and not class C.  The rest are queued for the exact
// FP64 phase, so that no warp pays for FP64 on behalf of a few lanes:
// point-triangle pairs from the start of the list (count nlist[0]), edge-edge
// pairs from its end backwards (count nlist[1]), so that the exact kernel's
// warps run one of the two distance routines.
__global__ void k_distance_screen(int64_t nc, const uint64_t* __restrict__ cand,
                                  const uint8_t* __restrict__ klass_in, const int32_t* __restrict__ ev0,
                                  const int32_t* __restrict__ ev1, const int32_t* __restrict__ tv, int T,
                                  const float4* __restrict__ xf, const double* __restrict__ cx,
                                  const int32_t* __restrict__ vsc, const MemberParams* __restrict__ mp, int n,
                                  double* __restrict__ dout, int8_t* __restrict__ tout, uint8_t* __restrict__ cls,
                                  uint32_t* __restrict__ flag, uint32_t* __restrict__ list,
                                  unsigned int* __restrict__ nlist) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool exact = false, ee = false;
  if (c < nc) {
    Stencil s = stencil_of(cand[c], ev0, ev1, tv, T);
    ee = s.ee;
    const int k = klass_in[c];
    const int mem = vsc[s.v[0]];
    const MemberParams& M = mp[mem];
    if (k == 3) {  // culled (Kaldor mode): no barrier, no distance needed
      dout[c] = __longlong_as_double(0x7ff0000000000000LL);
      tout[c] = -1;
      cls[c] = 3;
      flag[c] = 0;
      ee = false;
    } else {
      // thresholds beyond which a pair is surely inactive and not class C (the
      // 1e-9 margins cover the rounding of the FP64 decision; FP32 copies
      // rounded up, so the FP32 comparison is as safe)
      const float thr = k == 1 ? M.thrF32 : M.thrU32;
      const float X = (float)cx[4 * mem + 3];
      const float4 q0 = xf[s.v[0]], q1 = xf[s.v[1]], q2 = xf[s.v[2]], q3 = xf[s.v[3]];
      const float lb = cbb::lower_bound(s.ee, cbb::f3{q0.x, q0.y, q0.z}, cbb::f3{q1.x, q1.y, q1.z},
                                        cbb::f3{q2.x, q2.y, q2.z}, cbb::f3{q3.x, q3.y, q3.z}, X);
      if (lb >= thr) {
        dout[c] = __longlong_as_double(0x7ff0000000000000LL);
        tout[c] = -1;
        cls[c] = (uint8_t)k;
        flag[c] = 0;
      } else {
        exact = true;
      }
    }
  }
  warp_append(exact && !ee, (uint32_t)c, list, &nlist[0]);
  warp_append_back(exact && ee, (uint32_t)c, list, nc, &nlist[1]);
}

// phase 2: exact FP64 distance, class C and activity of the queued candidates
// (list entries [0, nlist[0]) and [cap - nlist[1], cap)).  With energy set
// (the energy-only pass), every active pair also adds kappa b(y) to its
// member's energy.
template <bool ENERGY>
__global__ void k_distance_exact(const uint32_t* __restrict__ list, int64_t cap, const unsigned int* __restrict__ nlist,
                                 const uint64_t* __restrict__ cand, const uint8_t* __restrict__ klass_in,
                                 const int32_t* __restrict__ ev0, const int32_t* __restrict__ ev1,
                                 const int32_t* __restrict__ tv, int T, const double* __restrict__ x, int n,
                                 const int32_t* __restrict__ vsc, const MemberParams* __restrict__ mp,
                                 double* __restrict__ dout, int8_t* __restrict__ tout,
                                 uint8_t* __restrict__ cls, uint32_t* __restrict__ flag,
                                 unsigned long long* __restrict__ status, unsigned long long* __restrict__ ncore,
                                 unsigned long long* __restrict__ macc, const int32_t* __restrict__ comp,
                                 const unsigned long long* __restrict__ dbar_comp, const double* __restrict__ elen2) {
  constexpr bool energy = ENERGY;  // energy only (barrier_energy): add kappa b per active pair
  const unsigned m0 = nlist[0], m = m0 + nlist[1];
  for (unsigned w = blockIdx.x * blockDim.x + threadIdx.x; w - threadIdx.x < m; w += gridDim.x * blockDim.x) {
    uint32_t is_core = 0;
    double e_local = 0.0;
    int e_mem = -1;
    if (w < m) {
      const uint32_t c = w < m0 ? list[w] : list[cap - 1 - (int64_t)(w - m0)];
      Stencil s = stencil_of(cand[c], ev0, ev1, tv, T);
      int k = klass_in[c];
      const int mem = vsc[s.v[0]];
      const PassParams P = member_pass(mp[mem]);
      double d;
      const int ty = cbg::stencil_distance(s.ee, load3(x, n, s.v[0]), load3(x, n, s.v[1]), load3(x, n, s.v[2]),
                                           load3(x, n, s.v[3]), d);
      if (k == 0 && P.core_temp && !P.single && d <= P.xi) k = 2;
      double xi_p, dh_p;
      pair_params(P, k, f_width(P, dbar_comp, comp, s.v[0]), xi_p, dh_p);
      const double y = xsub(d, xi_p);
      const uint32_t act = (y < dh_p) ? 1u : 0u;
      if (act && y <= 0.0) {
        atomicOr(status, (unsigned long long)CB_DEV_PENETRATION);
        atomicOr(&macc[(size_t)mem * MACC_STRIDE + MACC_STATUS], (unsigned long long)CB_DEV_PENETRATION);
      }
      dout[c] = d;
      tout[c] = (int8_t)ty;
      cls[c] = (uint8_t)k;
      flag[c] = act;
      is_core = (k == 2);
      if (energy && act && y > 0.0) {
        double mf = 1.0;
        if (P.mollify && s.ee) {  // IPC's edge-edge mollifier
          const double eps = 1e-3 * elen2[cb_key_i(cand[c])] * elen2[cb_key_j(cand[c])];
          double m1, m2;
          ee_mollifier(ee_cross2(load3(x, n, s.v[0]), load3(x, n, s.v[1]), load3(x, n, s.v[2]),
                                 load3(x, n, s.v[3])),
                       eps, mf, m1, m2);
        }
        e_local = P.kappa * mf * barrier_b(y, dh_p);
        e_mem = mem;
      }
    }
    if (energy) member_energy_add(macc, e_mem, e_local);
    const uint32_t b = __ballot_sync(0xffffffffu, is_core);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(ncore, (unsigned long long)__popc(b));
  }
}

// FP32 copy of a [3][n] FP64 vector, minus the member centre when cx is
// given, one float4 (x, y, z, 0) per vertex: the screens gather a vertex's
// three components in one 16-byte load
__global__ void k_to_f32(int n, const double* __restrict__ v, const double* __restrict__ cx,
                         const int32_t* __restrict__ vsc, float4* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double* c = cx ? cx + 4 * vsc[i] : nullptr;
  out[i] = make_float4((float)(v[i] - (c ? c[0] : 0.0)), (float)(v[(size_t)n + i] - (c ? c[1] : 0.0)),
                       (float)(v[2 * (size_t)n + i] - (c ? c[2] : 0.0)), 0.f);
}

__global__ void k_active_compact(int64_t nc, const uint32_t* __restrict__ flag, const uint32_t* __restrict__ pos,
                                 uint32_t* __restrict__ aidx) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < nc && flag[c]) aidx[pos[c]] = (uint32_t)c;
}

// ------------------------------------------------------------------ (d) ----

// 16 (row, col) block keys of each active stencil
// BSR pattern keys (row << bits_n | col) of the 16 blocks of every active
// stencil, made distinct within each run of BK_PAIRS active pairs (in
// candidate order, i.e. hash-cell order, a run shares most of its vertices:
// its 16 x 256 keys hold about a fifth as many distinct ones) through an
// open-addressing set in shared memory (linear probing, at most half full,
// each probe sequence bounded by the table size).  The distinct keys of each
// run are appended to bkey in no particular order -- the radix sort and the
// unique pass that follow make the pattern -- and their count to *m_out.
constexpr int BK_PAIRS = 256;
constexpr int BK_SLOTS = 8192;  // 2 x 16 keys x BK_PAIRS

__global__ void __launch_bounds__(BK_PAIRS) k_block_keys(int64_t na, const uint32_t* __restrict__ aidx,
                                                         const uint64_t* __restrict__ cand,
                                                         const int32_t* __restrict__ ev0,
                                                         const int32_t* __restrict__ ev1,
                                                         const int32_t* __restrict__ tv, int T, int bits_n,
                                                         uint64_t* __restrict__ bkey, unsigned int* __restrict__ m_out) {
  extern __shared__ unsigned long long tab[];  // BK_SLOTS
  __shared__ unsigned int wsum[BK_PAIRS / 32];
  __shared__ unsigned int base;
  constexpr unsigned long long EMPTY = ~0ull;  // no key: rows and columns are below 2^31
  const int tid = threadIdx.x;
  for (int k = tid; k < BK_SLOTS; k += BK_PAIRS) tab[k] = EMPTY;
  __syncthreads();
  const int64_t a = (int64_t)blockIdx.x * BK_PAIRS + tid;
  if (a < na) {
    const Stencil s = stencil_of(cand[aidx[a]], ev0, ev1, tv, T);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const unsigned long long key = ((unsigned long long)s.v[i] << bits_n) | (unsigned long long)s.v[j];
        // Fibonacci hashing (multiplicative, Knuth): the top bits of key x 2^64/phi
        unsigned h = (unsigned)((key * 0x9E3779B97F4A7C15ull) >> 51);
        for (int probe = 0; probe < BK_SLOTS; ++probe) {
          const unsigned long long prev = atomicCAS(&tab[h], EMPTY, key);
          if (prev == EMPTY || prev == key) break;
          h = (h + 1) & (BK_SLOTS - 1);
        }
      }
  }
  __syncthreads();
  // compaction: thread tid owns slots [tid * 32, tid * 32 + 32)
  constexpr int PER = BK_SLOTS / BK_PAIRS;
  unsigned c = 0;
#pragma unroll
  for (int k = 0; k < PER; ++k) c += tab[tid * PER + k] != EMPTY;
  const unsigned lane = tid & 31, wid = tid >> 5;
  unsigned incl = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
    if ((int)lane >= o) incl += v;
  }
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  unsigned woff = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < BK_PAIRS / 32; ++w) {
    woff += (w < (int)wid) ? wsum[w] : 0u;
    tot += wsum[w];
  }
  if (tid == 0) base = tot ? atomicAdd(m_out, tot) : 0u;
  __syncthreads();
  size_t pos = (size_t)base + woff + incl - c;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const unsigned long long key = tab[tid * PER + k];
    if (key != EMPTY) bkey[pos++] = key;
  }
}

__global__ void k_unique_flag(int64_t m, const uint64_t* __restrict__ k, uint32_t* __restrict__ flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) flag[i] = (i == 0 || k[i] != k[i - 1]) ? 1u : 0u;
}

__global__ void k_unique_write(int64_t m, const uint64_t* __restrict__ k, const uint32_t* __restrict__ flag,
                               const uint32_t* __restrict__ pos, int bits_n, int32_t* __restrict__ col,
                               uint32_t* __restrict__ row_cnt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m || !flag[i]) return;
  const uint64_t key = k[i];
  col[pos[i]] = (int32_t)(key & ((1ull << bits_n) - 1ull));
  atomicAdd(&row_cnt[key >> bits_n], 1u);
}

// --- analytic derivatives of the squared distance in relative variables ---
// z_m = sum_i C[m][i] x_i (m < nz) with C rows summing to zero.
//   PP:    z0 = b - a                       s = |z0|^2
//   PE:    z0 = w = q - e0, z1 = u = e1-e0  s = |w|^2 - (w.u)^2/|u|^2
//   plane: z0 = w, z1 = u, z2 = v           s = (w.(u x v))^2 / |u x v|^2
// (point-triangle face: w = p-t0, u = t1-t0, v = t2-t0; edge-edge interior:
//  w = b0-a0, u = a1-a0, v = b1-b0.)
struct TypeInfo {
  int8_t kind;   // 0 PP, 1 PE, 2 plane
  int8_t C[3][4];
};

__constant__ TypeInfo c_pt_types[7] = {
    {0, {{-1, 1, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}}},
    {0, {{-1, 0, 1, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}}},
    {0, {{-1, 0, 0, 1}, {0, 0, 0, 0}, {0, 0, 0, 0}}},
    {1, {{1, -1, 0, 0}, {0, -1, 1, 0}, {0, 0, 0, 0}}},
    {1, {{1, 0, -1, 0}, {0, 0, -1, 1}, {0, 0, 0, 0}}},
    {1, {{1, 0, 0, -1}, {0, 1, 0, -1}, {0, 0, 0, 0}}},
    {2, {{1, -1, 0, 0}, {0, -1, 1, 0}, {0, -1, 0, 1}}},
};
__constant__ TypeInfo c_ee_types[9] = {
    {0, {{-1, 0, 1, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}}},
    {0, {{-1, 0, 0, 1}, {0, 0, 0, 0}, {0, 0, 0, 0}}},
    {0, {{0, -1, 1, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}}},
    {0, {{0, -1, 0, 1}, {0, 0, 0, 0}, {0, 0, 0, 0}}},
    {1, {{1, 0, -1, 0}, {0, 0, -1, 1}, {0, 0, 0, 0}}},
    {1, {{0, 1, -1, 0}, {0, 0, -1, 1}, {0, 0, 0, 0}}},
    {1, {{-1, 0, 1, 0}, {-1, 1, 0, 0}, {0, 0, 0, 0}}},
    {1, {{-1, 0, 0, 1}, {-1, 1, 0, 0}, {0, 0, 0, 0}}},
    {2, {{-1, 0, 1, 0}, {-1, 1, 0, 0}, {0, 0, -1, 1}}},
};

// Orthonormal bases of the complement of rigid translations of the points a
// stencil type involves: K4[i][a] for 4 points (entries +-1/2), K3 for 3.
__constant__ double c_K4[4][3] = {{0.5, 0.5, 0.5}, {0.5, -0.5, -0.5}, {-0.5, 0.5, -0.5}, {-0.5, -0.5, 0.5}};
__constant__ double c_K3[3][2] = {{0.70710678118654752440, 0.40824829046386301637},
                                  {-0.70710678118654752440, 0.40824829046386301637},
                                  {0.0, -0.81649658092772603273}};

__host__ __device__ __forceinline__ int tri_idx(int i, int j, int D) {  // packed upper triangle, i <= j
  return i * D - (i * (i - 1)) / 2 + (j - i);
}

__host__ __device__ __forceinline__ double& zh(double* H, int r, int c) { return H[r * 9 + c]; }

// gradient gs[9] and Hessian Hs[81] (row-major, 3x3 blocks of z) of s
__host__ __device__ void s_derivs(int kind, const d3* z, double* gs, double* Hs) {
  for (int i = 0; i < 81; ++i) Hs[i] = 0.0;
  for (int i = 0; i < 9; ++i) gs[i] = 0.0;
  if (kind == 0) {
    gs[0] = 2.0 * z[0].x;
    gs[1] = 2.0 * z[0].y;
    gs[2] = 2.0 * z[0].z;
    zh(Hs, 0, 0) = zh(Hs, 1, 1) = zh(Hs, 2, 2) = 2.0;
    return;
  }
  if (kind == 1) {
    const double w[3] = {z[0].x, z[0].y, z[0].z}, u[3] = {z[1].x, z[1].y, z[1].z};
    const double al = w[0] * u[0] + w[1] * u[1] + w[2] * u[2];
    const double be = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const double ibe = 1.0 / be;  // one division; the rest multiply
    const double ga = al * ibe;
    for (int k = 0; k < 3; ++k) {
      gs[k] = 2.0 * w[k] - 2.0 * ga * u[k];
      gs[3 + k] = -2.0 * ga * w[k] + 2.0 * ga * ga * u[k];
    }
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        const double dij = (i == j) ? 1.0 : 0.0;
        const double ww = 2.0 * dij - 2.0 * u[i] * u[j] * ibe;
        const double wu = -2.0 * u[i] * w[j] * ibe - 2.0 * ga * dij + 4.0 * ga * u[i] * u[j] * ibe;
        const double uu = -2.0 * w[i] * w[j] * ibe + 4.0 * ga * (w[i] * u[j] + u[i] * w[j]) * ibe +
                          2.0 * ga * ga * dij - 8.0 * ga * ga * u[i] * u[j] * ibe;
        zh(Hs, i, j) = ww;
        zh(Hs, i, 3 + j) = wu;
        zh(Hs, 3 + j, i) = wu;
        zh(Hs, 3 + i, 3 + j) = uu;
      }
    return;
  }
  // plane: s = g^2 / N, g = w.(u x v), N = |u x v|^2
  const d3 w = z[0], u = z[1], v = z[2];
  const double nx = u.y * v.z - u.z * v.y, ny = u.z * v.x - u.x * v.z, nz = u.x * v.y - u.y * v.x;
  const double g = w.x * nx + w.y * ny + w.z * nz;
  const double uu = u.x * u.x + u.y * u.y + u.z * u.z;
  const double vv = v.x * v.x + v.y * v.y + v.z * v.z;
  const double uv = u.x * v.x + u.y * v.y + u.z * v.z;
  const double N = nx * nx + ny * ny + nz * nz;
  // grad g: (n, v x w, w x u)
  double gg[9] = {nx,
                  ny,
                  nz,
                  v.y * w.z - v.z * w.y,
                  v.z * w.x - v.x * w.z,
                  v.x * w.y - v.y * w.x,
                  w.y * u.z - w.z * u.y,
                  w.z * u.x - w.x * u.z,
                  w.x * u.y - w.y * u.x};
  // grad N: (0, 2 vv u - 2 uv v, 2 uu v - 2 uv u)
  const double ua[3] = {u.x, u.y, u.z}, va[3] = {v.x, v.y, v.z}, wa[3] = {w.x, w.y, w.z};
  double gN[9];
  for (int k = 0; k < 3; ++k) {
    gN[k] = 0.0;
    gN[3 + k] = 2.0 * vv * ua[k] - 2.0 * uv * va[k];
    gN[6 + k] = 2.0 * uu * va[k] - 2.0 * uv * ua[k];
  }
  const double iN = 1.0 / N;
  const double a1 = 2.0 * g * iN, a2 = g * g * iN * iN;
  for (int k = 0; k < 9; ++k) gs[k] = a1 * gg[k] - a2 * gN[k];
  // Hessian
  const double c_gg = 2.0 * iN;              // grad g grad g^T
  const double c_hg = 2.0 * g * iN;          // hess g
  const double c_gN = -2.0 * g * iN * iN;    // (grad g grad N^T + grad N grad g^T)
  const double c_hN = -g * g * iN * iN;      // hess N
  const double c_NN = 2.0 * g * g * iN * iN * iN;  // grad N grad N^T
  for (int r = 0; r < 9; ++r)
    for (int c = 0; c < 9; ++c)
      Hs[r * 9 + c] = c_gg * gg[r] * gg[c] + c_gN * (gg[r] * gN[c] + gN[r] * gg[c]) + c_NN * gN[r] * gN[c];
  // hess g: blocks (w,u) = -[v]x, (w,v) = [u]x, (u,v) = -[w]x and transposes
  auto skew_add = [&](int rb, int cb, const double* a, double sc) {
    // adds sc * [a]x to block (rb, cb) and sc * [a]x^T to block (cb, rb)
    const double m[3][3] = {{0.0, -a[2], a[1]}, {a[2], 0.0, -a[0]}, {-a[1], a[0], 0.0}};
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        Hs[(3 * rb + i) * 9 + 3 * cb + j] += sc * m[i][j];
        Hs[(3 * cb + j) * 9 + 3 * rb + i] += sc * m[i][j];
      }
  };
  skew_add(0, 1, va, -c_hg);
  skew_add(0, 2, ua, c_hg);
  skew_add(1, 2, wa, -c_hg);
  // hess N: (u,u) 2 vv I - 2 v v^T ; (v,v) 2 uu I - 2 u u^T ; (u,v) 4 u v^T - 2 v u^T - 2 uv I
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const double dij = (i == j) ? 1.0 : 0.0;
      Hs[(3 + i) * 9 + 3 + j] += c_hN * (2.0 * vv * dij - 2.0 * va[i] * va[j]);
      Hs[(6 + i) * 9 + 6 + j] += c_hN * (2.0 * uu * dij - 2.0 * ua[i] * ua[j]);
      const double uvb = c_hN * (4.0 * ua[i] * va[j] - 2.0 * va[i] * ua[j] - 2.0 * uv * dij);
      Hs[(3 + i) * 9 + 6 + j] += uvb;
      Hs[(6 + j) * 9 + 3 + i] += uvb;
    }
}

// Reduced barrier Hessian of a plane-type pair (point-triangle face,
// edge-edge interior) in the translation-free coordinates y of its four
// points, z = (M x I) y, differentiating the distance itself:
//   d = |g| / sqrt(N),  g = w.(u x v),  N = |n|^2,  n = u x v,
//   grad d = sg gam (grad g - h grad N),  gam = 1/sqrt(N), h = g / (2N), sg = sign g,
//   hess d = sg gam (hess g - h hess N - (grad g grad N^T + grad N grad g^T) / (2N)
//                    + (3h / (2N)) grad N grad N^T),
//   B = kappa b'' grad d grad d^T + kappa b' hess d.
// (Through s = d^2 instead, B = (b'' - b'/d) grad d grad d^T + b'/(2d) hess s
// adds and then cancels a term of order |grad g|^2 / N, which for
// near-parallel edges or slender triangles costs about 1/sin of the angle
// in digits.)  With q_b = M[2][b] u - M[1][b] v (so dn/dy_b = [q_b]x):
//   grad_y g = (M^T x I) grad_z g,   grad_y N = (M^T x I) grad_z N,
//   hess_y g, block (a,b) = [r_ab]x,
//     r_ab = -(M0a M1b - M1a M0b) v + (M0a M2b - M2a M0b) u - (M1a M2b - M2a M1b) w,
//   hess_y N, block (a,b) = 2 (q_a.q_b) I - 2 q_b q_a^T + 2 (M2a M1b - M1a M2b) [n]x.
// With e = grad_y g - h grad_y N the rank-one part is
//   kappa b'' gam^2 e e^T - (s1 / 2N)(e gN^T + gN e^T) + (h s1 / 2N) gN gN^T,
// s1 = kappa b' sg gam, gN = grad_y N.  Writes grad_z d (gd, 9) and the
// packed upper triangle of B (Bq, 45); kb1 = kappa b', kb2 = kappa b''.
__host__ __device__ __forceinline__ void plane_reduced(const double (&z)[3][3], const double (&M)[3][3], double kb1,
                                                       double kb2, double (&gd)[9], double (&Bq)[45]) {
  const double* w = z[0];
  const double* u = z[1];
  const double* v = z[2];
  const double n[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
  const double g = w[0] * n[0] + w[1] * n[1] + w[2] * n[2];
  const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const double vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  const double uv = u[0] * v[0] + u[1] * v[1] + u[2] * v[2];
  const double N = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
  const double gam = 1.0 / sqrt(N), iN = gam * gam;
  const double sg = g >= 0.0 ? 1.0 : -1.0;
  const double h = 0.5 * g * iN;
  // z-space gradients of g and N: (n, v x w, w x u) and (0, 2 vv u - 2 uv v, 2 uu v - 2 uv u)
  const double gg[3][3] = {{n[0], n[1], n[2]},
                           {v[1] * w[2] - v[2] * w[1], v[2] * w[0] - v[0] * w[2], v[0] * w[1] - v[1] * w[0]},
                           {w[1] * u[2] - w[2] * u[1], w[2] * u[0] - w[0] * u[2], w[0] * u[1] - w[1] * u[0]}};
  double gN[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    gN[0][k] = 0.0;
    gN[1][k] = 2.0 * vv * u[k] - 2.0 * uv * v[k];
    gN[2][k] = 2.0 * uu * v[k] - 2.0 * uv * u[k];
  }
  const double sgam = sg * gam;
#pragma unroll
  for (int m = 0; m < 3; ++m)
#pragma unroll
    for (int k = 0; k < 3; ++k) gd[3 * m + k] = sgam * (gg[m][k] - h * gN[m][k]);
  // y-space vectors
  double e[3][3], gNY[3][3], q[3][3];
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      gNY[b][k] = M[1][b] * gN[1][k] + M[2][b] * gN[2][k];
      e[b][k] = M[0][b] * gg[0][k] + M[1][b] * gg[1][k] + M[2][b] * gg[2][k] - h * gNY[b][k];
      q[b][k] = M[2][b] * u[k] - M[1][b] * v[k];
    }
  const double s1 = kb1 * sgam;
  const double A1 = kb2 * iN, B1 = -0.5 * s1 * iN, C1 = 0.5 * h * s1 * iN;
  const double kN = -2.0 * s1 * h;  // times hess N / 2
  const double kg = s1;             // times hess g
  double U[3][3], W[3][3];
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      U[b][k] = A1 * e[b][k] + B1 * gNY[b][k];
      W[b][k] = B1 * e[b][k] + C1 * gNY[b][k];
    }
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = a; b < 3; ++b) {
      const double G = q[a][0] * q[b][0] + q[a][1] * q[b][1] + q[a][2] * q[b][2];
      double X[3][3];  // [r]x part of the off-diagonal blocks
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) X[i][j] = 0.0;
      if (a < b) {
        const double mu = M[2][a] * M[1][b] - M[1][a] * M[2][b];
        const double m01 = M[0][a] * M[1][b] - M[1][a] * M[0][b];
        const double m02 = M[0][a] * M[2][b] - M[2][a] * M[0][b];
        const double m12 = M[1][a] * M[2][b] - M[2][a] * M[1][b];
        double r[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) r[k] = kg * (m02 * u[k] - m01 * v[k] - m12 * w[k]) + kN * mu * n[k];
        X[0][1] = -r[2];
        X[0][2] = r[1];
        X[1][0] = r[2];
        X[1][2] = -r[0];
        X[2][0] = -r[1];
        X[2][1] = r[0];
      }
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = (a == b ? i : 0); j < 3; ++j) {
          double val = e[a][i] * U[b][j] + gNY[a][i] * W[b][j] - kN * q[b][i] * q[a][j] + X[i][j];
          if (i == j) val += kN * G;
          Bq[tri_idx(3 * a + i, 3 * b + j, 9)] = val;
        }
    }
}

__device__ __forceinline__ int64_t find_block(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                              int r, int c) {
  int lo = row_ptr[r], hi = row_ptr[r + 1];
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (col[mid] < c) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

struct HessArgs {
  int64_t na;
  const uint32_t* __restrict__ order;  // prep thread -> active pair index
  const uint32_t* __restrict__ aidx;
  const uint64_t* __restrict__ cand;
  const double* __restrict__ cd;
  const int8_t* __restrict__ ctype;
  const uint8_t* __restrict__ ccls;
  const int32_t* __restrict__ ev0;
  const int32_t* __restrict__ ev1;
  const int32_t* __restrict__ tv;
  int T;
  const double* __restrict__ x;
  int n;
  const int32_t* __restrict__ vsc;
  const MemberParams* __restrict__ mp;
  unsigned long long* __restrict__ macc;
  const int32_t* __restrict__ comp;                 // component label per vertex
  const unsigned long long* __restrict__ dbar_comp; // per-component dbar_min bits (CB_DBAR_PER_COMPONENT)
  const int32_t* __restrict__ row_ptr;
  const int32_t* __restrict__ col;
  double* __restrict__ val;
  double* __restrict__ grad;
  unsigned long long* __restrict__ status;
  // reduced matrices handed to the projection kernels: B packed upper
  // triangle, element-major ([e * cap + slot]); slot -> active pair index
  double* __restrict__ B9;
  double* __restrict__ B6;
  double* __restrict__ B4;        // point-edge pairs in their own frame: p, r, Y (7), 2x2 (3), frame (9)
  uint32_t* __restrict__ slot9;
  uint32_t* __restrict__ slot6;
  uint32_t* __restrict__ slot4;
  unsigned int* __restrict__ n9;
  unsigned int* __restrict__ n6;
  unsigned int* __restrict__ n4;
  int64_t cap;
  // CB_EE_MOLLIFIER: pairs handled by k_moll_hess (hmoll null: none)
  const uint8_t* __restrict__ hmoll;
  const uint32_t* __restrict__ mlist;
  const unsigned* __restrict__ nmoll;
  const double* __restrict__ elen2;
};


__device__ __forceinline__ void add_block(const HessArgs& A, int r, int c, const double* blk, bool transpose) {
  const int64_t bi = find_block(A.row_ptr, A.col, r, c);
  if (bi >= A.row_ptr[r + 1] || A.col[bi] != c) {
    atomicOr(A.status, (unsigned long long)CB_DEV_CAPACITY);  // pattern miss: never expected
    return;
  }
  double* dst = A.val + 9 * bi;
  for (int al = 0; al < 3; ++al)
    for (int be = 0; be < 3; ++be) atomicAdd(&dst[3 * al + be], transpose ? blk[3 * be + al] : blk[3 * al + be]);
}

// The reduced matrix of one pair, B = c1 gB gB^T + c2 (M x I)^T hess s (M x I)
// with gB = (M x I)^T grad d, written as a packed upper triangle into the
// queue (element-major: entry e of slot at e * cap + slot).  D = 9 goes with
// three z-vectors (plane types), D = 6 with two (point-edge).
template <int D, int NZ>
__host__ __device__ __forceinline__ void write_reduced(double* __restrict__ Bo, int64_t cap, unsigned slot,
                                              const double (&M)[3][3], const double* gd, const double* Hs,
                                              double c1, double c2) {
  constexpr int NB = D / 3;
  double gB[D];
#pragma unroll
  for (int ab = 0; ab < NB; ++ab)
#pragma unroll
    for (int al = 0; al < 3; ++al) {
      double v = 0.0;
#pragma unroll
      for (int m = 0; m < NZ; ++m) v += M[m][ab] * gd[3 * m + al];
      gB[3 * ab + al] = v;
    }
#pragma unroll
  for (int row = 0; row < D; ++row) {
    const int ab = row / 3, al = row % 3;
#pragma unroll
    for (int col = row; col < D; ++col) {
      const int bb = col / 3, be = col % 3;
      double h = 0.0;
#pragma unroll
      for (int m = 0; m < NZ; ++m) {
        double hm = 0.0;
#pragma unroll
        for (int m2 = 0; m2 < NZ; ++m2) hm += M[m2][bb] * Hs[(3 * m + al) * 9 + 3 * m2 + be];
        h += M[m][ab] * hm;
      }
      Bo[(size_t)tri_idx(row, col, D) * cap + slot] = c1 * gB[row] * gB[col] + c2 * h;
    }
  }
}

// Point-edge pairs in their own frame: the 6x6 reduced matrix (rows 3 ab + al,
// al the local axis) has no coupling between the e3 rows (2, 5) and the
// rest, so it splits into an in-plane 4x4 block (rows 0, 1, 3, 4) and an
// out-of-plane 2x2 block (rows 2, 5).
// At w' = (wx, wy, 0), u' = (lu, 0, 0) the Hessian of s = |w|^2 - (w.u)^2/|u|^2
// has, per pair of axes, these 2x2 blocks over (w, u) (rows: first axis):
//   (x, x): 0;  (x, y): [[0, -2 wy/lu], [0, 2 wx wy/lu^2]];  (y, x): its transpose;
//   (y, y): [[2, -2 wx/lu], [-2 wx/lu, 2 (wx^2 - wy^2)/lu^2]];
//   (z, z): [[2, -2 wx/lu], [-2 wx/lu, 2 wx^2/lu^2]];  the rest 0,
// and grad d = (g0, g1) on the y axis only.  With H_z = c1 grad d grad d^T +
// c2 hess s, block (ab, al; bb, be) of B is (M^T H_z[al, be] M)[ab][bb].  So
// the 4x4 block, in the order (x of both reduced points, y of both), is
//   [[0, p r^T], [r p^T, Y]],  p_ab = M[0][ab] hxy01 + M[1][ab] hxy11,
//   r_bb = M[1][bb],  Y = (M^T H_z[y, y] M)
// (the (x, x) block is zero and the (x, y) block has rank one).  Queued:
// p (2), r (2), Y (3, packed), the 2x2 block (3, packed) and the frame R
// (row-major, columns e1 e2 e3; 9).  il = 1 / lu.
__device__ __forceinline__ void write_reduced_pe_local(double* __restrict__ Bo, int64_t cap, unsigned slot,
                                                       const double (&M)[3][3], double g0, double g1, double wx,
                                                       double wy, double il, double c1, double c2,
                                                       const double (&Rf)[9]) {
  const double hxy01 = c2 * (-2.0 * wy * il), hxy11 = c2 * (2.0 * wx * wy * il * il);
  const double hwu = -2.0 * wx * il;
  const double Hyy[2][2] = {{c1 * g0 * g0 + 2.0 * c2, c1 * g0 * g1 + c2 * hwu},
                            {c1 * g0 * g1 + c2 * hwu, c1 * g1 * g1 + c2 * 2.0 * (wx * wx - wy * wy) * il * il}};
  const double Hzz[2][2] = {{2.0 * c2, c2 * hwu}, {c2 * hwu, c2 * 2.0 * wx * wx * il * il}};
  auto mhm = [&](const double (&H)[2][2], int ab, int bb) {
    double v = 0.0;
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
      for (int m2 = 0; m2 < 2; ++m2) v += M[m][ab] * H[m][m2] * M[m2][bb];
    return v;
  };
  const double e[10] = {M[0][0] * hxy01 + M[1][0] * hxy11,
                        M[0][1] * hxy01 + M[1][1] * hxy11,
                        M[1][0],
                        M[1][1],
                        mhm(Hyy, 0, 0),
                        mhm(Hyy, 0, 1),
                        mhm(Hyy, 1, 1),
                        mhm(Hzz, 0, 0),
                        mhm(Hzz, 0, 1),
                        mhm(Hzz, 1, 1)};
#pragma unroll
  for (int k = 0; k < 10; ++k) Bo[(size_t)k * cap + slot] = e[k];
#pragma unroll
  for (int k = 0; k < 9; ++k) Bo[(size_t)(10 + k) * cap + slot] = Rf[k];
}

// Active pairs in the order k_hess_prep takes them: face / line-line pairs
// (the branch with the most FP64 work) first, the other pairs from the end
// backwards, so that a warp of the prep kernel runs one branch rather than
// both with few lanes each.  Warp-aggregated appends; inside each group the
// order follows warp arrival.
struct MollArgs {                   // CB_EE_MOLLIFIER scenes only (mp null: no mollifier)
  const double* __restrict__ x;
  int n;
  const int32_t* __restrict__ ev0;
  const int32_t* __restrict__ ev1;
  const int32_t* __restrict__ vsc;
  const MemberParams* __restrict__ mp;
  const double* __restrict__ elen2;
  uint8_t* __restrict__ hmoll;       // [na] 1: mollified edge-edge pair
  uint32_t* __restrict__ mlist;      // their active indices
  unsigned* __restrict__ nmoll;
};

__global__ void k_kind_split(int64_t na, const uint32_t* __restrict__ aidx, const uint64_t* __restrict__ cand,
                             const int8_t* __restrict__ ctype, uint32_t* __restrict__ order,
                             unsigned* __restrict__ cnt, MollArgs MA) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool plane = false, moll = false;
  if (a < na) {
    const uint32_t c = aidx[a];
    const int ty = ctype[c];
    const uint64_t key = cand[c];
    plane = (cb_key_type(key) == CB_KEY_PT ? c_pt_types[ty] : c_ee_types[ty]).kind == 2;
    if (MA.mp && cb_key_type(key) != CB_KEY_PT) {
      // edge-edge pair below its mollifier threshold: its energy, gradient
      // and 9x9 matrix come from k_moll_hess instead of k_hess_prep
      const uint32_t i = cb_key_i(key), j = cb_key_j(key);
      const int a0 = MA.ev0[i], a1 = MA.ev1[i], b0 = MA.ev0[j], b1 = MA.ev1[j];
      if (MA.mp[MA.vsc[a0]].mollify) {
        const double c2 = ee_cross2(load3(MA.x, MA.n, a0), load3(MA.x, MA.n, a1), load3(MA.x, MA.n, b0),
                                    load3(MA.x, MA.n, b1));
        moll = c2 < 1e-3 * MA.elen2[i] * MA.elen2[j];
      }
    }
    if (MA.mp) MA.hmoll[a] = moll ? 1 : 0;
  }
  if (MA.mp) warp_append(moll, (uint32_t)a, MA.mlist, MA.nmoll);
  const unsigned lane = threadIdx.x & 31, lt = (1u << lane) - 1u;
  const unsigned mp = __ballot_sync(0xffffffffu, a < na && plane);
  const unsigned mr = __ballot_sync(0xffffffffu, a < na && !plane);
  unsigned bp = 0, br = 0;
  if (lane == 0) {
    if (mp) bp = atomicAdd(&cnt[0], (unsigned)__popc(mp));
    if (mr) br = atomicAdd(&cnt[1], (unsigned)__popc(mr));
  }
  bp = __shfl_sync(0xffffffffu, bp, 0);
  br = __shfl_sync(0xffffffffu, br, 0);
  if (a < na) {
    if (plane) order[bp + __popc(mp & lt)] = (uint32_t)a;
    else order[na - 1 - (int64_t)(br + __popc(mr & lt))] = (uint32_t)a;
  }
}

// Stage (d), part 1, one thread per active pair: barrier value and
// derivatives, energy, gradient scatter, and the Hessian in the orthonormal
// translation-free basis of the points the distance type involves,
// B = (M x I)^T H_z (M x I) with M = C K.  Point-point stencils are projected
// in closed form here; the others are queued for the projection kernels.
__global__ void __launch_bounds__(128) k_hess_prep(HessArgs A) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t a = t < A.na ? (int64_t)A.order[t] : A.na;
  if (A.hmoll && a < A.na && A.hmoll[a]) a = A.na;  // mollified edge-edge pair: k_moll_hess
  double e_local = 0.0;
  int mem = -1;
  int want = 0;  // 9 or 6: reduced dimension of the queued matrix
  // the reduced matrix (packed upper triangle), written once the queue slot is known
  double Bq[45];
  double gd[9], M[3][3], Rf[9];
  double c1 = 0.0, c2 = 0.0;
  int nz = 0;
  if (a < A.na) {
    const uint32_t c = A.aidx[a];
    const uint64_t key = A.cand[c];
    Stencil s = stencil_of(key, A.ev0, A.ev1, A.tv, A.T);
    const int ty = A.ctype[c];
    const TypeInfo& TI = s.ee ? c_ee_types[ty] : c_pt_types[ty];
    const int kind = TI.kind;
    nz = kind + 1;
    d3 X[4];
    for (int i = 0; i < 4; ++i) X[i] = load3(A.x, A.n, s.v[i]);
    d3 Pl[4];
    for (int i = 0; i < 4; ++i) Pl[i] = mk3(X[i].x - X[0].x, X[i].y - X[0].y, X[i].z - X[0].z);
    d3 z[3];
    for (int m = 0; m < 3; ++m) {
      double zx = 0, zy = 0, zz = 0;
      for (int i = 1; i < 4; ++i) {
        const double cm = (double)TI.C[m][i];
        zx += cm * Pl[i].x;
        zy += cm * Pl[i].y;
        zz += cm * Pl[i].z;
      }
      z[m] = mk3(zx, zy, zz);
    }
    const double d = A.cd[c];
    mem = A.vsc[s.v[0]];
    const PassParams P = member_pass(A.mp[mem]);
    double xi_p, dh_p;
    pair_params(P, A.ccls[c], f_width(P, A.dbar_comp, A.comp, s.v[0]), xi_p, dh_p);
    const double y = d - xi_p;
    double b, b1, b2;
    barrier_b012(y, dh_p, b, b1, b2);
    const double kap = P.kappa;
    e_local = kap * b;
    // Point-edge: in the frame e1 along the edge (u), e3 normal to the plane
    // of the edge and the point (u x w), the configuration is symmetric under
    // e3 -> -e3, so hess s and grad d have no coupling between the e3
    // components and the others: the reduced matrix splits into an in-plane
    // 4x4 and an out-of-plane 2x2 block.  Evaluated at the local coordinates
    // w' = (w.e1, w.e2, 0), u' = (|u|, 0, 0) the coupling entries are exactly
    // zero.  The frame's direction error is about 1e-16 |w| |u| / |u x w|;
    // beyond a ratio of 64 the pair stays on the generic 6x6 path.
    bool pe_local = false;
    d3 zl[3];
    double piu = 0.0;  // 1 / |u| of a point-edge pair in its frame
    if (kind == 1) {
      const d3 w = z[0], u = z[1];
      const d3 n = mk3(u.y * w.z - u.z * w.y, u.z * w.x - u.x * w.z, u.x * w.y - u.y * w.x);
      // squared lengths; the conditioning test |w||u| <= 64 |u x w| squared
      const double nn2 = n.x * n.x + n.y * n.y + n.z * n.z;
      const double uu2 = u.x * u.x + u.y * u.y + u.z * u.z;
      const double ww2 = w.x * w.x + w.y * w.y + w.z * w.z;
      if (nn2 > 0.0 && ww2 * uu2 <= 4096.0 * nn2) {
        const double iu = rsqrt(uu2), inn = rsqrt(nn2), lu = uu2 * iu;
        piu = iu;
        const d3 e1 = mk3(u.x * iu, u.y * iu, u.z * iu), e3 = mk3(n.x * inn, n.y * inn, n.z * inn);
        const d3 e2 = mk3(e3.y * e1.z - e3.z * e1.y, e3.z * e1.x - e3.x * e1.z, e3.x * e1.y - e3.y * e1.x);
        zl[0] = mk3(w.x * e1.x + w.y * e1.y + w.z * e1.z, w.x * e2.x + w.y * e2.y + w.z * e2.z, 0.0);
        zl[1] = mk3(lu, 0.0, 0.0);
        zl[2] = mk3(0.0, 0.0, 0.0);
        Rf[0] = e1.x; Rf[1] = e2.x; Rf[2] = e3.x;
        Rf[3] = e1.y; Rf[4] = e2.y; Rf[5] = e3.y;
        Rf[6] = e1.z; Rf[7] = e2.z; Rf[8] = e3.z;
        pe_local = true;
      }
    }
    const double i2d = 0.5 / d;
    c1 = kap * (b2 - b1 * (2.0 * i2d));
    c2 = kap * b1 * i2d;
    if (kind > 0) {
      // M = C K: the z-vectors in the orthonormal translation-free basis of
      // the points the type involves
      int pts[4], np = 0;
      for (int i = 0; i < 4; ++i) {
        bool used = false;
        for (int m = 0; m < nz; ++m) used |= TI.C[m][i] != 0;
        if (used) pts[np++] = i;
      }
      const int nb = np - 1;
      for (int m = 0; m < 3; ++m)
        for (int bb = 0; bb < 3; ++bb) {
          double v = 0.0;
          if (m < nz && bb < nb)
            for (int q = 0; q < np; ++q)
              v += (double)TI.C[m][pts[q]] * (np == 4 ? c_K4[q][bb] : c_K3[q][bb]);
          M[m][bb] = v;
        }
    }
    if (pe_local) {
      // In the frame (w' = (wx, wy, 0), u' = (lu, 0, 0), s = wy^2) grad s has
      // only the y components 2 wy (w) and -2 wx wy / lu (u); hess s is
      // formed in write_reduced_pe_local
      const double pwx = zl[0].x, pwy = zl[0].y;
      for (int k = 0; k < 9; ++k) gd[k] = 0.0;
      gd[1] = 2.0 * pwy * i2d;
      gd[4] = -2.0 * pwx * pwy * piu * i2d;
      write_reduced_pe_local(Bq, 1, 0, M, gd[1], gd[4], pwx, pwy, piu, c1, c2, Rf);
      want = 4;
    } else if (kind == 2) {
      const double zz[3][3] = {{z[0].x, z[0].y, z[0].z}, {z[1].x, z[1].y, z[1].z}, {z[2].x, z[2].y, z[2].z}};
      plane_reduced(zz, M, kap * b1, kap * b2, gd, Bq);
      want = 9;
    } else {
      double gs[9], Hs[81];
      s_derivs(kind, z, gs, Hs);
      for (int k = 0; k < 9; ++k) gd[k] = gs[k] * i2d;
      if (kind == 1) {
        write_reduced<6, 2>(Bq, 1, 0, M, gd, Hs, c1, c2);
        want = 6;
      }
    }
    if (A.grad) {
      // grad d in world axes (rotated back from the frame when in it)
      double gw[9];
      for (int m = 0; m < 3; ++m)
        for (int i = 0; i < 3; ++i)
          gw[3 * m + i] = pe_local ? Rf[3 * i] * gd[3 * m] + Rf[3 * i + 1] * gd[3 * m + 1] + Rf[3 * i + 2] * gd[3 * m + 2]
                                   : gd[3 * m + i];
      for (int i = 0; i < 4; ++i) {
        bool used = false;
        for (int m = 0; m < nz; ++m) used |= TI.C[m][i] != 0;
        if (!used) continue;
        for (int al = 0; al < 3; ++al) {
          double v = 0.0;
          for (int m = 0; m < nz; ++m) v += (double)TI.C[m][i] * gw[3 * m + al];
          atomicAdd(&A.grad[(size_t)al * A.n + s.v[i]], kap * b1 * v);
        }
      }
    }
    if (kind == 0) {
      // point-point: H_z = kappa b'' n n^T + (kappa b'/d)(I - n n^T); clamp each part
      const double nh[3] = {gd[0], gd[1], gd[2]};
      const double lam_n = fmax(kap * b2, 0.0), lam_t = fmax(kap * b1 * (2.0 * i2d), 0.0);
      double Hz[9];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
          Hz[3 * i + j] = lam_n * nh[i] * nh[j] + lam_t * ((i == j ? 1.0 : 0.0) - nh[i] * nh[j]);
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
          const int cc = TI.C[0][i] * TI.C[0][j];
          if (cc == 0) continue;
          double blk[9];
          for (int q = 0; q < 9; ++q) blk[q] = (double)cc * Hz[q];
          add_block(A, s.v[i], s.v[j], blk, false);
        }
    }
  }
  // queue slot (warp-aggregated allocation), then the reduced matrix, packed
  // upper triangle, element-major (point-edge pairs in their frame: the
  // 4x4 and 2x2 blocks and the frame)
  const unsigned lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  unsigned slot = 0;
#pragma unroll
  for (int which = 0; which < 3; ++which) {
    const int Dw = which == 0 ? 9 : (which == 1 ? 6 : 4);
    const unsigned m = __ballot_sync(0xffffffffu, want == Dw);
    if (!m) continue;
    unsigned base = 0;
    const int leader = __ffs(m) - 1;
    if ((int)lane == leader)
      base = atomicAdd(which == 0 ? A.n9 : (which == 1 ? A.n6 : A.n4), (unsigned)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (want == Dw) slot = base + __popc(m & lt);
  }
  if (want != 0) {
    double* Bo = want == 9 ? A.B9 : (want == 6 ? A.B6 : A.B4);
    const int ne = want == 9 ? 45 : (want == 6 ? 21 : 19);
#pragma unroll
    for (int e = 0; e < 45; ++e)
      if (e < ne) Bo[(size_t)e * A.cap + slot] = Bq[e];
    (want == 9 ? A.slot9 : (want == 6 ? A.slot6 : A.slot4))[slot] = (uint32_t)a;
  }
  member_energy_add(A.macc, mem, e_local);
}

// ---- IPC's edge-edge mollifier (CB_EE_MOLLIFIER) -------------------------
// A mollified pair's energy m(c) kappa b(d) depends on all four points
// whatever its distance type, so it leaves the reduced paths of k_hess_prep.
// Its gradient and Hessian are formed here from analytic derivatives of the
// typed distance d and of c = |e0 x e1|^2, written in the difference vectors
// the distance is a function of and mapped to the four points:
//   point-point  r = q - p:              s = |r|^2
//   point-line   w = q - e0, u = e1 - e0: s = |w|^2 - (w.u)^2 / |u|^2
//     (then grad d = grad s / 2d, hess d = (hess s - 2 grad d grad d^T) / 2d)
//   line-line    w = b0 - a0, u = a1 - a0, v = b1 - b0, n = u x v:
//     d = |g| / sqrt(N), g = w.n, N = |n|^2, differentiated directly (no
//     squared distance, whose two large terms cancel for near-parallel edges)
//   c = N (the same u, v), grad and hess in closed form.
// The Hessian by the product rule,
//   H = kappa (m (b'' gd gd^T + b' Hd) + b' m' (gc gd^T + gd gc^T)
//              + b (m'' gc gc^T + m' Hc)),
// and the 9x9 matrix of the four-point translation-free basis
// (B = (K4 x I)^T H (K4 x I)) is queued for k_hess_proj<9>.
struct LocalDeriv {
  int nb;                  // difference vectors (blocks of 3)
  int plus[3], minus[3];   // block b = x[plus[b]] - x[minus[b]] (stencil points 0..3)
  double g[9];             // gradient in the blocks
  double H[9][9];          // Hessian in the blocks
};

// the gradient and Hessian of a function of the difference vectors, as
// functions of the 12 coordinates of the four stencil points
__device__ void local_to_points(const LocalDeriv& L, double (&g12)[12], double (&H12)[12][12]) {
  double cf[4][3];
  for (int P = 0; P < 4; ++P)
    for (int b = 0; b < 3; ++b) cf[P][b] = b < L.nb ? (L.plus[b] == P ? 1.0 : 0.0) - (L.minus[b] == P ? 1.0 : 0.0) : 0.0;
  for (int P = 0; P < 4; ++P)
    for (int i = 0; i < 3; ++i) {
      double v = 0.0;
      for (int b = 0; b < L.nb; ++b) v += cf[P][b] * L.g[3 * b + i];
      g12[3 * P + i] = v;
    }
  for (int P = 0; P < 4; ++P)
    for (int Q = 0; Q < 4; ++Q)
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          double v = 0.0;
          for (int b = 0; b < L.nb; ++b) {
            if (cf[P][b] == 0.0) continue;
            for (int e = 0; e < L.nb; ++e) v += cf[P][b] * cf[Q][e] * L.H[3 * b + i][3 * e + j];
          }
          H12[3 * P + i][3 * Q + j] = v;
        }
}

// |u x v|^2 of u (block bu) and v (block bv): gradient and Hessian entries added with weight w
__device__ void add_cross2(LocalDeriv& L, int bu, int bv, const d3& u, const d3& v, double wg, double wh) {
  const double uu = dot3(u, u), vv = dot3(v, v), uv = dot3(u, v);
  const double U[3] = {u.x, u.y, u.z}, V[3] = {v.x, v.y, v.z};
  for (int i = 0; i < 3; ++i) {
    L.g[3 * bu + i] += wg * (2.0 * vv * U[i] - 2.0 * uv * V[i]);
    L.g[3 * bv + i] += wg * (2.0 * uu * V[i] - 2.0 * uv * U[i]);
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const double dl = i == j ? 1.0 : 0.0;
      L.H[3 * bu + i][3 * bu + j] += wh * (2.0 * vv * dl - 2.0 * V[i] * V[j]);
      L.H[3 * bv + i][3 * bv + j] += wh * (2.0 * uu * dl - 2.0 * U[i] * U[j]);
      const double m = 4.0 * U[i] * V[j] - 2.0 * V[i] * U[j] - 2.0 * uv * dl;  // d2/du_i dv_j
      L.H[3 * bu + i][3 * bv + j] += wh * m;
      L.H[3 * bv + j][3 * bu + i] += wh * m;
    }
}

// gradient and Hessian of the typed edge-edge distance d (types as in
// geometry.cuh) in difference vectors of the stencil X (a0 a1 b0 b1)
__device__ void ee_distance_derivs(int ty, const d3 (&X)[4], double d, LocalDeriv& L) {
  for (int i = 0; i < 9; ++i) {
    L.g[i] = 0.0;
    for (int j = 0; j < 9; ++j) L.H[i][j] = 0.0;
  }
  if (ty <= 7) {
    // squared distance s in (r) or (w, u), then d
    if (ty <= 3) {
      const int p = ty <= 1 ? 0 : 1, q = (ty & 1) ? 3 : 2;
      L.nb = 1;
      L.plus[0] = q;
      L.minus[0] = p;
      const d3 r = sub3(X[q], X[p]);
      const double R[3] = {r.x, r.y, r.z};
      for (int i = 0; i < 3; ++i) {
        L.g[i] = 2.0 * R[i];
        L.H[i][i] = 2.0;
      }
    } else {
      // point q, line e0 e1: 4 PE(a0, b), 5 PE(a1, b), 6 PE(b0, a), 7 PE(b1, a)
      const int q = ty == 4 ? 0 : ty == 5 ? 1 : ty == 6 ? 2 : 3;
      const int e0 = ty <= 5 ? 2 : 0, e1 = ty <= 5 ? 3 : 1;
      L.nb = 2;
      L.plus[0] = q;
      L.minus[0] = e0;
      L.plus[1] = e1;
      L.minus[1] = e0;
      const d3 w = sub3(X[q], X[e0]), u = sub3(X[e1], X[e0]);
      const double a = dot3(w, u), gg = dot3(u, u), ig = 1.0 / gg;
      const double W[3] = {w.x, w.y, w.z}, U[3] = {u.x, u.y, u.z};
      for (int i = 0; i < 3; ++i) {
        L.g[i] = 2.0 * W[i] - 2.0 * a * U[i] * ig;
        L.g[3 + i] = -2.0 * a * W[i] * ig + 2.0 * a * a * U[i] * ig * ig;
      }
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          const double dl = i == j ? 1.0 : 0.0;
          L.H[i][j] = 2.0 * dl - 2.0 * U[i] * U[j] * ig;
          const double wu = -2.0 * U[i] * W[j] * ig - 2.0 * a * dl * ig + 4.0 * a * U[i] * U[j] * ig * ig;
          L.H[i][3 + j] = wu;
          L.H[3 + j][i] = wu;
          L.H[3 + i][3 + j] = -2.0 * W[i] * W[j] * ig + 4.0 * a * (W[i] * U[j] + U[i] * W[j]) * ig * ig +
                              2.0 * a * a * dl * ig * ig - 8.0 * a * a * U[i] * U[j] * ig * ig * ig;
        }
    }
    // s -> d: grad d = grad s / 2d, hess d = (hess s - 2 grad d grad d^T) / 2d
    const double h = 0.5 / d;
    for (int i = 0; i < 3 * L.nb; ++i) L.g[i] *= h;
    for (int i = 0; i < 3 * L.nb; ++i)
      for (int j = 0; j < 3 * L.nb; ++j) L.H[i][j] = (L.H[i][j] - 2.0 * L.g[i] * L.g[j]) * h;
    return;
  }
  // line-line: d = |g| / sqrt(N), blocks w = b0 - a0, u = a1 - a0, v = b1 - b0
  L.nb = 3;
  L.plus[0] = 2;
  L.minus[0] = 0;
  L.plus[1] = 1;
  L.minus[1] = 0;
  L.plus[2] = 3;
  L.minus[2] = 2;
  const d3 w = sub3(X[2], X[0]), u = sub3(X[1], X[0]), v = sub3(X[3], X[2]);
  const d3 n = cross3(u, v), vw = cross3(v, w), wu = cross3(w, u);
  const double g = dot3(w, n), N = dot3(n, n);
  const double sg = g >= 0.0 ? 1.0 : -1.0, r = 1.0 / sqrt(N), r3 = r * r * r, r5 = r3 * r * r;
  // grad g = (n, v x w, w x u); hess g: the cross-product blocks
  const double Gg[9] = {n.x, n.y, n.z, vw.x, vw.y, vw.z, wu.x, wu.y, wu.z};
  // grad N and hess N (blocks u, v)
  LocalDeriv Nd;
  Nd.nb = 3;
  for (int i = 0; i < 9; ++i) {
    Nd.g[i] = 0.0;
    for (int j = 0; j < 9; ++j) Nd.H[i][j] = 0.0;
  }
  add_cross2(Nd, 1, 2, u, v, 1.0, 1.0);
  // hess g: d2g/dw du = -[v]x, d2g/dw dv = [u]x, d2g/du dv = -[w]x ([a]x b = a x b)
  auto crossm = [](const d3& a, double sgn, double (&M)[3][3]) {
    M[0][0] = 0.0;
    M[0][1] = -sgn * a.z;
    M[0][2] = sgn * a.y;
    M[1][0] = sgn * a.z;
    M[1][1] = 0.0;
    M[1][2] = -sgn * a.x;
    M[2][0] = -sgn * a.y;
    M[2][1] = sgn * a.x;
    M[2][2] = 0.0;
  };
  double Hg[9][9];
  for (int i = 0; i < 9; ++i)
    for (int j = 0; j < 9; ++j) Hg[i][j] = 0.0;
  {
    double M[3][3], T[3][3];
    crossm(v, -1.0, M);  // rows w, cols u
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        Hg[i][3 + j] = M[i][j];
        Hg[3 + j][i] = M[i][j];
      }
    crossm(u, 1.0, T);  // rows w, cols v
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        Hg[i][6 + j] = T[i][j];
        Hg[6 + j][i] = T[i][j];
      }
    crossm(w, -1.0, M);  // rows u, cols v
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        Hg[3 + i][6 + j] = M[i][j];
        Hg[6 + j][3 + i] = M[i][j];
      }
  }
  for (int i = 0; i < 9; ++i) L.g[i] = sg * (r * Gg[i] - 0.5 * g * r3 * Nd.g[i]);
  for (int i = 0; i < 9; ++i)
    for (int j = 0; j < 9; ++j)
      L.H[i][j] = sg * (r * Hg[i][j] - 0.5 * r3 * (Gg[i] * Nd.g[j] + Nd.g[i] * Gg[j]) - 0.5 * g * r3 * Nd.H[i][j] +
                        0.75 * g * r5 * Nd.g[i] * Nd.g[j]);
}

// one thread per mollified pair (listed by k_kind_split)
__global__ void __launch_bounds__(128) k_moll_hess(HessArgs A) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double e_local = 0.0;
  int mem = -1;
  if (t < (int64_t)*A.nmoll) {
    const uint32_t a = A.mlist[t];
    const uint32_t c = A.aidx[a];
    const uint64_t key = A.cand[c];
    const Stencil s = stencil_of(key, A.ev0, A.ev1, A.tv, A.T);
    const int ty = A.ctype[c];
    mem = A.vsc[s.v[0]];
    const PassParams P = member_pass(A.mp[mem]);
    double xi_p, dh_p;
    pair_params(P, A.ccls[c], f_width(P, A.dbar_comp, A.comp, s.v[0]), xi_p, dh_p);
    const double d = A.cd[c];
    double b, b1, b2;
    barrier_b012(d - xi_p, dh_p, b, b1, b2);
    // points relative to the first one (translation changes no derivative)
    const d3 X0 = load3(A.x, A.n, s.v[0]);
    d3 X[4];
    for (int q = 0; q < 4; ++q) X[q] = sub3(load3(A.x, A.n, s.v[q]), X0);
    double gd[12], gc[12], Hd[12][12], Hc[12][12];
    {
      LocalDeriv L;
      ee_distance_derivs(ty, X, d, L);
      local_to_points(L, gd, Hd);
    }
    double cval;
    {
      LocalDeriv L;
      L.nb = 2;
      L.plus[0] = 1;
      L.minus[0] = 0;
      L.plus[1] = 3;
      L.minus[1] = 2;
      for (int i = 0; i < 9; ++i) {
        L.g[i] = 0.0;
        for (int j = 0; j < 9; ++j) L.H[i][j] = 0.0;
      }
      const d3 u = sub3(X[1], X[0]), v = sub3(X[3], X[2]);
      const d3 n = cross3(u, v);
      cval = dot3(n, n);
      add_cross2(L, 0, 1, u, v, 1.0, 1.0);
      local_to_points(L, gc, Hc);
    }
    const double eps = 1e-3 * A.elen2[cb_key_i(key)] * A.elen2[cb_key_j(key)];
    double m, m1, m2;
    ee_mollifier(cval, eps, m, m1, m2);
    const double kap = P.kappa;
    e_local = kap * m * b;
    if (A.grad)
      for (int i = 0; i < 12; ++i) {
        const double g = kap * (m * b1 * gd[i] + b * m1 * gc[i]);
        if (g != 0.0) atomicAdd(&A.grad[(size_t)(i % 3) * A.n + s.v[i / 3]], g);
      }
    double Bf[81];
    for (int k = 0; k < 81; ++k) Bf[k] = 0.0;
    for (int i = 0; i < 12; ++i)
      for (int j = i; j < 12; ++j) {
        const double h = kap * (m * (b2 * gd[i] * gd[j] + b1 * Hd[i][j]) + b1 * m1 * (gc[i] * gd[j] + gd[i] * gc[j]) +
                                b * (m2 * gc[i] * gc[j] + m1 * Hc[i][j]));
        const int q1 = i / 3, al = i % 3, q2 = j / 3, be = j % 3;
        for (int p1 = 0; p1 < 3; ++p1)
          for (int p2 = 0; p2 < 3; ++p2) {
            const double w = c_K4[q1][p1] * c_K4[q2][p2] * h;
            Bf[(3 * p1 + al) * 9 + 3 * p2 + be] += w;
            if (i != j) Bf[(3 * p2 + be) * 9 + 3 * p1 + al] += w;
          }
      }
    const unsigned slot = atomicAdd(A.n9, 1u);
    for (int i = 0; i < 9; ++i)
      for (int j = i; j < 9; ++j) A.B9[(size_t)tri_idx(i, j, 9) * A.cap + slot] = Bf[i * 9 + j];
    A.slot9[slot] = a;
  }
  member_energy_add(A.macc, mem, e_local);
}

// Cyclic Jacobi with symmetric updates on a packed upper-triangular matrix
// held in shared memory (element e of this thread at Am[e * S]); rotations are
// accumulated into V (column-major: row i of column k at V[(k * D + i) * S]).
// Rotations with |a_pq| below
// 1e-16 of the norm are skipped; stops when off^2 <= tol2 * ||A||^2.
template <typename R, int D>
__device__ __forceinline__ void jacobi_packed(R* Am, R* V, const int S, const R tol2, const int max_sweeps) {
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    R off = 0, fro = 0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const R d = Am[tri_idx(i, i, D) * S];
      fro += d * d;
#pragma unroll
      for (int j = i + 1; j < D; ++j) {
        const R v = Am[tri_idx(i, j, D) * S];
        off += R(2) * v * v;
      }
    }
    fro += off;
    if (fro == R(0) || off <= tol2 * fro) break;
    const R skip = R(1e-16) * sqrt(fro);
    for (int p = 0; p < D - 1; ++p)
      for (int q = p + 1; q < D; ++q) {
        const R apq = Am[tri_idx(p, q, D) * S];
        if (fabs(apq) <= skip) continue;
        const R app = Am[tri_idx(p, p, D) * S], aqq = Am[tri_idx(q, q, D) * S];
        const R tau = (aqq - app) / (R(2) * apq);
        const R t = (tau >= R(0) ? R(1) : R(-1)) / (fabs(tau) + sqrt(R(1) + tau * tau));
        const R c = R(1) / sqrt(R(1) + t * t), s = t * c;
        Am[tri_idx(p, p, D) * S] = app - t * apq;
        Am[tri_idx(q, q, D) * S] = aqq + t * apq;
        Am[tri_idx(p, q, D) * S] = R(0);
        for (int k = 0; k < D; ++k) {
          if (k == p || k == q) continue;
          const int ikp = (k < p ? tri_idx(k, p, D) : tri_idx(p, k, D)) * S;
          const int ikq = (k < q ? tri_idx(k, q, D) : tri_idx(q, k, D)) * S;
          const R akp = Am[ikp], akq = Am[ikq];
          Am[ikp] = c * akp - s * akq;
          Am[ikq] = s * akp + c * akq;
        }
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const R vkp = V[(p * D + k) * S], vkq = V[(q * D + k) * S];
          V[(p * D + k) * S] = c * vkp - s * vkq;
          V[(q * D + k) * S] = s * vkp + c * vkq;
        }
      }
  }
}

// 1 / sqrt(u) for u >= 1 in FP64 without the FP64 square root and division:
// the FP32 estimate (relative error < 1e-7) refined by two Newton steps
// (error squared each time, so to FP64 rounding).
__device__ __forceinline__ double rsqrt_refined(double u) {
  double c = (double)rsqrtf((float)u);
  c = c * (1.5 - 0.5 * u * c * c);
  c = c * (1.5 - 0.5 * u * c * c);
  return c;
}

// The FP64 sweeps of the projection, after the FP32 eigenvectors: cyclic
// Jacobi where each rotation's tangent comes from FP32 arithmetic on values
// scaled by the matrix norm, and the rotation itself is exact: c = 1/sqrt(1+t^2)
// to FP64 rounding (rsqrt_refined), s = t c, and the 2x2 pivot block is
// transformed with the full similarity formulas.  A tangent off by a relative
// 1e-7 leaves a_pq at 1e-7 of its value -- quadratically small after the FP32
// phase -- for the next sweep, while A stays an exact similarity of the input
// and V stays orthonormal.  This avoids every FP64 division and square root
// in the rotations.  Stops when off^2 <= tol2 ||A||^2.
template <int D>
__device__ __forceinline__ void jacobi_refine64(double* Am, double* V, const int S, const double tol2,
                                                const int max_sweeps) {
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    double off = 0, fro = 0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const double d = Am[tri_idx(i, i, D) * S];
      fro += d * d;
#pragma unroll
      for (int j = i + 1; j < D; ++j) {
        const double v = Am[tri_idx(i, j, D) * S];
        off += 2.0 * v * v;
      }
    }
    fro += off;
    if (fro == 0.0 || off <= tol2 * fro) break;
    const double nrm = sqrt(fro);
    const double skip = 1e-16 * nrm;
    const double inv = 1.0 / nrm;
    for (int p = 0; p < D - 1; ++p)
      for (int q = p + 1; q < D; ++q) {
        const double apq = Am[tri_idx(p, q, D) * S];
        if (fabs(apq) <= skip) continue;
        const double app = Am[tri_idx(p, p, D) * S], aqq = Am[tri_idx(q, q, D) * S];
        // |apq| > 1e-16 ||A||, so the scaled FP32 values stay normal
        const float apq32 = (float)(apq * inv), dd32 = (float)((aqq - app) * inv);
        const float tau = dd32 / (2.f * apq32);
        const float t32 = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
        const double t = (double)t32;
        if (__all_sync(__activemask(), fabs(t) < 1e-8)) {
          // small angle in every lane (warp-uniform, so no lane runs both
          // paths): c = 1/sqrt(1+t^2) rounds to 1 in FP64, s = t; the residual
          // a_pq (a relative 1e-7 of a_pq, below 1e-15 ||A||) is dropped
          Am[tri_idx(p, p, D) * S] = app - t * apq;
          Am[tri_idx(q, q, D) * S] = aqq + t * apq;
          Am[tri_idx(p, q, D) * S] = 0.0;
          for (int k = 0; k < D; ++k) {
            if (k == p || k == q) continue;
            const int ikp = (k < p ? tri_idx(k, p, D) : tri_idx(p, k, D)) * S;
            const int ikq = (k < q ? tri_idx(k, q, D) : tri_idx(q, k, D)) * S;
            const double akp = Am[ikp], akq = Am[ikq];
            Am[ikp] = akp - t * akq;
            Am[ikq] = akq + t * akp;
          }
#pragma unroll
          for (int k = 0; k < D; ++k) {
            const double vkp = V[(p * D + k) * S], vkq = V[(q * D + k) * S];
            V[(p * D + k) * S] = vkp - t * vkq;
            V[(q * D + k) * S] = vkq + t * vkp;
          }
          continue;
        }
        const double c = rsqrt_refined(1.0 + t * t), s = t * c;
        const double cc = c * c, ss = s * s, cs = c * s;
        Am[tri_idx(p, p, D) * S] = cc * app - 2.0 * cs * apq + ss * aqq;
        Am[tri_idx(q, q, D) * S] = ss * app + 2.0 * cs * apq + cc * aqq;
        Am[tri_idx(p, q, D) * S] = cs * (app - aqq) + (cc - ss) * apq;
        for (int k = 0; k < D; ++k) {
          if (k == p || k == q) continue;
          const int ikp = (k < p ? tri_idx(k, p, D) : tri_idx(p, k, D)) * S;
          const int ikq = (k < q ? tri_idx(k, q, D) : tri_idx(q, k, D)) * S;
          const double akp = Am[ikp], akq = Am[ikq];
          Am[ikp] = c * akp - s * akq;
          Am[ikq] = s * akp + c * akq;
        }
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const double vkp = V[(p * D + k) * S], vkq = V[(q * D + k) * S];
          V[(p * D + k) * S] = c * vkp - s * vkq;
          V[(q * D + k) * S] = s * vkp + c * vkq;
        }
      }
  }
}

// Threads (= queued pairs) per block of the projection kernels.  One warp per
// block: each block's warp moves through the FP32 and FP64 phases on its
// own, so on every SM some warps keep the scarce FP64 pipe busy while others
// are in their FP32 phase (with larger blocks the phase barrier would hold all
// of an SM's warps in step).
#ifndef PROJ_THREADS
#define PROJ_THREADS 32
#endif
// squared relative off-diagonal norm at which the FP32 Jacobi phase stops
#ifndef PROJ_FP32_TOL2
#define PROJ_FP32_TOL2 1e-12f
#endif

// The 4-point transform behind K4 = H / 2 (H rows (1,1,1), (1,-1,-1),
// (-1,1,-1), (-1,-1,1)): h = H p in six additions.
__host__ __device__ __forceinline__ void had3(double p0, double p1, double p2, double (&h)[4]) {
  const double t = p1 + p2, d = p1 - p2;
  h[0] = p0 + t;
  h[1] = p0 - t;
  h[2] = d - p0;
  h[3] = -d - p0;
}

// Entries (i, j) of all sixteen 3x3 blocks of (K4 x I) B+ (K4 x I)^T: with
// P[a][b] = B+[3a+i][3b+j] / 4 (Bq holds B+ / 4), X = H P H^T, block
// (q1, q2) gets X[q1][q2] at (i, j) and, for i != j, X[q2][q1] at (j, i)
// (B+ is symmetric).  Additions only, instead of the products with K4.
__host__ __device__ __forceinline__ void hadamard_block_entries(const double* Bq, int S, int i, int j,
                                                                double (&X)[4][4]) {
  double Q[3][4];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double p[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const int r = 3 * a + i, cl = 3 * b + j;
      p[b] = Bq[(r <= cl ? tri_idx(r, cl, 9) : tri_idx(cl, r, 9)) * S];
    }
    had3(p[0], p[1], p[2], Q[a]);
  }
#pragma unroll
  for (int q2 = 0; q2 < 4; ++q2) {
    double h[4];
    had3(Q[0][q2], Q[1][q2], Q[2][q2], h);
#pragma unroll
    for (int q1 = 0; q1 < 4; ++q1) X[q1][q2] = h[q1];
  }
}

__device__ __forceinline__ void hadamard_scatter(const HessArgs& A, const Stencil& st, const double* Bq, int S) {
  int64_t off[4][4];
  bool miss = false;
#pragma unroll
  for (int q1 = 0; q1 < 4; ++q1)
#pragma unroll
    for (int q2 = 0; q2 < 4; ++q2) {
      const int r = st.v[q1], cc = st.v[q2];
      const int64_t bi = find_block(A.row_ptr, A.col, r, cc);
      const bool hit = bi < A.row_ptr[r + 1] && A.col[bi] == cc;
      miss |= !hit;
      off[q1][q2] = hit ? 9 * bi : -1;
    }
  if (miss) atomicOr(A.status, (unsigned long long)CB_DEV_CAPACITY);  // pattern miss: never expected
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      double X[4][4];
      hadamard_block_entries(Bq, S, i, j, X);
#pragma unroll
      for (int q1 = 0; q1 < 4; ++q1)
#pragma unroll
        for (int q2 = 0; q2 < 4; ++q2) {
          if (off[q1][q2] < 0) continue;
          double* dst = A.val + off[q1][q2];
          atomicAdd(&dst[3 * i + j], X[q1][q2]);
          if (i != j) atomicAdd(&dst[3 * j + i], X[q2][q1]);
        }
    }
}

template <int D>
struct ProjSmem {
  static constexpr int NP = D * (D + 1) / 2;
  // per thread: V (D*D doubles, column-major; the FP32 eigenvectors occupy its
  // first D*D floats during the FP32 phase) | A (NP doubles; the FP32 matrix in
  // its first NP floats during the FP32 phase, then the FP64 matrix, then B+)
  static constexpr int PER_THREAD = (D * D + NP) * 8;
};

// Stage (d), part 2, one thread per queued pair: PSD projection of the D x D
// reduced matrix and the BSR scatter.  The input B stays in registers; the
// eigenvectors V and the working matrix A live in shared memory laid out
// element-major ([element][thread]), so a warp touches 32 consecutive words
// per access, 1008 B per thread for D = 9.  The eigen-decomposition is FP32
// first (Jacobi on the cheap pipe to ~1e-6), its arrays inside the V and A
// regions; then FP64: modified Gram-Schmidt on the eigenvectors, A = V^T B V,
// and symmetric Jacobi sweeps to an off-diagonal norm of 1e-14 ||A||.
// Projection onto the PSD cone is non-expansive in the Frobenius norm, so the
// projected matrix is exact to 1e-14 of ||B||.  B+ is mapped back to the
// involved points with K (x) I and scattered.
template <int D, int S>
__global__ void __launch_bounds__(S) k_hess_proj(HessArgs A) {
  constexpr int NP = D * (D + 1) / 2;
  extern __shared__ double smem[];
  const int tid = threadIdx.x;
  const int64_t m = (int64_t)*(D == 9 ? A.n9 : A.n6);
  // grid-stride over the queue, S pairs per step; the loop bound is the same
  // for every thread of a block, and a thread past the end leaves only in the
  // block's last step, after its last barrier
  for (int64_t base = (int64_t)blockIdx.x * S; base < m; base += (int64_t)gridDim.x * S) {
    // the previous step's B+ and V (double layout) overlap other threads' FP32
    // arrays of this step
    __syncthreads();
    const int64_t w = base + tid;
    double* Vs = smem + tid;                            // V: row i of column k at [(k * D + i) * S]
    double* Ad = smem + D * D * S + tid;                // A: element e at [e * S]
    float* V32 = (float*)smem + tid;                    // FP32 V, same indexing, inside the V region
    float* A32 = (float*)(smem + D * D * S) + tid;      // FP32 A, same indexing, inside the A region
    const bool act = w < m;                             // no early exit before the last barrier
    const double* Bg = D == 9 ? A.B9 : A.B6;
    const uint32_t a = act ? (D == 9 ? A.slot9 : A.slot6)[w] : 0u;
    // B stays in registers until B+ is formed
    double Br[NP];
    double mx = 0.0;
#pragma unroll
    for (int e = 0; e < NP; ++e) {
      Br[e] = act ? Bg[(size_t)e * A.cap + w] : 0.0;
      mx = fmax(mx, fabs(Br[e]));
    }
    const bool work = act && mx != 0.0;
    if (work) {
      const double inv = 1.0 / mx;
#pragma unroll
      for (int e = 0; e < NP; ++e) A32[e * S] = (float)(Br[e] * inv);
      for (int k = 0; k < D; ++k)
        for (int i = 0; i < D; ++i) V32[(k * D + i) * S] = (i == k) ? 1.f : 0.f;
      jacobi_packed<float, D>(A32, V32, S, PROJ_FP32_TOL2, 12);
    }
    // FP64 re-orthonormalisation of the FP32 eigenvectors (modified Gram-Schmidt),
    // columns in descending order.  Double column k takes the bytes of float
    // columns 2k and 2k+1 (column 0: 0 and 1), all read before it is written:
    // higher columns in earlier steps, column k itself before the barrier.
    for (int k = D - 1; k >= 0; --k) {
      double v[D];
#pragma unroll
      for (int i = 0; i < D; ++i) v[i] = work ? (double)V32[(k * D + i) * S] : 0.0;
      __syncthreads();
      if (work) {
        for (int j = k + 1; j < D; ++j) {
          double dp = 0.0;
#pragma unroll
          for (int i = 0; i < D; ++i) dp += Vs[(j * D + i) * S] * v[i];
#pragma unroll
          for (int i = 0; i < D; ++i) v[i] -= dp * Vs[(j * D + i) * S];
        }
        double nn = 0.0;
#pragma unroll
        for (int i = 0; i < D; ++i) nn += v[i] * v[i];
        nn = rsqrt_refined(nn);  // nn is 1 to FP32 accuracy here
#pragma unroll
        for (int i = 0; i < D; ++i) Vs[(k * D + i) * S] = v[i] * nn;
      }
    }
    // from here on every thread touches only its own elements: no more barriers
    if (!act) continue;  // the block's last step
    // eigenvalues -> diagonal of Ad, eigenvectors -> Vs
    if (!work) {
      for (int e = 0; e < NP; ++e) Ad[e * S] = 0.0;
      for (int k = 0; k < D; ++k)
        for (int i = 0; i < D; ++i) Vs[(k * D + i) * S] = (i == k) ? 1.0 : 0.0;
    } else {
      // A = V^T B V, column by column (the FP32 A is dead: every thread passed
      // the Gram-Schmidt barriers after its FP32 phase)
      for (int l = 0; l < D; ++l) {
        double vl[D], t[D];
#pragma unroll
        for (int j = 0; j < D; ++j) vl[j] = Vs[(l * D + j) * S];
#pragma unroll
        for (int i = 0; i < D; ++i) {
          double v = 0.0;
#pragma unroll
          for (int j = 0; j < D; ++j) v += Br[i <= j ? tri_idx(i, j, D) : tri_idx(j, i, D)] * vl[j];
          t[i] = v;
        }
        for (int k = 0; k <= l; ++k) {
          double v = 0.0;
#pragma unroll
          for (int i = 0; i < D; ++i) v += Vs[(k * D + i) * S] * t[i];
          Ad[tri_idx(k, l, D) * S] = v;
        }
      }
      jacobi_refine64<D>(Ad, Vs, S, 1e-28, 12);
    }
    // B+ (into the A region) from the side with fewer terms: the sum over the
    // positive eigenpairs of lam v v^T, or B minus the sum over the negative
    // ones (B = V A V^T to the FP64 sweeps' tolerance).  The loop runs as many
    // terms as the warp's busiest lane needs; each lane adds its own j-th term.
    double lam[D];
    int npos = 0, nneg = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      lam[k] = Ad[tri_idx(k, k, D) * S];
      npos += lam[k] > 0.0;
      nneg += lam[k] < 0.0;
    }
    const bool from_b = nneg < npos;
    const int nterm = from_b ? nneg : npos;
    const int wterm = __reduce_max_sync(__activemask(), nterm);
    double* Bs = Ad;  // B+ replaces A (for D = 9 scaled by 1/4, the square of K4's entries)
    constexpr double bsc = D == 9 ? 0.25 : 1.0;
#pragma unroll
    for (int e = 0; e < NP; ++e) Bs[e * S] = from_b ? Br[e] * bsc : 0.0;
    for (int j = 0; j < wterm; ++j) {
      int k = -1, cnt = 0;
      double wk = 0.0;
#pragma unroll
      for (int kk = 0; kk < D; ++kk) {
        const bool sel = from_b ? lam[kk] < 0.0 : lam[kk] > 0.0;
        if (sel && cnt == j) {
          k = kk;
          wk = (from_b ? -lam[kk] : lam[kk]) * bsc;
        }
        cnt += sel;
      }
      if (k < 0) continue;
      double v[D];
#pragma unroll
      for (int i = 0; i < D; ++i) v[i] = Vs[(k * D + i) * S];
#pragma unroll
      for (int i = 0; i < D; ++i) {
        const double wi = wk * v[i];
#pragma unroll
        for (int jj = i; jj < D; ++jj) Bs[tri_idx(i, jj, D) * S] += wi * v[jj];
      }
    }
    const uint32_t c = A.aidx[a];
    const Stencil st = stencil_of(A.cand[c], A.ev0, A.ev1, A.tv, A.T);
    if constexpr (D == 9) {
      // the plane types involve all four points, in stencil order
      hadamard_scatter(A, st, Bs, S);
    } else {
      // scatter: block (q1, q2) of the involved points
      //   = sum_ab K[q1][ab] R[q2][ab],  R[q2][ab] = sum_bb K[q2][bb] B+[ab, bb]
      // (3x3 blocks; R for one q2 at a time)
      const TypeInfo& TI = st.ee ? c_ee_types[A.ctype[c]] : c_pt_types[A.ctype[c]];
      const int nz = TI.kind + 1;
      int pts[4], np = 0;
      for (int i = 0; i < 4; ++i) {
        bool used = false;
        for (int mm = 0; mm < nz; ++mm) used |= TI.C[mm][i] != 0;
        if (used) pts[np++] = i;
      }
      constexpr int NB = D / 3;
      for (int q2 = 0; q2 < np; ++q2) {
        double R[NB][9];
#pragma unroll
        for (int ab = 0; ab < NB; ++ab)
#pragma unroll
          for (int al = 0; al < 3; ++al)
#pragma unroll
            for (int be = 0; be < 3; ++be) {
              double v = 0.0;
#pragma unroll
              for (int bb = 0; bb < NB; ++bb) {
                const int r = 3 * ab + al, cl = 3 * bb + be;
                v += c_K3[q2][bb] * Bs[(r <= cl ? tri_idx(r, cl, D) : tri_idx(cl, r, D)) * S];
              }
              R[ab][3 * al + be] = v;
            }
        for (int q1 = 0; q1 <= q2; ++q1) {
          double blk[9];
#pragma unroll
          for (int e = 0; e < 9; ++e) {
            double v = 0.0;
#pragma unroll
            for (int ab = 0; ab < NB; ++ab) v += c_K3[q1][ab] * R[ab][e];
            blk[e] = v;
          }
          const int r = st.v[pts[q1]], cc = st.v[pts[q2]];
          add_block(A, r, cc, blk, false);
          if (q1 != q2) add_block(A, cc, r, blk, true);
        }
      }
    }
  }
}

// ---- the 9x9 projection for short queues: a warp per pair ----------------
// One thread per pair runs some 8,500 dependent FP64 instructions, and an FP64
// warp instruction occupies a warp for 64 cycles however many of its lanes
// are active (measured on GB300: 64 cycles per dependent or independent DFMA
// of a lone warp; 76 with one warp per SM sub-partition, the SM's FP64 unit
// then full at one warp instruction per ~19 cycles), so a short queue (a
// small scene) waits for that chain however idle the device is.  This form
// spreads one pair over a warp, the three lanes (r, t) = (l / 3, l % 3) of
// row r (lanes 0..26) owning entries t, t + 3, t + 6 of row and column r,
// and orders the Jacobi rotations round robin: in round k of a sweep row r
// pairs with (2k - r) mod 9 (row k rests), the four disjoint rotations of a
// round are applied at once (X = A J by columns, then J^T X by rows, V J by
// columns), so a sweep is 9 rounds of 18 FP64 instructions per lane
// instead of 36 rotations in sequence.  Each lane computes its own row's
// rotation, the same bits in every lane of the pair's two rows.  The arithmetic is
// otherwise that of k_hess_proj<9>: FP32 Jacobi on the scaled matrix to
// the same tolerance, FP64 modified Gram-Schmidt, A = V^T B V, FP64 sweeps
// with FP32 tangents and FP64-normalised rotations to an off-diagonal norm
// of 1e-14 ||A||, B+ from the positive eigenpairs, the Hadamard scatter.
constexpr int PL_PAIRS = 4;                 // pairs per block
constexpr int PL_THREADS = 32 * PL_PAIRS;   // one warp per pair: three lanes per row
// doubles per pair: A, X (A J; later the Hadamard staging, 108), V, and the
// FP32 phase's A, X, V (3 x 81 floats)
constexpr int PL_SMEM = 81 + 108 + 81 + 122;
// queues of at most this many active pairs take the lane-parallel form
constexpr int64_t PL_MAX_ACTIVE = 4096;

// sum over the warp: a butterfly, so every lane gets the same bits
template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// one round of simultaneous rotations on a 9x9 matrix As and vectors Vs held
// in shared memory ([9 i + j]); the three lanes (r, t) of row r apply its
// pair's rotation (c, sg: sg = -s for the lower index of the pair, +s for the
// upper, 0 and c = 1 for a resting row or a skipped pair) to entries
// t, t + 3, t + 6 of column r, then of row r
template <typename R>
__device__ __forceinline__ void rr_apply3(R* As, R* Xs, R* Vs, int r, int t, int pr, R c, R sg, bool row) {
  R vr[3], vp[3];
  if (row) {
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const int i = t + 3 * m;
      Xs[9 * i + r] = c * As[9 * i + r] + sg * As[9 * i + pr];
      vr[m] = Vs[9 * i + r];
      vp[m] = Vs[9 * i + pr];
    }
  }
  __syncwarp();  // X complete; every lane holds the V entries it needs
  if (row) {
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const int i = t + 3 * m;
      Vs[9 * i + r] = c * vr[m] + sg * vp[m];
      As[9 * r + i] = c * Xs[9 * r + i] + sg * Xs[9 * pr + i];
    }
  }
  __syncwarp();
}

// the rotation of row r's pair (r, pr) in a round: c and sg as rr_apply3 takes
// them; every lane of the pair's two rows computes the same bits
template <typename R>
__device__ __forceinline__ void pl_rotation(const R* As, int r, int pr, bool row, R skip, double inv, R& c, R& sg);

template <>
__device__ __forceinline__ void pl_rotation<float>(const float* As, int r, int pr, bool row, float skip, double,
                                                   float& c, float& sg) {
  c = 1.f;
  sg = 0.f;
  if (!row || pr == r) return;
  const int p = min(r, pr), q = max(r, pr);
  const float apq = As[9 * p + q];
  if (!(fabsf(apq) > skip)) return;
  const float app = As[9 * p + p], aqq = As[9 * q + q];
  const float tau = (aqq - app) / (2.f * apq);
  const float t = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
  c = 1.f / sqrtf(1.f + t * t);
  sg = r == p ? -t * c : t * c;
}

// FP64: the tangent from FP32 arithmetic on the values scaled by the norm,
// c = 1/sqrt(1 + t^2) to FP64 rounding
template <>
__device__ __forceinline__ void pl_rotation<double>(const double* As, int r, int pr, bool row, double skip,
                                                    double inv, double& c, double& sg) {
  c = 1.0;
  sg = 0.0;
  if (!row || pr == r) return;
  const int p = min(r, pr), q = max(r, pr);
  const double apq = As[9 * p + q];
  if (!(fabs(apq) > skip)) return;
  const double app = As[9 * p + p], aqq = As[9 * q + q];
  const float apq32 = (float)(apq * inv), dd32 = (float)((aqq - app) * inv);
  const float tau = dd32 / (2.f * apq32);
  const float t32 = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
  const double t = (double)t32;
  c = rsqrt_refined(1.0 + t * t);
  sg = r == p ? -t * c : t * c;
}

__device__ __forceinline__ void proj_lanes_block(const HessArgs& A, int block) {
  extern __shared__ double pl_smem[];
  const int seg = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = lane / 3, t = lane - 3 * r;  // row r (< 9 for lanes 0..26), third t
  const bool row = lane < 27;
  const int64_t w = (int64_t)block * PL_PAIRS + seg;
  if (w >= (int64_t)*A.n9) return;  // the whole warp leaves together
  double* As = pl_smem + (size_t)seg * PL_SMEM;  // A[i][j] at [9 i + j]
  double* Xs = As + 81;                          // A J; later the Hadamard staging
  double* Vs = Xs + 108;                         // V[i][k]: component i of eigenvector k
  float* A32 = (float*)(Vs + 81);
  float* X32 = A32 + 81;
  float* V32 = X32 + 81;
  const uint32_t a = A.slot9[w];
  double Br[9];  // row r of B
  double mx = 0.0;
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    Br[j] = row ? A.B9[(size_t)(r <= j ? tri_idx(r, j, 9) : tri_idx(j, r, 9)) * A.cap + w] : 0.0;
    mx = fmax(mx, fabs(Br[j]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (mx == 0.0) return;  // B+ = 0: nothing to add
  // FP32 phase on B / max|B|
  {
    const double inv = 1.0 / mx;
    if (row)
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const int j = t + 3 * m;
        A32[9 * r + j] = (float)(Br[j] * inv);
        V32[9 * r + j] = r == j ? 1.f : 0.f;
      }
    __syncwarp();
    for (int sweep = 0; sweep < 12; ++sweep) {
      float off = 0.f, fro = 0.f;
      if (row)
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          const int j = t + 3 * m;
          const float v = A32[9 * r + j];
          if (j == r) fro += v * v;
          else off += v * v;
        }
      off = warp_sum(off);
      fro = warp_sum(fro) + off;
      if (fro == 0.f || off <= PROJ_FP32_TOL2 * fro) break;
      const float skip = 1e-16f * sqrtf(fro);
      for (int k = 0; k < 9; ++k) {
        const int pr = row ? (2 * k - r + 18) % 9 : r;
        float c, sg;
        pl_rotation<float>(A32, r, pr, row, skip, 0.0, c, sg);
        rr_apply3<float>(A32, X32, V32, r, t, pr, c, sg, row);
      }
    }
  }
  // FP64 modified Gram-Schmidt on the FP32 eigenvectors, columns in
  // descending order; the three lanes of row r hold component r (the same
  // bits), and only lane t = 0 of each row enters the sums
  for (int k = 8; k >= 0; --k) {
    double v = row ? (double)V32[9 * r + k] : 0.0;
    for (int j = k + 1; j < 9; ++j) {
      const double vj = row ? Vs[9 * r + j] : 0.0;
      const double dp = warp_sum(t == 0 ? vj * v : 0.0);
      v -= dp * vj;
    }
    const double nn = rsqrt_refined(warp_sum(t == 0 ? v * v : 0.0));  // 1 to FP32 accuracy here
    if (row) Vs[9 * r + k] = v * nn;  // each lane of the row writes the same bits, then reads its own
  }
  __syncwarp();
  // A = V^T (B V): entries t, t + 3, t + 6 of row r of W = B V into X, then
  // those of the upper triangle of row r of A from the columns of V and W, mirrored
  if (row)
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const int l = t + 3 * m;
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < 9; ++j) s += Br[j] * Vs[9 * j + l];
      Xs[9 * r + l] = s;
    }
  __syncwarp();
  if (row)
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const int l = t + 3 * m;
      if (l < r) continue;
      double s = 0.0;
#pragma unroll
      for (int i = 0; i < 9; ++i) s += Vs[9 * i + r] * Xs[9 * i + l];
      As[9 * r + l] = s;
      As[9 * l + r] = s;
    }
  __syncwarp();
  // FP64 sweeps to an off-diagonal norm of 1e-14 ||A||
  for (int sweep = 0; sweep < 12; ++sweep) {
    double off = 0.0, fro = 0.0;
    if (row)
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const int j = t + 3 * m;
        const double v = As[9 * r + j];
        if (j == r) fro += v * v;
        else off += v * v;
      }
    off = warp_sum(off);
    fro = warp_sum(fro) + off;
    if (fro == 0.0 || off <= 1e-28 * fro) break;
    const double nrm = sqrt(fro);
    const double skip = 1e-16 * nrm, inv = 1.0 / nrm;
    for (int k = 0; k < 9; ++k) {
      const int pr = row ? (2 * k - r + 18) % 9 : r;
      double c, sg;
      pl_rotation<double>(As, r, pr, row, skip, inv, c, sg);
      rr_apply3<double>(As, Xs, Vs, r, t, pr, c, sg, row);
    }
  }
  // B+ / 4 (the square of K4's entries), entries j = t, t + 3, t + 6 of row
  // r: sum over the positive eigenpairs of lam v v^T (the product v_r v_j is
  // formed first, so rows r and j get the same bits); then the point
  // transform over those three column points (axis t) into the staging rows
  double P[3] = {0.0, 0.0, 0.0};
  if (row)
    for (int k = 0; k < 9; ++k) {
      const double lam = As[9 * k + k];
      if (!(lam > 0.0)) continue;
      const double l4 = 0.25 * lam, vr = Vs[9 * r + k];
#pragma unroll
      for (int m = 0; m < 3; ++m) P[m] = fma(vr * Vs[9 * (t + 3 * m) + k], l4, P[m]);
    }
  __syncwarp();  // every lane is done with X
  if (row) {
    double h[4];
    had3(P[0], P[1], P[2], h);
#pragma unroll
    for (int q2 = 0; q2 < 4; ++q2) Xs[12 * r + 3 * q2 + t] = h[q2];
  }
  __syncwarp();
  // lane l < 12 takes block row q1 = l / 3, axis i = l % 3: the transform
  // over the row points, and the sixteen blocks' entries of that row
  if (lane < 12) {
    const int q1 = lane / 3, i = lane % 3;
    const uint32_t ci = A.aidx[a];
    const Stencil st = stencil_of(A.cand[ci], A.ev0, A.ev1, A.tv, A.T);
    const int rv = st.v[q1];
#pragma unroll
    for (int q2 = 0; q2 < 4; ++q2) {
      const int cv = st.v[q2];
      const int64_t bi = find_block(A.row_ptr, A.col, rv, cv);
      if (!(bi < A.row_ptr[rv + 1] && A.col[bi] == cv)) {
        atomicOr(A.status, (unsigned long long)CB_DEV_CAPACITY);  // pattern miss: never expected
        continue;
      }
      double* dst = A.val + 9 * bi + 3 * i;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        double h[4];
        had3(Xs[12 * i + 3 * q2 + j], Xs[12 * (3 + i) + 3 * q2 + j], Xs[12 * (6 + i) + 3 * q2 + j], h);
        atomicAdd(&dst[j], h[q1]);
      }
    }
  }
}

// k_hess_proj<D> over at most one resident wave of blocks (the occupancy
// looked up once per scene)
template <int D>
cb_status launch_proj(cb_scene* s, const HessArgs& A, int64_t cap, cudaStream_t st) {
  const int smem = ProjSmem<D>::PER_THREAD * PROJ_THREADS;
  int& occ = s->proj_occ[D == 9 ? 0 : 1];
  CB_CUDA(cudaFuncSetAttribute(k_hess_proj<D, PROJ_THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  if (occ <= 0) {
    CB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_hess_proj<D, PROJ_THREADS>, PROJ_THREADS, smem));
    occ = std::max(1, occ);
  }
  const int64_t g = std::min<int64_t>(cb_grid(cap, PROJ_THREADS), (int64_t)s->n_sms * occ);
  k_hess_proj<D, PROJ_THREADS><<<(int)std::max<int64_t>(1, g), PROJ_THREADS, smem, cb_count(st)>>>(A);
  CB_CUDA(cudaGetLastError());
  return CB_OK;
}

// Register-resident versions of the two Jacobi phases for the 4x4 block of
// the point-edge path: the same arithmetic as jacobi_packed / jacobi_refine64
// on arrays held in registers (every loop unrolled, every index static).  V
// is column-major: row i of column k at V[k * D + i].
template <typename R, int D>
__device__ __forceinline__ void jacobi_reg(R (&Am)[D * (D + 1) / 2], R (&V)[D * D], const R tol2,
                                           const int max_sweeps) {
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    R off = 0, fro = 0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      fro += Am[tri_idx(i, i, D)] * Am[tri_idx(i, i, D)];
#pragma unroll
      for (int j = i + 1; j < D; ++j) off += R(2) * Am[tri_idx(i, j, D)] * Am[tri_idx(i, j, D)];
    }
    fro += off;
    if (fro == R(0) || off <= tol2 * fro) break;
    const R skip = R(1e-16) * sqrt(fro);
#pragma unroll
    for (int p = 0; p < D - 1; ++p)
#pragma unroll
      for (int q = p + 1; q < D; ++q) {
        const R apq = Am[tri_idx(p, q, D)];
        if (fabs(apq) <= skip) continue;
        const R app = Am[tri_idx(p, p, D)], aqq = Am[tri_idx(q, q, D)];
        const R tau = (aqq - app) / (R(2) * apq);
        const R t = (tau >= R(0) ? R(1) : R(-1)) / (fabs(tau) + sqrt(R(1) + tau * tau));
        const R c = R(1) / sqrt(R(1) + t * t), s = t * c;
        Am[tri_idx(p, p, D)] = app - t * apq;
        Am[tri_idx(q, q, D)] = aqq + t * apq;
        Am[tri_idx(p, q, D)] = R(0);
#pragma unroll
        for (int k = 0; k < D; ++k) {
          if (k == p || k == q) continue;
          const int ikp = k < p ? tri_idx(k, p, D) : tri_idx(p, k, D);
          const int ikq = k < q ? tri_idx(k, q, D) : tri_idx(q, k, D);
          const R akp = Am[ikp], akq = Am[ikq];
          Am[ikp] = c * akp - s * akq;
          Am[ikq] = s * akp + c * akq;
        }
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const R vkp = V[p * D + k], vkq = V[q * D + k];
          V[p * D + k] = c * vkp - s * vkq;
          V[q * D + k] = s * vkp + c * vkq;
        }
      }
  }
}

template <int D>
__device__ __forceinline__ void jacobi_refine64_reg(double (&Am)[D * (D + 1) / 2], double (&V)[D * D],
                                                    const double tol2, const int max_sweeps) {
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    double off = 0, fro = 0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      fro += Am[tri_idx(i, i, D)] * Am[tri_idx(i, i, D)];
#pragma unroll
      for (int j = i + 1; j < D; ++j) off += 2.0 * Am[tri_idx(i, j, D)] * Am[tri_idx(i, j, D)];
    }
    fro += off;
    if (fro == 0.0 || off <= tol2 * fro) break;
    const double nrm = sqrt(fro);
    const double skip = 1e-16 * nrm;
    const double inv = 1.0 / nrm;
#pragma unroll
    for (int p = 0; p < D - 1; ++p)
#pragma unroll
      for (int q = p + 1; q < D; ++q) {
        const double apq = Am[tri_idx(p, q, D)];
        if (fabs(apq) <= skip) continue;
        const double app = Am[tri_idx(p, p, D)], aqq = Am[tri_idx(q, q, D)];
        const float apq32 = (float)(apq * inv), dd32 = (float)((aqq - app) * inv);
        const float tau = dd32 / (2.f * apq32);
        const float t32 = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
        const double t = (double)t32;
        const double c = rsqrt_refined(1.0 + t * t), s = t * c;
        const double cc = c * c, ss = s * s, cs = c * s;
        Am[tri_idx(p, p, D)] = cc * app - 2.0 * cs * apq + ss * aqq;
        Am[tri_idx(q, q, D)] = ss * app + 2.0 * cs * apq + cc * aqq;
        Am[tri_idx(p, q, D)] = cs * (app - aqq) + (cc - ss) * apq;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          if (k == p || k == q) continue;
          const int ikp = k < p ? tri_idx(k, p, D) : tri_idx(p, k, D);
          const int ikq = k < q ? tri_idx(k, q, D) : tri_idx(q, k, D);
          const double akp = Am[ikp], akq = Am[ikq];
          Am[ikp] = c * akp - s * akq;
          Am[ikq] = s * akp + c * akq;
        }
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const double vkp = V[p * D + k], vkq = V[q * D + k];
          V[p * D + k] = c * vkp - s * vkq;
          V[q * D + k] = s * vkp + c * vkq;
        }
      }
  }
}

// PSD projection of a small symmetric D x D (packed upper triangle) in
// registers: FP32 Jacobi, FP64 Gram-Schmidt, A = V^T B V, FP64 sweeps, then
// B+ from the side with fewer eigenpairs (as k_hess_proj).
template <int D>
__device__ __forceinline__ void psd_small(const double (&B)[D * (D + 1) / 2], double (&P)[D * (D + 1) / 2]) {
  constexpr int NP = D * (D + 1) / 2;
  double mx = 0.0;
#pragma unroll
  for (int e = 0; e < NP; ++e) mx = fmax(mx, fabs(B[e]));
  if (mx == 0.0) {
#pragma unroll
    for (int e = 0; e < NP; ++e) P[e] = 0.0;
    return;
  }
  double V[D * D], Am[NP];
  {
    float A32[NP], V32[D * D];
    const double inv = 1.0 / mx;
#pragma unroll
    for (int e = 0; e < NP; ++e) A32[e] = (float)(B[e] * inv);
#pragma unroll
    for (int e = 0; e < D * D; ++e) V32[e] = (e % (D + 1) == 0) ? 1.f : 0.f;
    jacobi_reg<float, D>(A32, V32, PROJ_FP32_TOL2, 12);
#pragma unroll
    for (int k = 0; k < D; ++k) {
#pragma unroll
      for (int i = 0; i < D; ++i) V[k * D + i] = (double)V32[k * D + i];
#pragma unroll
      for (int j = 0; j < k; ++j) {
        double dp = 0.0;
#pragma unroll
        for (int i = 0; i < D; ++i) dp += V[j * D + i] * V[k * D + i];
#pragma unroll
        for (int i = 0; i < D; ++i) V[k * D + i] -= dp * V[j * D + i];
      }
      double nn = 0.0;
#pragma unroll
      for (int i = 0; i < D; ++i) nn += V[k * D + i] * V[k * D + i];
      nn = rsqrt_refined(nn);
#pragma unroll
      for (int i = 0; i < D; ++i) V[k * D + i] *= nn;
    }
  }
#pragma unroll
  for (int l = 0; l < D; ++l) {
    double t[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      double v = 0.0;
#pragma unroll
      for (int j = 0; j < D; ++j) v += B[i <= j ? tri_idx(i, j, D) : tri_idx(j, i, D)] * V[l * D + j];
      t[i] = v;
    }
#pragma unroll
    for (int k = 0; k <= l; ++k) {
      double v = 0.0;
#pragma unroll
      for (int i = 0; i < D; ++i) v += V[k * D + i] * t[i];
      Am[tri_idx(k, l, D)] = v;
    }
  }
  jacobi_refine64_reg<D>(Am, V, 1e-28, 12);
  double lam[D];
  int npos = 0, nneg = 0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    lam[k] = Am[tri_idx(k, k, D)];
    npos += lam[k] > 0.0;
    nneg += lam[k] < 0.0;
  }
  const bool from_b = nneg < npos;
#pragma unroll
  for (int e = 0; e < NP; ++e) P[e] = from_b ? B[e] : 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const double wk = from_b ? (lam[k] < 0.0 ? -lam[k] : 0.0) : (lam[k] > 0.0 ? lam[k] : 0.0);
    if (wk == 0.0) continue;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const double wi = wk * V[k * D + i];
#pragma unroll
      for (int j = i; j < D; ++j) P[tri_idx(i, j, D)] += wi * V[k * D + j];
    }
  }
}

// PSD projection of a symmetric 2x2 [[a, b], [b, c]] in closed form: with
// h = (a - c)/2, r = hypot(h, b), m = (a + c)/2 the eigenvalues are m +- r;
// if one is positive and one negative the result is l+ v v^T with
// v v^T = [[h + r, b], [b, r - h]] / (2 r), each entry formed without
// cancellation (h + r = b^2 / (r - h) when h < 0, and the mirror case), and
// l+ = m + r or det / (m - r) whichever avoids cancellation.
__device__ __forceinline__ void psd2(double a, double b, double c, double& pa, double& pb, double& pc) {
  const double h = 0.5 * (a - c), m = 0.5 * (a + c);
  const double r = hypot(h, b);
  const double lp = m + r, lm = m - r;
  if (lm >= 0.0) {
    pa = a;
    pb = b;
    pc = c;
    return;
  }
  if (lp <= 0.0) {
    pa = pb = pc = 0.0;
    return;
  }
  const double det = fma(a, c, -b * b);
  const double lpos = m >= 0.0 ? lp : det / lm;
  const double hp = h >= 0.0 ? h + r : (b * b) / (r - h);
  const double hm = h >= 0.0 ? (b * b) / (r + h) : r - h;
  const double sc = lpos / (2.0 * r);
  pa = sc * hp;
  pb = sc * b;
  pc = sc * hm;
}

// Stage (d), part 2 for point-edge pairs queued in their own frame.  The
// in-plane 4x4 block [[0, p r^T], [r p^T, Y]] (x of both reduced points, then
// y) has the null vector (p_perp, 0) and equals Q T Q^T with
// Q = [[p/|p|, 0], [0, I]] (orthonormal columns) and the 3x3
// T = [[0, |p| r^T], [|p| r, Y]], so its projection is Q T+ Q^T: a 3x3
// eigenproblem instead of a 4x4.  The 2x2 block is projected in closed form,
// the 6x6 result rotated back block by block (B+ = (I x R) B'+ (I x R)^T) and
// scattered as in k_hess_proj<6>.
__device__ __forceinline__ void proj_pe_block(const HessArgs& A, int block) {
  const int64_t w = (int64_t)block * 128 + threadIdx.x;
  if (w >= (int64_t)*A.n4) return;
  const uint32_t a = A.slot4[w];
  double q[10], R[9];
#pragma unroll
  for (int e = 0; e < 10; ++e) q[e] = A.B4[(size_t)e * A.cap + w];
#pragma unroll
  for (int k = 0; k < 9; ++k) R[k] = A.B4[(size_t)(10 + k) * A.cap + w];
  const double pn = sqrt(q[0] * q[0] + q[1] * q[1]);
  double ph0 = 1.0, ph1 = 0.0;
  if (pn > 0.0) {
    const double ipn = 1.0 / pn;
    ph0 = q[0] * ipn;
    ph1 = q[1] * ipn;
  }
  const double T[6] = {0.0, pn * q[2], pn * q[3], q[4], q[5], q[6]};
  double Tp[6], p2[3];
  psd_small<3>(T, Tp);
  psd2(q[7], q[8], q[9], p2[0], p2[1], p2[2]);
  // Q T+ Q^T in the order (0x, 0y, 1x, 1y), packed
  const double P4[10] = {ph0 * ph0 * Tp[0], ph0 * Tp[1], ph0 * ph1 * Tp[0], ph0 * Tp[2], Tp[3],
                         ph1 * Tp[1],       Tp[4],       ph1 * ph1 * Tp[0], ph1 * Tp[2], Tp[5]};
  // Back to the three points and to world axes.  Local block (ab, bb) of the
  // reduced matrix: L_ab,bb = [[in-plane 2x2 from P4, 0], [0, e3-e3 entry from
  // p2]]; block (q1, q2) of the points is R L'(q1, q2) R^T with
  // L'(q1, q2) = sum K3[q1][ab] K3[q2][bb] L_ab,bb.  K3's rows are (c, s),
  // (-c, s), (0, -2s), c = 1/sqrt2, s = 1/sqrt6, so with X = L00/2,
  // Y = L11/6, W = L11/3, S = cs (L01 + L10), Dm = cs (L01 - L10),
  // Z = 2cs L01 (cs = 1/sqrt12):
  //   L'00 = X + S + Y, L'11 = X - S + Y, L'22 = 2W,
  //   L'01 = -X + Dm + Y, L'02 = -Z - W, L'12 = Z - W.
  constexpr double cs = 0.28867513459481288225;  // 1/sqrt(12)
  const double L00[2][2] = {{P4[0], P4[1]}, {P4[1], P4[4]}}, L01[2][2] = {{P4[2], P4[3]}, {P4[5], P4[6]}},
               L11[2][2] = {{P4[7], P4[8]}, {P4[8], P4[9]}};
  double Lq[6][2][2], zq[6];  // 00, 11, 22, 01, 02, 12
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const double X = 0.5 * L00[i][j], Y = L11[i][j] * (1.0 / 6.0), W = L11[i][j] * (1.0 / 3.0);
      const double S = cs * (L01[i][j] + L01[j][i]), Dm = cs * (L01[i][j] - L01[j][i]), Z = 2.0 * cs * L01[i][j];
      Lq[0][i][j] = X + S + Y;
      Lq[1][i][j] = X - S + Y;
      Lq[2][i][j] = 2.0 * W;
      Lq[3][i][j] = -X + Dm + Y;
      Lq[4][i][j] = -Z - W;
      Lq[5][i][j] = Z - W;
    }
  {
    const double X = 0.5 * p2[0], Y = p2[2] * (1.0 / 6.0), W = p2[2] * (1.0 / 3.0), S = 2.0 * cs * p2[1],
                 Z = 2.0 * cs * p2[1];
    zq[0] = X + S + Y;
    zq[1] = X - S + Y;
    zq[2] = 2.0 * W;
    zq[3] = -X + Y;
    zq[4] = -Z - W;
    zq[5] = Z - W;
  }
  // world block: E2 A2 E2^T + z e3 e3^T, E2 = (e1, e2) = columns 0, 1 of R
  auto world = [&](const double (&A2)[2][2], double z, double (&w)[9]) {
    double T[3][2];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int bb = 0; bb < 2; ++bb) T[i][bb] = R[3 * i] * A2[0][bb] + R[3 * i + 1] * A2[1][bb];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const double ze = z * R[3 * i + 2];
#pragma unroll
      for (int j = 0; j < 3; ++j) w[3 * i + j] = T[i][0] * R[3 * j] + T[i][1] * R[3 * j + 1] + ze * R[3 * j + 2];
    }
  };
  // scatter: the three points the point-edge type involves, in stencil order
  const uint32_t c = A.aidx[a];
  const Stencil st = stencil_of(A.cand[c], A.ev0, A.ev1, A.tv, A.T);
  const TypeInfo& TI = st.ee ? c_ee_types[A.ctype[c]] : c_pt_types[A.ctype[c]];
  int pts[4], np = 0;
  for (int i = 0; i < 4; ++i) {
    bool used = false;
    for (int mm = 0; mm < 2; ++mm) used |= TI.C[mm][i] != 0;
    if (used) pts[np++] = i;
  }
  const int qa[6] = {0, 1, 2, 0, 0, 1}, qb[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    double blk[9];
    world(Lq[k], zq[k], blk);
    const int r = st.v[pts[qa[k]]], cc = st.v[pts[qb[k]]];
    add_block(A, r, cc, blk, false);
    if (k >= 3) add_block(A, cc, r, blk, true);
  }
}

// the point-edge pairs projected in their own frame, one thread per pair
__global__ void __launch_bounds__(128) k_hess_proj_pe(HessArgs A) { proj_pe_block(A, blockIdx.x); }

// Short queues (a small scene): the warp-per-pair 9x9 projection in blocks
// [0, nb9) and the point-edge pairs in the blocks after them, one launch, so
// that the two independent queues run side by side (both only add into the
// BSR values, atomically) instead of one after the other.
__global__ void __launch_bounds__(PL_THREADS) k_hess_proj_short(HessArgs A, int nb9) {
  static_assert(PL_THREADS == 128, "both halves run 128-thread blocks");
  if ((int)blockIdx.x < nb9) proj_lanes_block(A, blockIdx.x);
  else proj_pe_block(A, blockIdx.x - nb9);
}

__global__ void k_energy_final(int count, const unsigned long long* __restrict__ macc, double* __restrict__ out) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= count) return;
  double e = __longlong_as_double(macc[(size_t)m * MACC_STRIDE + MACC_E]);
  if (macc[(size_t)m * MACC_STRIDE + MACC_STATUS] & CB_DEV_PENETRATION) e = __longlong_as_double(0x7ff0000000000000LL);
  out[m] = e;
}

__global__ void k_macc_reset(int count, unsigned long long* __restrict__ macc, int slot, unsigned long long v) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < count) macc[(size_t)m * MACC_STRIDE + slot] = v;
}

__global__ void k_set_u64(unsigned long long* p, unsigned long long v) { *p = v; }

// One launch for the resets at the start of a barrier pass: the scalar slots
// in sc_mask and, for every member, the accumulator slots in macc_mask.
__global__ void k_pass_reset(unsigned long long* __restrict__ sc, uint32_t sc_mask, int count,
                             unsigned long long* __restrict__ macc, uint32_t macc_mask) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < SC_N && ((sc_mask >> i) & 1u)) sc[i] = 0ull;
  if (i < count)
    for (int k = 0; k < MACC_STRIDE; ++k)
      if ((macc_mask >> k) & 1u) macc[(size_t)i * MACC_STRIDE + k] = 0ull;
}

}  // namespace

__global__ void k_fill_u64(int64_t n, unsigned long long* __restrict__ p, unsigned long long v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

cb_status filter_precompute(cb_scene* s, cudaStream_t st) {
  uint64_t* sc = scalars(s);
  unsigned long long* dmin = (unsigned long long*)(sc + SC_DBAR_MIN_BITS);
  unsigned long long* nf = (unsigned long long*)(sc + SC_NFILT);
  k_set_u64<<<1, 1, 0, cb_count(st)>>>(dmin, 0x7ff0000000000000ull);
  k_set_u64<<<1, 1, 0, cb_count(st)>>>(nf, 0ull);
  // per-component minima, by component label (rods: polyline index; shells: a vertex id)
  CB_TRY(buf_ensure(s->dbar_comp, sizeof(unsigned long long) * (size_t)std::max(1, s->n), st));
  unsigned long long* dcomp = bp<unsigned long long>(s->dbar_comp);
  k_fill_u64<<<cb_grid(std::max(1, s->n)), CB_THREADS, 0, cb_count(st)>>>(std::max(1, s->n), dcomp,
                                                                          0x7ff0000000000000ull);
  if (s->kind == CB_ROD) {
    CB_TRY(buf_ensure(s->S, sizeof(double) * (size_t)s->n, st));
    CB_TRY(buf_ensure(s->win, sizeof(int32_t) * (size_t)std::max(1, s->E), st));
    CB_TRY(buf_ensure(s->wst, sizeof(int32_t) * (size_t)std::max(1, s->E), st));
    k_arclength<<<cb_grid(s->n_rods), CB_THREADS, 0, cb_count(st)>>>(s->n_rods, bp<int32_t>(s->rod_ptr), bp<double>(s->rest),
                                                           s->n, bp<double>(s->S));
    if (s->E > 0)
      k_rod_window<<<cb_grid(s->E), CB_THREADS, 0, cb_count(st)>>>(
          s->E, bp<int32_t>(s->ev0), bp<int32_t>(s->ev1), bp<int32_t>(s->comp), bp<double>(s->S),
          bp<double>(s->rest), s->n, bp<int32_t>(s->rlast), s->a, bp<int32_t>(s->win), bp<int32_t>(s->wst), dmin,
          nf, dcomp);
    CB_CUDA(cudaGetLastError());
    uint64_t h[2];
    CB_TRY(read_scalars(s, SC_DBAR_MIN_BITS, 1, &h[0], st));
    CB_TRY(read_scalars(s, SC_NFILT, 1, &h[1], st));
    memcpy(&s->dbar_min, &h[0], 8);
    s->n_frest = (int64_t)h[1];
  } else {
    // rest broad phase at the full activation, then rest distances below a (a
    // geodesic distance is at least the 3D one, so the same candidates serve it)
    int64_t nr = 0;
    ScopedBuf rcs(st);
    DevBuf& rc = rcs.b;
    // positions of the reference distances: the flat pattern when given, else the rest shape
    const double* rf = s->ruv.p ? bp<double>(s->ruv) : bp<double>(s->rest);
    CB_TRY(broad_phase(s, s->bw, rf, nullptr, false, true, rc, &nr, st));
    if (nr > 0) {
      ScopedBuf flags(st), poss(st), dbars(st);
      DevBuf &flag = flags.b, &pos = poss.b, &dbar = dbars.b;
      CB_TRY(buf_ensure(flag, sizeof(uint32_t) * (size_t)nr, st));
      CB_TRY(buf_ensure(pos, sizeof(uint32_t) * ((size_t)nr + 1), st));
      CB_TRY(buf_ensure(dbar, sizeof(double) * (size_t)nr, st));
      CB_TRY(buf_ensure(s->scan_tmp, sizeof(uint64_t) * (size_t)(cbp::scan_tmp_elems(nr) + 8), st));
      if (s->geodesic) {
        CB_TRY(geo_rest_dbar(s, bp<uint64_t>(rc), nr, bp<uint32_t>(flag), bp<double>(dbar), dmin, dcomp, st));
      } else {
        k_rest_filter<<<cb_grid(nr), CB_THREADS, 0, cb_count(st)>>>(nr, bp<uint64_t>(rc), bp<int32_t>(s->ev0),
                                                          bp<int32_t>(s->ev1), bp<int32_t>(s->tv), s->T,
                                                          bp<int32_t>(s->comp), rf, s->n, s->a,
                                                          bp<uint32_t>(flag), bp<double>(dbar), dmin, dcomp);
      }
      uint32_t* tot = (uint32_t*)(sc + SC_COUNT1);
      cbp::exclusive_scan<uint32_t, uint32_t>(bp<uint32_t>(flag), bp<uint32_t>(pos), nr, bp<uint32_t>(s->scan_tmp),
                                              tot, st);
      uint64_t h[2];
      CB_CUDA(cudaGetLastError());
      CB_TRY(read_scalars(s, SC_COUNT1, 1, &h[0], st));
      const int64_t nf_ = (int64_t)(uint32_t)h[0];
      CB_TRY(buf_ensure(s->frest, sizeof(uint64_t) * (size_t)std::max<int64_t>(1, nf_), st));
      CB_TRY(buf_ensure(s->frest_dbar, sizeof(double) * (size_t)std::max<int64_t>(1, nf_), st));
      cbp::k_compact<uint64_t, uint32_t><<<cb_grid(nr), CB_THREADS, 0, cb_count(st)>>>(bp<uint64_t>(rc), bp<uint32_t>(flag),
                                                                         bp<uint32_t>(pos), nr, bp<uint64_t>(s->frest));
      cbp::k_compact<double, uint32_t><<<cb_grid(nr), CB_THREADS, 0, cb_count(st)>>>(bp<double>(dbar), bp<uint32_t>(flag),
                                                                       bp<uint32_t>(pos), nr,
                                                                       bp<double>(s->frest_dbar));
      CB_CUDA(cudaGetLastError());
      CB_TRY(read_scalars(s, SC_DBAR_MIN_BITS, 1, &h[1], st));
      memcpy(&s->dbar_min, &h[1], 8);
      s->n_frest = nf_;
    } else {
      s->dbar_min = INFINITY;
      s->n_frest = 0;
    }
  }
  if (s->n_frest > 0 && !(s->dbar_min > 0.0)) return CB_ERR_DEGENERATE;
  s->dbar_fmax = s->dbar_min;
  if (s->hmp.size() == 1 && s->hmp[0].per_comp) {
    std::vector<unsigned long long> h((size_t)std::max(1, s->n));
    CB_CUDA(cudaMemcpyAsync(h.data(), dcomp, sizeof(unsigned long long) * h.size(), cudaMemcpyDeviceToHost, st));
    CB_CUDA(cudaStreamSynchronize(st));
    double mx = -INFINITY;
    for (unsigned long long b : h) {
      double v;
      memcpy(&v, &b, 8);
      if (std::isfinite(v)) mx = std::max(mx, v);
    }
    if (std::isfinite(mx)) s->dbar_fmax = mx;
  }
  return CB_OK;
}

// Row offsets of the sorted rest-filter table: row[r] = first index whose key
// is at or above (type, r, 0), for r = 0..nrows (row[nrows] ends the type).
__global__ void k_frest_rows(int64_t nrows, uint32_t type, const uint64_t* __restrict__ frest, int64_t nf,
                             uint32_t* __restrict__ row) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r > nrows) return;
  const uint64_t bound = ((uint64_t)type << 62) | ((uint64_t)r << 31);
  int64_t lo = 0, hi = nf;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (frest[mid] < bound) lo = mid + 1;
    else hi = mid;
  }
  row[r] = (uint32_t)lo;
}

// the partner index j of every rest-filtered key (the low 31 bits)
__global__ void k_frest_j(int64_t nf, const uint64_t* __restrict__ frest, uint32_t* __restrict__ fj) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nf) fj[k] = cb_key_j(frest[k]);
}

cb_status frest_rows_build(cb_scene* s, cudaStream_t st) {
  if (s->kind != CB_SHELL || s->n_frest <= 0) return CB_OK;
  CB_TRY(buf_ensure(s->frest_j, sizeof(uint32_t) * (size_t)s->n_frest, st));
  k_frest_j<<<cb_grid(s->n_frest), CB_THREADS, 0, cb_count(st)>>>(s->n_frest, bp<uint64_t>(s->frest),
                                                                  bp<uint32_t>(s->frest_j));
  CB_TRY(buf_ensure(s->frow_pt, sizeof(uint32_t) * ((size_t)s->n + 1), st));
  CB_TRY(buf_ensure(s->frow_ee, sizeof(uint32_t) * ((size_t)s->E + 1), st));
  k_frest_rows<<<cb_grid((int64_t)s->n + 1), CB_THREADS, 0, cb_count(st)>>>(s->n, CB_KEY_PT, bp<uint64_t>(s->frest),
                                                                           s->n_frest, bp<uint32_t>(s->frow_pt));
  k_frest_rows<<<cb_grid((int64_t)s->E + 1), CB_THREADS, 0, cb_count(st)>>>(s->E, CB_KEY_EE, bp<uint64_t>(s->frest),
                                                                           s->n_frest, bp<uint32_t>(s->frow_ee));
  CB_CUDA(cudaGetLastError());
  return CB_OK;
}

cb_status filter_apply(cb_scene* s, cudaStream_t st) {
  const int64_t nc = s->n_cand;
  CB_TRY(buf_ensure(s->klass, (size_t)std::max<int64_t>(1, nc), st));
  unsigned long long* nf = (unsigned long long*)(scalars(s) + SC_NFILT);
  k_set_u64<<<1, 1, 0, cb_count(st)>>>(nf, 0ull);
  s->n_dropped = 0;
  if (nc == 0) return CB_OK;
  const bool ps = s->per_stencil();
  unsigned long long* ndrop = (unsigned long long*)(scalars(s) + SC_COUNT1);
  if (ps) {
    if (!s->bw.box_raw.p) return CB_ERR_ARG;  // the candidates came from before the mode was set
    k_set_u64<<<1, 1, 0, cb_count(st)>>>(ndrop, 0ull);
  }
  const StencilArgs SA{ps ? bp<double>(s->bw.box_raw) : nullptr, bp<unsigned long long>(s->dbar_comp),
                       bp<int32_t>(s->comp), ndrop};
  if (s->kind == CB_ROD)
    k_filter_rod<<<cb_grid(nc), CB_THREADS, 0, cb_count(st)>>>(
        nc, bp<uint64_t>(s->cand), bp<int32_t>(s->ev0), bp<int32_t>(s->comp), bp<int32_t>(s->win),
        bp<int32_t>(s->wst), bp<int32_t>(s->rloop), bp<int32_t>(s->vsc), bp<MemberParams>(s->mp),
        bp<uint8_t>(s->klass), nf, SA);
  else
    k_filter_shell<<<cb_grid(nc), CB_THREADS, 0, cb_count(st)>>>(
        nc, bp<uint64_t>(s->cand), bp<uint32_t>(s->frest_j), bp<uint32_t>(s->frow_pt), bp<uint32_t>(s->frow_ee),
        s->n_frest, bp<int32_t>(s->ev0), bp<int32_t>(s->vsc), bp<MemberParams>(s->mp), bp<uint8_t>(s->klass), nf,
        s->n, s->T, SA);
  CB_CUDA(cudaGetLastError());
  if (!ps) return CB_OK;
  // per-stencil activation: drop the class-F candidates outside their own width
  uint64_t hd;
  CB_TRY(read_scalars(s, SC_COUNT1, 1, &hd, st));
  s->n_dropped = (int64_t)hd;
  if (hd == 0) return CB_OK;
  CB_TRY(buf_ensure(s->cflag, sizeof(uint32_t) * (size_t)nc, st));
  CB_TRY(buf_ensure(s->cpos, sizeof(uint32_t) * ((size_t)nc + 1), st));
  CB_TRY(buf_ensure(s->scan_tmp, sizeof(uint64_t) * (size_t)(cbp::scan_tmp_elems(nc) + 8), st));
  CB_TRY(buf_ensure(s->cand_alt, sizeof(uint64_t) * (size_t)nc, st));
  CB_TRY(buf_ensure(s->klass_alt, (size_t)nc, st));
  k_keep_flag<<<cb_grid(nc), CB_THREADS, 0, cb_count(st)>>>(nc, bp<uint8_t>(s->klass), bp<uint32_t>(s->cflag));
  cbp::exclusive_scan<uint32_t, uint32_t>(bp<uint32_t>(s->cflag), bp<uint32_t>(s->cpos), nc,
                                          bp<uint32_t>(s->scan_tmp), (uint32_t*)nullptr, st);
  k_keep_write<<<cb_grid(nc), CB_THREADS, 0, cb_count(st)>>>(nc, bp<uint64_t>(s->cand), bp<uint8_t>(s->klass),
                                                            bp<uint32_t>(s->cflag), bp<uint32_t>(s->cpos),
                                                            bp<uint64_t>(s->cand_alt), bp<uint8_t>(s->klass_alt));
  CB_CUDA(cudaGetLastError());
  std::swap(s->cand, s->cand_alt);
  std::swap(s->klass, s->klass_alt);
  s->n_cand = nc - s->n_dropped;
  return CB_OK;
}

cb_status to_f32(cb_scene* s, const double* v, const double* cx, DevBuf& out, cudaStream_t st) {
  CB_TRY(buf_ensure(out, sizeof(float4) * (size_t)std::max(1, s->n), st));
  k_to_f32<<<cb_grid(s->n), CB_THREADS, 0, cb_count(st)>>>(s->n, v, cx, bp<int32_t>(s->vsc), bp<float4>(out));
  CB_CUDA(cudaGetLastError());
  return CB_OK;
}

static int bits_for(int64_t v) {
  int b = 1;
  while ((1ll << b) <= v) ++b;
  return b;
}

cb_status barrier_run(cb_scene* s, const double* x, double* energy, double* grad, bool energy_only,
                      cudaStream_t st) {
  const int64_t nc = s->n_cand;
  uint64_t* sc = scalars(s);
  unsigned long long* status = (unsigned long long*)(sc + SC_STATUS);
  unsigned long long* ncore = (unsigned long long*)(sc + SC_NCORE);
  unsigned long long* macc = bp<unsigned long long>(s->macc);
  const int M = s->count;
  s->cd_split = false;
  // the pass's counters (the queue lengths stay readable until the next pass)
  {
    const uint32_t scm = (1u << SC_NCORE) | (1u << SC_NLIST) | (1u << SC_KSPLIT) | (1u << SC_NMOLL) |
                         (1u << SC_N9) | (1u << SC_N6) | (1u << SC_N4);
    k_pass_reset<<<cb_grid(std::max(M, (int)SC_N)), CB_THREADS, 0, cb_count(st)>>>(
        (unsigned long long*)sc, scm, M, macc, (1u << MACC_E) | (1u << MACC_STATUS));
  }
  if (grad) CB_CUDA(cudaMemsetAsync(grad, 0, sizeof(double) * 3 * (size_t)s->n, st));
  s->n_active = 0;
  s->nnzb = 0;
  CB_TRY(buf_ensure(s->bsr_row, sizeof(int32_t) * ((size_t)s->n + 1), st));
  CB_CUDA(cudaMemsetAsync(s->bsr_row.p, 0, sizeof(int32_t) * ((size_t)s->n + 1), st));
  if (nc > 0) {
    CB_TRY(buf_ensure(s->cd, sizeof(double) * (size_t)nc, st));
    CB_TRY(buf_ensure(s->ctype, (size_t)nc, st));
    CB_TRY(buf_ensure(s->ccls, (size_t)nc, st));
    CB_TRY(buf_ensure(s->cflag, sizeof(uint32_t) * (size_t)nc, st));
    CB_TRY(buf_ensure(s->cpos, sizeof(uint32_t) * ((size_t)nc + 1), st));
    CB_TRY(buf_ensure(s->scan_tmp, sizeof(uint64_t) * (size_t)(cbp::scan_tmp_elems(nc) + 8), st));
    CB_TRY(to_f32(s, x, bp<double>(s->bw.cx), s->xf, st));
    CB_TRY(buf_ensure(s->dlist, sizeof(uint32_t) * (size_t)nc, st));
    unsigned int* nl = (unsigned int*)(sc + SC_NLIST);
    k_distance_screen<<<cb_grid(nc), CB_THREADS, 0, cb_count(st)>>>(
        nc, bp<uint64_t>(s->cand), bp<uint8_t>(s->klass), bp<int32_t>(s->ev0), bp<int32_t>(s->ev1),
        bp<int32_t>(s->tv), s->T, bp<float4>(s->xf), bp<double>(s->bw.cx), bp<int32_t>(s->vsc),
        bp<MemberParams>(s->mp), s->n, bp<double>(s->cd),
        bp<int8_t>(s->ctype), bp<uint8_t>(s->ccls), bp<uint32_t>(s->cflag), bp<uint32_t>(s->dlist), nl);
    (energy_only ? k_distance_exact<true> : k_distance_exact<false>)<<<std::min<int64_t>(cb_grid(nc), (int64_t)s->n_sms * 16), CB_THREADS, 0, cb_count(st)>>>(
        bp<uint32_t>(s->dlist), nc, nl, bp<uint64_t>(s->cand), bp<uint8_t>(s->klass), bp<int32_t>(s->ev0),
        bp<int32_t>(s->ev1), bp<int32_t>(s->tv), s->T, x, s->n, bp<int32_t>(s->vsc), bp<MemberParams>(s->mp),
        bp<double>(s->cd), bp<int8_t>(s->ctype), bp<uint8_t>(s->ccls), bp<uint32_t>(s->cflag), status, ncore,
        macc, bp<int32_t>(s->comp), bp<unsigned long long>(s->dbar_comp), bp<double>(s->elen2));
    if (energy_only) {
      if (energy) k_energy_final<<<cb_grid(M), CB_THREADS, 0, cb_count(st)>>>(M, macc, energy);
      CB_CUDA(cudaGetLastError());
      return CB_OK;
    }
    uint32_t* tot = (uint32_t*)(sc + SC_COUNT1);
    cbp::exclusive_scan<uint32_t, uint32_t>(bp<uint32_t>(s->cflag), bp<uint32_t>(s->cpos), nc,
                                            bp<uint32_t>(s->scan_tmp), tot, st);
    CB_CUDA(cudaGetLastError());
    uint64_t h;
    CB_TRY(read_scalars(s, SC_COUNT1, 1, &h, st));
    s->n_active = (int64_t)(uint32_t)h;
    // end of stage (c): distances, classes and the active set
    if (s->timing) cudaEventRecord(s->ev[12], st);
    s->cd_split = true;
  }
  const int64_t na = s->n_active;
  if (na > 0) {
    CB_TRY(buf_ensure(s->aidx, sizeof(uint32_t) * (size_t)na, st));
    k_active_compact<<<cb_grid(nc), CB_THREADS, 0, cb_count(st)>>>(nc, bp<uint32_t>(s->cflag), bp<uint32_t>(s->cpos),
                                                         bp<uint32_t>(s->aidx));
    // BSR pattern: sorted unique (row, col) of the 16 blocks of every active stencil
    int64_t m = 16 * na;  // capacity; the keys actually sorted are counted by k_block_keys
    const int bn = bits_for(s->n);
    for (int b = 0; b < 2; ++b) CB_TRY(buf_ensure(s->bkey[b], sizeof(uint64_t) * (size_t)m, st));
    CB_TRY(buf_ensure(s->bflag, sizeof(uint32_t) * (size_t)m, st));
    CB_TRY(buf_ensure(s->bpos, sizeof(uint32_t) * ((size_t)m + 1), st));
    CB_TRY(buf_ensure(s->hist, sizeof(uint32_t) * (size_t)cbp::radix_hist_elems(m), st));
    CB_TRY(buf_ensure(s->scan_tmp, sizeof(uint64_t) * (size_t)(cbp::scan_tmp_elems(cbp::radix_hist_elems(m)) +
                                                                cbp::scan_tmp_elems(m) + 8),
                      st));
    unsigned int* nbk = (unsigned int*)(sc + SC_NBK);
    CB_CUDA(cudaMemsetAsync(nbk, 0, sizeof(unsigned int), st));
    {
      const int smem = BK_SLOTS * (int)sizeof(unsigned long long);
      CB_CUDA(cudaFuncSetAttribute(k_block_keys, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
      k_block_keys<<<(int)((na + BK_PAIRS - 1) / BK_PAIRS), BK_PAIRS, smem, cb_count(st)>>>(
          na, bp<uint32_t>(s->aidx), bp<uint64_t>(s->cand), bp<int32_t>(s->ev0), bp<int32_t>(s->ev1),
          bp<int32_t>(s->tv), s->T, bn, bp<uint64_t>(s->bkey[0]), nbk);
      CB_CUDA(cudaGetLastError());
    }
    uint64_t hm;
    CB_TRY(read_scalars(s, SC_NBK, 1, &hm, st));
    m = (int64_t)(uint32_t)hm;  // keys left after the per-run sets (at most 16 na)
    int r = cbp::radix_sort<uint64_t, uint32_t, false>(bp<uint64_t>(s->bkey[0]), nullptr, bp<uint64_t>(s->bkey[1]),
                                                       nullptr, m, 0, 2 * bn, bp<uint32_t>(s->hist),
                                                       bp<uint32_t>(s->scan_tmp), st);
    const uint64_t* bk = bp<uint64_t>(s->bkey[r]);
    k_unique_flag<<<cb_grid(m), CB_THREADS, 0, cb_count(st)>>>(m, bk, bp<uint32_t>(s->bflag));
    uint32_t* tot = (uint32_t*)(sc + SC_COUNT1);
    cbp::exclusive_scan<uint32_t, uint32_t>(bp<uint32_t>(s->bflag), bp<uint32_t>(s->bpos), m,
                                            bp<uint32_t>(s->scan_tmp), tot, st);
    CB_CUDA(cudaGetLastError());
    uint64_t h;
    CB_TRY(read_scalars(s, SC_COUNT1, 1, &h, st));
    s->nnzb = (int64_t)(uint32_t)h;
    CB_TRY(buf_ensure(s->bsr_col, sizeof(int32_t) * (size_t)s->nnzb, st));
    CB_TRY(buf_ensure(s->bsr_val, sizeof(double) * 9 * (size_t)s->nnzb, st));
    CB_TRY(buf_ensure(s->row_cnt, sizeof(uint32_t) * ((size_t)s->n + 1), st));
    CB_CUDA(cudaMemsetAsync(s->row_cnt.p, 0, sizeof(uint32_t) * ((size_t)s->n + 1), st));
    CB_CUDA(cudaMemsetAsync(s->bsr_val.p, 0, sizeof(double) * 9 * (size_t)s->nnzb, st));
    k_unique_write<<<cb_grid(m), CB_THREADS, 0, cb_count(st)>>>(m, bk, bp<uint32_t>(s->bflag), bp<uint32_t>(s->bpos), bn,
                                                      bp<int32_t>(s->bsr_col), bp<uint32_t>(s->row_cnt));
    cbp::exclusive_scan<uint32_t, int32_t>(bp<uint32_t>(s->row_cnt), bp<int32_t>(s->bsr_row), (int64_t)s->n + 1,
                                           (int32_t*)bp<uint32_t>(s->scan_tmp), (int32_t*)nullptr, st);
    CB_TRY(buf_ensure(s->horder, sizeof(uint32_t) * (size_t)na, st));
    bool mollify = false;
    for (const MemberParams& mpm : s->hmp) mollify |= mpm.mollify != 0;
    MollArgs MA{};
    if (mollify) {
      CB_TRY(buf_ensure(s->hmoll, (size_t)na, st));
      CB_TRY(buf_ensure(s->mlist, sizeof(uint32_t) * (size_t)na, st));
      MA = MollArgs{x, s->n, bp<int32_t>(s->ev0), bp<int32_t>(s->ev1), bp<int32_t>(s->vsc),
                    bp<MemberParams>(s->mp), bp<double>(s->elen2), bp<uint8_t>(s->hmoll),
                    bp<uint32_t>(s->mlist), (unsigned*)(sc + SC_NMOLL)};
    }
    k_kind_split<<<cb_grid(na), CB_THREADS, 0, cb_count(st)>>>(na, bp<uint32_t>(s->aidx), bp<uint64_t>(s->cand),
                                                             bp<int8_t>(s->ctype), bp<uint32_t>(s->horder),
                                                             (unsigned*)(sc + SC_KSPLIT), MA);
    HessArgs A;
    A.na = na;
    A.order = bp<uint32_t>(s->horder);
    A.aidx = bp<uint32_t>(s->aidx);
    A.cand = bp<uint64_t>(s->cand);
    A.cd = bp<double>(s->cd);
    A.ctype = bp<int8_t>(s->ctype);
    A.ccls = bp<uint8_t>(s->ccls);
    A.ev0 = bp<int32_t>(s->ev0);
    A.ev1 = bp<int32_t>(s->ev1);
    A.tv = bp<int32_t>(s->tv);
    A.T = s->T;
    A.x = x;
    A.n = s->n;
    A.vsc = bp<int32_t>(s->vsc);
    A.mp = bp<MemberParams>(s->mp);
    A.macc = macc;
    A.comp = bp<int32_t>(s->comp);
    A.dbar_comp = bp<unsigned long long>(s->dbar_comp);
    A.row_ptr = bp<int32_t>(s->bsr_row);
    A.col = bp<int32_t>(s->bsr_col);
    A.val = bp<double>(s->bsr_val);
    A.grad = grad;
    A.status = status;
    CB_TRY(buf_ensure(s->hB9, sizeof(double) * 45 * (size_t)na, st));
    CB_TRY(buf_ensure(s->hB6, sizeof(double) * 21 * (size_t)na, st));
    CB_TRY(buf_ensure(s->hB4, sizeof(double) * 19 * (size_t)na, st));
    CB_TRY(buf_ensure(s->hslot, sizeof(uint32_t) * 3 * (size_t)na, st));
    A.B9 = bp<double>(s->hB9);
    A.B6 = bp<double>(s->hB6);
    A.B4 = bp<double>(s->hB4);
    A.slot9 = bp<uint32_t>(s->hslot);
    A.slot6 = bp<uint32_t>(s->hslot) + na;
    A.slot4 = bp<uint32_t>(s->hslot) + 2 * na;
    A.n9 = (unsigned int*)(sc + SC_N9);
    A.n6 = (unsigned int*)(sc + SC_N6);
    A.n4 = (unsigned int*)(sc + SC_N4);
    A.cap = na;
    A.hmoll = mollify ? bp<uint8_t>(s->hmoll) : nullptr;
    A.mlist = bp<uint32_t>(s->mlist);
    A.nmoll = (const unsigned*)(sc + SC_NMOLL);
    A.elen2 = bp<double>(s->elen2);
    if (s->timing) cudaEventRecord(s->ev[10], st);
    k_hess_prep<<<cb_grid(na, 128), 128, 0, cb_count(st)>>>(A);
    if (mollify) k_moll_hess<<<cb_grid(na, 128), 128, 0, cb_count(st)>>>(A);
    CB_CUDA(cudaGetLastError());
    // the three queues' lengths stay on the device: every projection kernel
    // reads its own, the point-edge one over a grid for all active pairs, the
    // shared-memory ones over at most one wave of blocks (grid-stride)
    if (na <= PL_MAX_ACTIVE) {
      const int smem = PL_SMEM * (int)sizeof(double) * PL_PAIRS;
      const int nb9 = (int)((na + PL_PAIRS - 1) / PL_PAIRS);
      k_hess_proj_short<<<nb9 + (int)cb_grid(na, 128), PL_THREADS, smem, cb_count(st)>>>(A, nb9);
      CB_CUDA(cudaGetLastError());
    } else {
      k_hess_proj_pe<<<cb_grid(na, 128), 128, 0, cb_count(st)>>>(A);
      CB_TRY(launch_proj<9>(s, A, na, st));
    }
    CB_TRY(launch_proj<6>(s, A, na, st));
    if (s->timing) cudaEventRecord(s->ev[11], st);
    CB_CUDA(cudaGetLastError());
  }
  if (energy) k_energy_final<<<cb_grid(M), CB_THREADS, 0, cb_count(st)>>>(M, macc, energy);
  CB_CUDA(cudaGetLastError());
  return CB_OK;
}
