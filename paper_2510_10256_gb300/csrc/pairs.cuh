// pairs.cuh -- per-pair pieces shared by the barrier pass (narrow.cu) and the
// lagged friction (friction.cu): a pair key's stencil, the per-class offset
// and width of Eq. 2-4, and the barrier with its first two derivatives.
#pragma once
#include "common.cuh"
#include "scene.cuh"

namespace {

struct Stencil {
  int v[4];
  bool ee;
};

__device__ __forceinline__ Stencil stencil_of(uint64_t key, const int32_t* __restrict__ ev0,
                                              const int32_t* __restrict__ ev1, const int32_t* __restrict__ tv,
                                              int T) {
  Stencil s;
  const uint32_t ty = cb_key_type(key), i = cb_key_i(key), j = cb_key_j(key);
  if (ty == CB_KEY_PT) {
    s.v[0] = (int)i;
    s.v[1] = tv[j];
    s.v[2] = tv[T + j];
    s.v[3] = tv[2 * T + j];
    s.ee = false;
  } else {
    s.v[0] = ev0[i];
    s.v[1] = ev1[i];
    s.v[2] = ev0[j];
    s.v[3] = ev1[j];
    s.ee = true;
  }
  return s;
}

__device__ __forceinline__ d3 load3(const double* __restrict__ x, int n, int v) {
  return mk3(x[v], x[(size_t)n + v], x[2 * (size_t)n + v]);
}

struct PassParams {
  double xi, dhat, a, dbar_min, kappa;
  int single, core_temp, per_comp;
};

__device__ __forceinline__ PassParams member_pass(const MemberParams& m) {
  PassParams P;
  P.xi = m.xi;
  P.dhat = m.dhat;
  P.a = m.a;
  P.dbar_min = m.dbar_min;
  P.kappa = m.kappa;
  P.single = m.single;
  P.core_temp = m.core_temp;
  P.per_comp = m.per_comp;
  return P;
}

// pair parameters: offset xi_p and width dhat_p of a class (0 U, 1 F, 2 C)
// class-F width of a pair whose first vertex is v0: the scene's dbar_min, or
// its component's (CB_DBAR_PER_COMPONENT)
__device__ __forceinline__ double f_width(const PassParams& P, const unsigned long long* __restrict__ dbar_comp,
                                          const int32_t* __restrict__ comp, int v0) {
  return P.per_comp ? __longlong_as_double((long long)dbar_comp[comp[v0]]) : P.dbar_min;
}

// offset and width of a pair of class k (U 0, F 1, C 2); fw: its class-F width
__device__ __forceinline__ void pair_params(const PassParams& P, int k, double fw, double& xi_p, double& dh_p) {
  if (k == 1) {
    xi_p = 0.0;
    dh_p = fw;
  } else if (k == 2 || P.single) {
    xi_p = 0.0;
    dh_p = P.a;
  } else {
    xi_p = P.xi;
    dh_p = P.dhat;
  }
}

// The IPC barrier of Eq. 2-4 in y = d - xi_p with width dh:
//   b = -(y - dh)^2 log(y / dh) for 0 < y < dh, and its first two derivatives.
__device__ __forceinline__ double barrier_b(double y, double dh) {
  const double r = y - dh;
  return -(r * r) * log(y / dh);
}
__device__ __forceinline__ void barrier_b012(double y, double dh, double& b, double& b1, double& b2) {
  const double r = y - dh, l = log(y / dh), iy = 1.0 / y;
  b = -(r * r) * l;
  b1 = -2.0 * r * l - (r * r) * iy;
  b2 = -2.0 * l - 4.0 * r * iy + (r * r) * (iy * iy);
}

}  // namespace
