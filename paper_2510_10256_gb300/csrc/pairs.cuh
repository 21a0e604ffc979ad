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
  int single, core_temp, per_comp, mollify;
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
  P.mollify = m.mollify;
  return P;
}

// IPC's edge-edge mollifier of c = |e0 x e1|^2 with threshold eps:
// m = -c^2/eps^2 + 2c/eps below eps, 1 above, and its first two derivatives
__device__ __forceinline__ void ee_mollifier(double c, double eps, double& m, double& m1, double& m2) {
  if (!(c < eps)) {
    m = 1.0;
    m1 = 0.0;
    m2 = 0.0;
    return;
  }
  const double ie = 1.0 / eps;
  m = -(c * c) * (ie * ie) + 2.0 * c * ie;
  m1 = -2.0 * c * (ie * ie) + 2.0 * ie;
  m2 = -2.0 * (ie * ie);
}

// c = |(a1 - a0) x (b1 - b0)|^2 of an edge-edge stencil and the mollifier's
// threshold 1e-3 |rest e0|^2 |rest e1|^2
__device__ __forceinline__ double ee_cross2(d3 a0, d3 a1, d3 b0, d3 b1) {
  const double ux = a1.x - a0.x, uy = a1.y - a0.y, uz = a1.z - a0.z;
  const double vx = b1.x - b0.x, vy = b1.y - b0.y, vz = b1.z - b0.z;
  const double nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;
  return nx * nx + ny * ny + nz * nz;
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
