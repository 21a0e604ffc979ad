// geometry.cuh -- exact FP64 point-triangle / edge-edge distance and its type.
//
// The distance between two stencil primitives is the minimum over their
// points.  Its closed form depends on where the closest points lie (the
// distance "type"); the barrier of Eq. 2-4 is evaluated on it.
//
//  point-triangle (p; t0,t1,t2):
//    0 PP(p,t0) 1 PP(p,t1) 2 PP(p,t2) 3 PE(p,t0t1) 4 PE(p,t1t2) 5 PE(p,t2t0) 6 face
//  edge-edge (a0,a1; b0,b1):
//    0 PP(a0,b0) 1 PP(a0,b1) 2 PP(a1,b0) 3 PP(a1,b1)
//    4 PE(a0,b) 5 PE(a1,b) 6 PE(b0,a) 7 PE(b1,a) 8 line-line interior
//
// Rules (fixed so that every IEEE-754 evaluation gives the same answer):
//  * coordinates are taken relative to the first vertex of the stencil;
//  * point-triangle is "face" iff the triangle is non-degenerate and the
//    projection of p lies strictly inside it; otherwise the nearest of the three
//    point-segment distances;
//  * edge-edge is "interior" iff the edges are not parallel
//    (|u x v|^2 > 1e-20 |u|^2 |v|^2) and the unconstrained closest-point
//    parameters lie strictly inside (0,1)^2; otherwise the nearest of the four
//    point-segment distances;
//  * a point-segment distance is PP at an end when the projection parameter is
//    <= 0 or >= 1, else PE;  ties go to the lowest type id;
//  * squared distances: PP |b-a|^2, PE |(q-e0)x(e1-e0)|^2/|e1-e0|^2,
//    face ((q-t0).n)^2/|n|^2 with n = (t1-t0)x(t2-t0), line-line
//    ((b0-a0).n)^2/|n|^2 with n = (a1-a0)x(b1-b0).
// All arithmetic uses xmul/xadd/xsub/xdiv (no contraction).
#pragma once
#include "common.cuh"

namespace cbg {

__device__ __forceinline__ double d2_pp(d3 a, d3 b) {
  d3 d = sub3(b, a);
  return dot3(d, d);
}
__device__ __forceinline__ double d2_pe(d3 q, d3 e0, d3 e1) {
  d3 u = sub3(e1, e0), w = sub3(q, e0);
  d3 c = cross3(w, u);
  return xdiv(dot3(c, c), dot3(u, u));
}
__device__ __forceinline__ double d2_pf(d3 q, d3 t0, d3 t1, d3 t2) {
  d3 u = sub3(t1, t0), v = sub3(t2, t0);
  d3 n = cross3(u, v);
  d3 w = sub3(q, t0);
  double g = dot3(w, n);
  return xdiv(xmul(g, g), dot3(n, n));
}
__device__ __forceinline__ double d2_ll(d3 a0, d3 a1, d3 b0, d3 b1) {
  d3 u = sub3(a1, a0), v = sub3(b1, b0);
  d3 n = cross3(u, v);
  d3 w = sub3(b0, a0);
  double g = dot3(w, n);
  return xdiv(xmul(g, g), dot3(n, n));
}

// point-segment region: 0 nearest e0, 1 nearest e1, 2 interior
__device__ __forceinline__ int seg_region(d3 q, d3 e0, d3 e1) {
  d3 u = sub3(e1, e0), w = sub3(q, e0);
  double lam = dot3(w, u);
  if (lam <= 0.0) return 0;
  if (lam >= dot3(u, u)) return 1;
  return 2;
}

// squared distance of q to segment e0 e1 given its region r (0: e0, 1: e1,
// 2: interior): the point-point value on the selected end (d2_pp is symmetric
// bit for bit: b - a and a - b differ only in sign), the point-edge value
// computed only when some lane of the warp needs it, so the lanes of a warp
// run one instruction stream whatever their regions
__device__ __forceinline__ double seg_d2(d3 q, d3 e0, d3 e1, int r) {
  const double dpp = d2_pp(q, r == 0 ? e0 : e1);
  double dpe = dpp;
  if (__any_sync(__activemask(), r == 2)) dpe = d2_pe(q, e0, e1);
  return r == 2 ? dpe : dpp;
}

__device__ __forceinline__ void take_min(int& bt, double& bd, int t, double d2) {
  if (d2 < bd || (d2 == bd && t < bt)) {
    bt = t;
    bd = d2;
  }
}

// Local frame of a stencil: X[0] is the first vertex, P[k] = X[k] - X[0].
struct Local {
  d3 P0, P1, P2, P3;
};

__device__ __forceinline__ Local make_local(d3 x0, d3 x1, d3 x2, d3 x3) {
  Local L;
  L.P0 = sub3(x0, x0);
  L.P1 = sub3(x1, x0);
  L.P2 = sub3(x2, x0);
  L.P3 = sub3(x3, x0);
  return L;
}

// squared distance for a fixed type (point-triangle: P0 = q, P1..3 = t0..t2)
__device__ __forceinline__ double pt_d2(const Local& L, int type) {
  switch (type) {
    case 0: return d2_pp(L.P0, L.P1);
    case 1: return d2_pp(L.P0, L.P2);
    case 2: return d2_pp(L.P0, L.P3);
    case 3: return d2_pe(L.P0, L.P1, L.P2);
    case 4: return d2_pe(L.P0, L.P2, L.P3);
    case 5: return d2_pe(L.P0, L.P3, L.P1);
    default: return d2_pf(L.P0, L.P1, L.P2, L.P3);
  }
}

// edge-edge: P0 = a0, P1 = a1, P2 = b0, P3 = b1
__device__ __forceinline__ double ee_d2(const Local& L, int type) {
  switch (type) {
    case 0: return d2_pp(L.P0, L.P2);
    case 1: return d2_pp(L.P0, L.P3);
    case 2: return d2_pp(L.P1, L.P2);
    case 3: return d2_pp(L.P1, L.P3);
    case 4: return d2_pe(L.P0, L.P2, L.P3);
    case 5: return d2_pe(L.P1, L.P2, L.P3);
    case 6: return d2_pe(L.P2, L.P0, L.P1);
    case 7: return d2_pe(L.P3, L.P0, L.P1);
    default: return d2_ll(L.P0, L.P1, L.P2, L.P3);
  }
}

// type and squared distance of a point-triangle stencil
__device__ __forceinline__ int pt_type(const Local& L, double& d2) {
  const d3 Q = L.P0, T0 = L.P1, T1 = L.P2, T2 = L.P3;
  d3 e1 = sub3(T1, T0), e2 = sub3(T2, T0);
  d3 n = cross3(e1, e2);
  double nn = dot3(n, n);
  if (nn > 0.0) {
    double s0 = dot3(cross3(T1, T2), n);
    double s1 = dot3(cross3(T2, T0), n);
    double s2 = dot3(cross3(T0, T1), n);
    if (s0 > 0.0 && s1 > 0.0 && s2 > 0.0) {
      d2 = pt_d2(L, 6);
      return 6;
    }
  }
  int bt = 99;
  double bd = __longlong_as_double(0x7ff0000000000000LL);
  int r, t;
  r = seg_region(Q, T0, T1);
  t = (r == 0) ? 0 : (r == 1) ? 1 : 3;
  take_min(bt, bd, t, seg_d2(Q, T0, T1, r));
  r = seg_region(Q, T1, T2);
  t = (r == 0) ? 1 : (r == 1) ? 2 : 4;
  take_min(bt, bd, t, seg_d2(Q, T1, T2, r));
  r = seg_region(Q, T2, T0);
  t = (r == 0) ? 2 : (r == 1) ? 0 : 5;
  take_min(bt, bd, t, seg_d2(Q, T2, T0, r));
  d2 = bd;
  return bt;
}

__device__ __forceinline__ int ee_type(const Local& L, double& d2) {
  const d3 A0 = L.P0, A1 = L.P1, B0 = L.P2, B1 = L.P3;
  d3 u = sub3(A1, A0), v = sub3(B1, B0), w = sub3(A0, B0);
  d3 cr = cross3(u, v);
  double cc = dot3(cr, cr), uu = dot3(u, u), vv = dot3(v, v);
  if (cc > xmul(xmul(1e-20, uu), vv)) {
    double B = dot3(u, v), D = dot3(u, w), E = dot3(v, w);
    double sN = xsub(xmul(B, E), xmul(vv, D));
    double tN = xsub(xmul(uu, E), xmul(B, D));
    if (sN > 0.0 && sN < cc && tN > 0.0 && tN < cc) {
      d2 = ee_d2(L, 8);
      return 8;
    }
  }
  int bt = 99;
  double bd = __longlong_as_double(0x7ff0000000000000LL);
  int r, t;
  r = seg_region(A0, B0, B1);
  t = (r == 0) ? 0 : (r == 1) ? 1 : 4;
  take_min(bt, bd, t, seg_d2(A0, B0, B1, r));
  r = seg_region(A1, B0, B1);
  t = (r == 0) ? 2 : (r == 1) ? 3 : 5;
  take_min(bt, bd, t, seg_d2(A1, B0, B1, r));
  r = seg_region(B0, A0, A1);
  t = (r == 0) ? 0 : (r == 1) ? 2 : 6;
  take_min(bt, bd, t, seg_d2(B0, A0, A1, r));
  r = seg_region(B1, A0, A1);
  t = (r == 0) ? 1 : (r == 1) ? 3 : 7;
  take_min(bt, bd, t, seg_d2(B1, A0, A1, r));
  d2 = bd;
  return bt;
}

// distance and type of a stencil given its 4 global points
__device__ __forceinline__ int stencil_distance(bool is_ee, d3 x0, d3 x1, d3 x2, d3 x3, double& d) {
  Local L = make_local(x0, x1, x2, x3);
  double d2;
  int t = is_ee ? ee_type(L, d2) : pt_type(L, d2);
  d = __dsqrt_rn(d2);
  return t;
}

}  // namespace cbg
