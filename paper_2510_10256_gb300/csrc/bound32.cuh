// bound32.cuh -- rigorous FP32 lower bound of a stencil's distance.
//
// For two convex point sets A and B and any direction a != 0,
//   dist(A, B) >= (min_{p in A} a.p - max_{q in B} a.q) / |a|
// (the slab between the two supporting planes separates them).  The bound is
// tight when a joins the closest points, so a is taken from an approximate
// FP32 closest-point computation; its accuracy only affects tightness, never
// validity.  The support values are extremes over the primitives' vertices
// (point-triangle: A = {p}, B = {t0, t1, t2}; edge-edge: the two segments).
//
// Rounding is accounted for explicitly (u = 2^-24, every term scaled by 4):
//  * positions are FP32 copies of (x - c) for a scene centre c, so each
//    vertex is off by at most sqrt(3) u X with X = max |x - c|, and the
//    distance by at most twice that;
//  * the local frame (vertex 0 subtracted in FP32) moves vertices by at most
//    sqrt(3) u R, R = max local |coordinate|;
//  * each 3-term dot product a.p errs by at most 3 u sum |a_k p_k| <= 3 u |a|_1 R;
//    |a| by at most 4 u relative.
// Callers compare the bound against thresholds with a further 1e-12 relative
// margin for the rounding of the FP64 decision itself.
#pragma once
#include "common.cuh"

namespace cbb {

struct f3 {
  float x, y, z;
};
__device__ __forceinline__ f3 fsub3(f3 a, f3 b) { return f3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ f3 fadd3(f3 a, f3 b) { return f3{a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ f3 fscale3(f3 a, float s) { return f3{a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ float fdot3(f3 a, f3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float fclamp01(float v) { return fminf(fmaxf(v, 0.f), 1.f); }
__device__ __forceinline__ float fmaxabs3(f3 a) { return fmaxf(fabsf(a.x), fmaxf(fabsf(a.y), fabsf(a.z))); }

// approximate closest point of triangle (a, b, c) to the origin, by Voronoi
// regions of the vertices, edges and face
__device__ __forceinline__ f3 closest_on_triangle(f3 a, f3 b, f3 c) {
  const f3 ab = fsub3(b, a), ac = fsub3(c, a);
  const f3 ap = fscale3(a, -1.f);
  const float d1 = fdot3(ab, ap), d2 = fdot3(ac, ap);
  if (d1 <= 0.f && d2 <= 0.f) return a;
  const f3 bp = fscale3(b, -1.f);
  const float d3 = fdot3(ab, bp), d4 = fdot3(ac, bp);
  if (d3 >= 0.f && d4 <= d3) return b;
  const float vc = d1 * d4 - d3 * d2;
  if (vc <= 0.f && d1 >= 0.f && d3 <= 0.f) return fadd3(a, fscale3(ab, d1 / (d1 - d3)));
  const f3 cp = fscale3(c, -1.f);
  const float d5 = fdot3(ab, cp), d6 = fdot3(ac, cp);
  if (d6 >= 0.f && d5 <= d6) return c;
  const float vb = d5 * d2 - d1 * d6;
  if (vb <= 0.f && d2 >= 0.f && d6 <= 0.f) return fadd3(a, fscale3(ac, d2 / (d2 - d6)));
  const float va = d3 * d6 - d5 * d4;
  if (va <= 0.f && (d4 - d3) >= 0.f && (d5 - d6) >= 0.f)
    return fadd3(b, fscale3(fsub3(c, b), (d4 - d3) / ((d4 - d3) + (d5 - d6))));
  const float den = 1.f / (va + vb + vc);
  return fadd3(a, fadd3(fscale3(ab, vb * den), fscale3(ac, vc * den)));
}

// approximate closest points of segments (p0, p1) and (q0, q1)
__device__ __forceinline__ void closest_on_segments(f3 p0, f3 p1, f3 q0, f3 q1, f3& c1, f3& c2) {
  const f3 d1 = fsub3(p1, p0), d2 = fsub3(q1, q0), r = fsub3(p0, q0);
  const float a = fdot3(d1, d1), e = fdot3(d2, d2), f = fdot3(d2, r);
  float s, t;
  const float eps = 1e-30f;
  if (a <= eps && e <= eps) {
    s = t = 0.f;
  } else if (a <= eps) {
    s = 0.f;
    t = fclamp01(f / e);
  } else {
    const float c = fdot3(d1, r);
    if (e <= eps) {
      t = 0.f;
      s = fclamp01(-c / a);
    } else {
      const float b = fdot3(d1, d2);
      const float den = a * e - b * b;
      s = den > 0.f ? fclamp01((b * f - c * e) / den) : 0.f;
      t = (b * s + f) / e;
      if (t < 0.f) {
        t = 0.f;
        s = fclamp01(-c / a);
      } else if (t > 1.f) {
        t = 1.f;
        s = fclamp01((b - c) / a);
      }
    }
  }
  c1 = fadd3(p0, fscale3(d1, s));
  c2 = fadd3(q0, fscale3(d2, t));
}

// Lower bound of the distance of a stencil whose vertices are x_i = c + P_i,
// given FP32 copies Pf_i of (x_i - c); X = max |x - c| over the scene.
// Returns 0 when no useful bound exists.
__device__ __forceinline__ float lower_bound(bool ee, f3 W0, f3 W1, f3 W2, f3 W3, float X) {
  const f3 P0 = f3{0.f, 0.f, 0.f}, P1 = fsub3(W1, W0), P2 = fsub3(W2, W0), P3 = fsub3(W3, W0);
  const float R = fmaxf(fmaxabs3(P1), fmaxf(fmaxabs3(P2), fmaxabs3(P3)));
  f3 a;
  float smin, smax;
  if (!ee) {
    const f3 c = closest_on_triangle(P1, P2, P3);
    a = fscale3(c, -1.f);  // from the triangle towards the point (at the origin)
    smin = 0.f;
    smax = fmaxf(fdot3(a, P1), fmaxf(fdot3(a, P2), fdot3(a, P3)));
  } else {
    f3 c1, c2;
    closest_on_segments(P0, P1, P2, P3, c1, c2);
    a = fsub3(c1, c2);
    smin = fminf(0.f, fdot3(a, P1));
    smax = fmaxf(fdot3(a, P2), fdot3(a, P3));
  }
  const float an = sqrtf(fdot3(a, a));
  if (!(an > 0.f)) return 0.f;
  const float u = 5.9604645e-8f;  // 2^-24
  const float a1 = fabsf(a.x) + fabsf(a.y) + fabsf(a.z);
  const float s = (smin - smax) - 4.f * (6.f * u * a1 * R);
  if (!(s > 0.f)) return 0.f;
  const float lb = s / (an * (1.f + 16.f * u)) - 4.f * (3.5f * u * (X + R));
  return lb > 0.f ? lb : 0.f;
}

}  // namespace cbb
