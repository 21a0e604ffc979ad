// geodesic.cu -- reference distances of a shell as geodesic distances on its
// rest mesh (CB_DBAR_GEODESIC): the rest-filter precompute for rest shapes
// that are not cut from a flat pattern (doubly curved).
//
// Sec. 3.2 takes a shell stencil pair's reference distance in the shell's 2D
// rest domain; the paper names non-flat rest shapes as future work.  Here the
// rest domain is the rest mesh itself:
//   dbar(P, Q) = min over p in P, q in Q of g(p, q),
// g the shortest-path length on the polyhedral rest surface.  Shortest paths
// are straight across every face and edge they cross and bend only at
// vertices, so dbar reduces to vertex-to-edge distances g(w, e):
//   point-triangle (p; t): min over the three edges e of t of g(p, e) (a path
//     from p meets t on its boundary first);
//   edge-edge (A, B): min over vertices w of g(w, A) + g(w, B) (between
//     interior points without a bend the minimizing path is perpendicular to
//     both edges and slides along them, at constant length, to an end point
//     or a vertex; w an end point of A has g(w, A) = 0).
//
// g(v, .) below the activation a, for every vertex v: a Dijkstra over the
// vertices a path may bend at (all of them: a bend at a vertex of angle sum
// at most 2 pi never shortens a path, it only costs work), each settled vertex
// u expanded by unfolding, face by face, the strips a straight segment from u
// can cross within a - g(v, u).  A strip carries its wedge -- the directions
// from u, laid at the origin, that cross every edge of the strip -- as the two
// end points of the reached part of the edge last crossed.  The face beyond
// that edge is unfolded across it, away from the face before; its third
// vertex W is reached if it lies in the wedge, and splits the wedge in two if
// it lies strictly inside.  An edge whose reached part has positive length
// records u's distance plus the distance from the origin to that part; a
// strip reaching an edge in a single point runs through a vertex and is the
// path that bends there.
//
// Layout: persistent threads, each taking source vertices in turn.  A
// thread's Dijkstra table (vertex -> distance), edge table (edge -> distance),
// their lists of used slots and its strip stack live in global scratch sized
// for the launch, thread-interleaved ([slot][thread]) so that a warp's
// accesses to the same slot coalesce.  Every capacity is fixed; a source that
// would overflow one sets an error bit (the scene create then returns
// CB_ERR_TOO_LARGE) instead of writing past it, and every loop is bounded.
// Each source appends its (edge, vertex, g) entries with g < a to one global
// list (one atomicAdd per source; a second run with the exact capacity when
// the first guess was short).  The list is sorted by (edge, vertex) and each
// rest-broad-phase candidate combines its rows (binary search for a
// point-triangle pair, a merge of two rows for an edge-edge pair).
#include <algorithm>
#include <cstdint>
#include <vector>

#include "geometry.cuh"
#include "pairs.cuh"
#include "prims.cuh"
#include "scene.cuh"

using namespace cbg;

namespace {

constexpr int GEO_HV = 256;        // Dijkstra table slots (power of two)
constexpr int GEO_VL = 192;        // vertices a source may reach below a
constexpr int GEO_HE = 512;        // edge table slots (power of two)
constexpr int GEO_EL = 384;        // edges a source may reach below a
constexpr int GEO_STACK = 64;      // strip stack frames
constexpr int GEO_STEPS = 1 << 18; // strip steps per source
constexpr int GEO_T = 64;          // threads per block
constexpr uint64_t GEO_ERR_TABLE = 1, GEO_ERR_STACK = 2, GEO_ERR_STEPS = 4;

struct P2 {
  double x, y;
};
__device__ __forceinline__ double gcross(P2 a, P2 b) { return xsub(xmul(a.x, b.y), xmul(a.y, b.x)); }
__device__ __forceinline__ double gdot(P2 a, P2 b) { return xadd(xmul(a.x, b.x), xmul(a.y, b.y)); }
__device__ __forceinline__ P2 gsub(P2 a, P2 b) { return P2{xsub(a.x, b.x), xsub(a.y, b.y)}; }
__device__ __forceinline__ P2 gat(P2 a, P2 d, double s) { return P2{xadd(a.x, xmul(s, d.x)), xadd(a.y, xmul(s, d.y))}; }

// the part [lo, hi] of s where c0 + c1 s >= 0
__device__ __forceinline__ void gclip(double c0, double c1, double& lo, double& hi) {
  if (c1 > 0.0) {
    lo = fmax(lo, xdiv(-c0, c1));
  } else if (c1 < 0.0) {
    hi = fmin(hi, xdiv(-c0, c1));
  } else if (c0 < 0.0) {
    lo = 1.0;
    hi = 0.0;
  }
}

// Thread-interleaved scratch of the persistent threads.
struct GeoScratch {
  int nt;                // threads of the launch
  int32_t* vkey;         // [HV][nt] vertex id, -1 free
  double* vdist;         // [HV][nt]
  uint8_t* vdone;        // [HV][nt]
  uint16_t* vlist;       // [VL][nt] used Dijkstra slots
  int32_t* ekey;         // [HE][nt] edge id, -1 free
  double* edist;         // [HE][nt]
  uint16_t* elist;       // [EL][nt] used edge slots
  double* fd;            // [STACK][10][nt] frame points A, B, C, L, R
  int32_t* fi;           // [STACK][3][nt] frame ids ia, ib, face
};

struct GeoMesh {
  const int32_t* tv;     // [3][T]
  int T;
  const int32_t* te;     // [T][3]: edge of (t_k, t_k+1)
  const int32_t* ef;     // [E][2]: faces of an edge, -1 none
  const int32_t* vfp;    // [n+1] faces around a vertex
  const int32_t* vf;
  const double* elen;    // [E] rest length
};

__device__ __forceinline__ uint32_t ghash(uint32_t k, int bits) { return (k * 0x9E3779B1u) >> (32 - bits); }

// One source's state, with its tables in the thread's scratch.
struct GeoSource {
  GeoScratch S;
  int tid;
  double a;
  int nv = 0, ne = 0;
  uint64_t err = 0;
  __device__ GeoSource(const GeoScratch& s, int t, double a_) : S(s), tid(t), a(a_) {}
  __device__ __forceinline__ size_t at(int slot) const { return (size_t)slot * S.nt + tid; }

  __device__ void relax(int w, double d) {
    if (!(d < a)) return;
    uint32_t h = ghash((uint32_t)w, 8);
    for (int probe = 0; probe < GEO_HV; ++probe, h = (h + 1) & (GEO_HV - 1)) {
      const int32_t k = S.vkey[at(h)];
      if (k == w) {
        if (d < S.vdist[at(h)]) S.vdist[at(h)] = d;
        return;
      }
      if (k < 0) {
        if (nv >= GEO_VL) {
          err |= GEO_ERR_TABLE;
          return;
        }
        S.vkey[at(h)] = w;
        S.vdist[at(h)] = d;
        S.vdone[at(h)] = 0;
        S.vlist[at(nv++)] = (uint16_t)h;
        return;
      }
    }
    err |= GEO_ERR_TABLE;
  }

  __device__ void record(int e, double d) {
    if (!(d < a)) return;
    uint32_t h = ghash((uint32_t)e, 9);
    for (int probe = 0; probe < GEO_HE; ++probe, h = (h + 1) & (GEO_HE - 1)) {
      const int32_t k = S.ekey[at(h)];
      if (k == e) {
        if (d < S.edist[at(h)]) S.edist[at(h)] = d;
        return;
      }
      if (k < 0) {
        if (ne >= GEO_EL) {
          err |= GEO_ERR_TABLE;
          return;
        }
        S.ekey[at(h)] = e;
        S.edist[at(h)] = d;
        S.elist[at(ne++)] = (uint16_t)h;
        return;
      }
    }
    err |= GEO_ERR_TABLE;
  }

  // frees the used slots for the next source
  __device__ void clear() {
    for (int i = 0; i < nv; ++i) S.vkey[at(S.vlist[at(i)])] = -1;
    for (int i = 0; i < ne; ++i) S.ekey[at(S.elist[at(i)])] = -1;
    nv = ne = 0;
  }
};

// edge of face f between vertices p and q
__device__ __forceinline__ int face_edge(const GeoMesh& M, int f, int p, int q) {
  int e = -1;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int x = M.tv[(size_t)k * M.T + f], y = M.tv[(size_t)((k + 1) % 3) * M.T + f];
    if ((x == p && y == q) || (x == q && y == p)) e = M.te[3 * (size_t)f + k];
  }
  return e;
}

// A strip on the stack: the edge last crossed (A on the wedge's left, B on its
// right: cross(A, B) > 0), the third vertex C of the face before it, the wedge
// boundary points L, R (directions from the origin), the edge's vertex ids and
// the face before it.
struct Frame {
  P2 A, B, C, L, R;
  int ia, ib, f;
};

struct GeoStack {
  GeoScratch S;
  int tid, sp = 0;
  __device__ GeoStack(const GeoScratch& s, int t) : S(s), tid(t) {}
  __device__ __forceinline__ size_t dd(int k) const { return ((size_t)sp * 10 + k) * S.nt + tid; }
  __device__ __forceinline__ size_t di(int k) const { return ((size_t)sp * 3 + k) * S.nt + tid; }
  __device__ bool push(const Frame& F) {
    if (sp >= GEO_STACK) return false;
    const double v[10] = {F.A.x, F.A.y, F.B.x, F.B.y, F.C.x, F.C.y, F.L.x, F.L.y, F.R.x, F.R.y};
#pragma unroll
    for (int k = 0; k < 10; ++k) S.fd[dd(k)] = v[k];
    S.fi[di(0)] = F.ia;
    S.fi[di(1)] = F.ib;
    S.fi[di(2)] = F.f;
    ++sp;
    return true;
  }
  __device__ Frame pop() {
    --sp;
    double v[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) v[k] = S.fd[dd(k)];
    Frame F;
    F.A = P2{v[0], v[1]};
    F.B = P2{v[2], v[3]};
    F.C = P2{v[4], v[5]};
    F.L = P2{v[6], v[7]};
    F.R = P2{v[8], v[9]};
    F.ia = S.fi[di(0)];
    F.ib = S.fi[di(1)];
    F.f = S.fi[di(2)];
    return F;
  }
};

// the vertex at distances la from A and lb from B (|AB| = lab), on the side
// of line AB away from C
__device__ __forceinline__ P2 unfold_across(P2 A, P2 B, P2 C, double la, double lb, double lab) {
  const P2 AB = gsub(B, A);
  const double nab = __dsqrt_rn(gdot(AB, AB));
  const P2 u{xdiv(AB.x, nab), xdiv(AB.y, nab)};
  const double x = xdiv(xadd(xsub(xmul(la, la), xmul(lb, lb)), xmul(lab, lab)), xmul(2.0, lab));
  const double y2 = xsub(xmul(la, la), xmul(x, x));
  double y = y2 > 0.0 ? __dsqrt_rn(y2) : 0.0;
  if (gcross(AB, gsub(C, A)) > 0.0) y = -y;
  return P2{xadd(xadd(A.x, xmul(x, u.x)), xmul(y, -u.y)), xadd(xadd(A.y, xmul(x, u.y)), xmul(y, u.x))};
}

// One strip step: the reached part of the frame's edge, its record, and the
// strips beyond it.  Returns false if the stack overflowed.
__device__ bool strip_step(const GeoMesh& M, GeoSource& G, GeoStack& K, const Frame& F, double du, double rem) {
  if (!(gcross(F.A, F.B) > 0.0)) return true;
  const P2 D = gsub(F.B, F.A);
  double lo = 0.0, hi = 1.0;
  gclip(gcross(F.L, F.A), gcross(F.L, D), lo, hi);   // cross(L, X) >= 0
  gclip(gcross(F.A, F.R), gcross(D, F.R), lo, hi);   // cross(X, R) >= 0
  if (!(lo < hi)) return true;
  const P2 XL = gat(F.A, D, lo), XR = gat(F.A, D, hi);
  const double dd = gdot(D, D);
  double sf = dd > 0.0 ? xdiv(-gdot(F.A, D), dd) : lo;
  sf = fmin(fmax(sf, lo), hi);
  const P2 X = gat(F.A, D, sf);
  const double dmin = __dsqrt_rn(gdot(X, X));
  const int e = face_edge(M, F.f, F.ia, F.ib);
  G.record(e, xadd(du, dmin));
  if (!(dmin < rem)) return true;
  const int f2 = M.ef[2 * (size_t)e] == F.f ? M.ef[2 * (size_t)e + 1] : M.ef[2 * (size_t)e];
  if (f2 < 0) return true;
  int w = -1;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int c = M.tv[(size_t)k * M.T + f2];
    if (c != F.ia && c != F.ib) w = c;
  }
  const P2 W = unfold_across(F.A, F.B, F.C, M.elen[face_edge(M, f2, F.ia, w)], M.elen[face_edge(M, f2, F.ib, w)],
                             M.elen[e]);
  const double cl = gcross(XL, W), cr = gcross(W, XR);
  if (cl >= 0.0 && cr >= 0.0) G.relax(w, xadd(du, __dsqrt_rn(gdot(W, W))));
  if (cl > 0.0 && cr > 0.0) {
    return K.push(Frame{F.A, W, F.B, XL, W, F.ia, w, f2}) && K.push(Frame{W, F.B, F.A, W, XR, w, F.ib, f2});
  }
  if (cl <= 0.0) return K.push(Frame{W, F.B, F.A, XL, XR, w, F.ib, f2});
  return K.push(Frame{F.A, W, F.B, XL, XR, F.ia, w, f2});
}

// Persistent threads over the source vertices; each source's (edge, vertex,
// g) entries appended to (key, g) at one atomicAdd of count.
__global__ void __launch_bounds__(GEO_T) k_geo_ball(int n, double a, GeoMesh M, GeoScratch S,
                                                     uint64_t* __restrict__ out_key, double* __restrict__ out_g,
                                                     unsigned long long cap, unsigned long long* __restrict__ count,
                                                     unsigned long long* __restrict__ errbits) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= S.nt) return;
  GeoSource G(S, tid, a);
  GeoStack K(S, tid);
  for (int v = tid; v < n; v += S.nt) {
    G.err = 0;
    G.relax(v, 0.0);
    int steps = 0;
    for (int settle = 0; settle < GEO_VL && !G.err; ++settle) {
      int best = -1;
      double bd = 0.0;
      for (int i = 0; i < G.nv; ++i) {
        const int h = S.vlist[G.at(i)];
        const double d = S.vdist[G.at(h)];
        if (!S.vdone[G.at(h)] && (best < 0 || d < bd)) {
          best = h;
          bd = d;
        }
      }
      if (best < 0) break;
      S.vdone[G.at(best)] = 1;
      const int u = S.vkey[G.at(best)];
      const double du = bd, rem = xsub(a, bd);
      for (int q = M.vfp[u]; q < M.vfp[u + 1] && !G.err; ++q) {
        const int f = M.vf[q];
        int k = 0;
        while (k < 2 && M.tv[(size_t)k * M.T + f] != u) ++k;
        const int p = M.tv[(size_t)((k + 1) % 3) * M.T + f], r = M.tv[(size_t)((k + 2) % 3) * M.T + f];
        const int eup = face_edge(M, f, u, p), eur = face_edge(M, f, u, r);
        const double lup = M.elen[eup], lur = M.elen[eur], lpr = M.elen[face_edge(M, f, p, r)];
        G.relax(p, xadd(du, lup));
        G.relax(r, xadd(du, lur));
        G.record(eup, du);
        G.record(eur, du);
        const double x = xdiv(xsub(xadd(xmul(lup, lup), xmul(lur, lur)), xmul(lpr, lpr)), xmul(2.0, lup));
        const double y2 = xsub(xmul(lur, lur), xmul(x, x));
        const P2 P{lup, 0.0}, Q{x, y2 > 0.0 ? __dsqrt_rn(y2) : 0.0}, O{0.0, 0.0};
        K.sp = 0;
        K.push(Frame{P, Q, O, P, Q, p, r, f});
        while (K.sp > 0) {
          if (++steps > GEO_STEPS) {
            G.err |= GEO_ERR_STEPS;
            break;
          }
          const Frame F = K.pop();
          if (!strip_step(M, G, K, F, du, rem)) {
            G.err |= GEO_ERR_STACK;
            break;
          }
        }
      }
    }
    if (G.err) {
      atomicOr(errbits, (unsigned long long)G.err);
    } else if (G.ne > 0) {
      const unsigned long long base = atomicAdd(count, (unsigned long long)G.ne);
      for (int i = 0; i < G.ne; ++i) {
        if (base + i >= cap) break;
        const int h = S.elist[G.at(i)];
        out_key[base + i] = ((uint64_t)(uint32_t)S.ekey[G.at(h)] << 32) | (uint32_t)v;
        out_g[base + i] = S.edist[G.at(h)];
      }
    }
    G.clear();
  }
}

// rest length of every edge, summed in a fixed order without contraction
__global__ void k_geo_elen(int E, const int32_t* __restrict__ ev0, const int32_t* __restrict__ ev1,
                           const double* __restrict__ rest, int n, double* __restrict__ elen) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const d3 d = sub3(load3(rest, n, ev1[e]), load3(rest, n, ev0[e]));
  elen[e] = __dsqrt_rn(dot3(d, d));
}

__global__ void k_geo_iota(int64_t m, uint32_t* __restrict__ idx) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) idx[i] = (uint32_t)i;
}

__global__ void k_geo_gather(int64_t m, const uint32_t* __restrict__ idx, const double* __restrict__ g,
                             double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) out[i] = g[idx[i]];
}

// row[e] = first entry whose key has edge e in its high word, e = 0..E
__global__ void k_geo_rows(int E, const uint64_t* __restrict__ key, int64_t nk, int64_t* __restrict__ row) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e > E) return;
  const uint64_t bound = (uint64_t)e << 32;
  int64_t lo = 0, hi = nk;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (key[mid] < bound) lo = mid + 1;
    else hi = mid;
  }
  row[e] = lo;
}

// g(w, e) from edge e's row (sorted by vertex), +inf if not below a
__device__ __forceinline__ double geo_lookup(const uint64_t* __restrict__ key, const double* __restrict__ g,
                                             const int64_t* __restrict__ row, int e, int w) {
  int64_t lo = row[e], hi = row[e + 1];
  const int64_t end = hi;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((uint32_t)key[mid] < (uint32_t)w) lo = mid + 1;
    else hi = mid;
  }
  return (lo < end && (uint32_t)key[lo] == (uint32_t)w) ? g[lo] : __longlong_as_double(0x7ff0000000000000LL);
}

// Reference distance of each rest-broad-phase candidate; the same outputs as
// the planar rest filter: flag (dbar < a, same component), dbar, and the
// scene's and each component's smallest dbar of the flagged pairs.
__global__ void k_geo_dbar(int64_t nc, const uint64_t* __restrict__ cand, const int32_t* __restrict__ ev0,
                           const int32_t* __restrict__ ev1, const int32_t* __restrict__ tv, int T,
                           const int32_t* __restrict__ te, const int32_t* __restrict__ comp,
                           const uint64_t* __restrict__ key, const double* __restrict__ g,
                           const int64_t* __restrict__ row, double a, uint32_t* __restrict__ flag,
                           double* __restrict__ dbar, unsigned long long* __restrict__ dmin_bits,
                           unsigned long long* __restrict__ dmin_comp) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long mb = 0x7ff0000000000000ull;
  if (c < nc) {
    const uint64_t k = cand[c];
    const Stencil s = stencil_of(k, ev0, ev1, tv, T);
    double d = __longlong_as_double(0x7ff0000000000000LL);
    uint32_t f = 0;
    if (comp[s.v[0]] == comp[s.v[2]]) {
      const int i = (int)((k >> 31) & 0x7FFFFFFFu), j = (int)(k & 0x7FFFFFFFu);
      if (!s.ee) {
#pragma unroll
        for (int q = 0; q < 3; ++q) d = fmin(d, geo_lookup(key, g, row, te[3 * (size_t)j + q], i));
      } else {
        int64_t p = row[i], q = row[j];
        const int64_t pe = row[i + 1], qe = row[j + 1];
        while (p < pe && q < qe) {
          const uint32_t wp = (uint32_t)key[p], wq = (uint32_t)key[q];
          if (wp < wq) {
            ++p;
          } else if (wq < wp) {
            ++q;
          } else {
            d = fmin(d, xadd(g[p], g[q]));
            ++p;
            ++q;
          }
        }
      }
      if (d < a) {
        f = 1;
        mb = (unsigned long long)__double_as_longlong(d);
        atomicMin(&dmin_comp[comp[s.v[0]]], mb);
      }
    }
    flag[c] = f;
    dbar[c] = d;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long u = __shfl_xor_sync(0xffffffffu, mb, o);
    mb = u < mb ? u : mb;
  }
  if ((threadIdx.x & 31) == 0 && mb != 0x7ff0000000000000ull) atomicMin(dmin_bits, mb);
}

}  // namespace

static size_t geo_align(size_t b) { return (b + 255) & ~(size_t)255; }

template <typename T>
static cb_status geo_upload(DevBuf& b, const std::vector<T>& h, cudaStream_t st) {
  CB_TRY(buf_ensure(b, sizeof(T) * std::max<size_t>(h.size(), 1), st));
  if (!h.empty()) CB_CUDA(cudaMemcpyAsync(b.p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, st));
  return CB_OK;
}

static uint64_t geo_mask(uint64_t v) {
  uint64_t m = 0;
  while (m < v) m = (m << 1) | 1;
  return m;
}

cb_status geo_rest_dbar(cb_scene* s, const uint64_t* cand, int64_t nc, uint32_t* flag, double* dbar,
                        unsigned long long* dmin, unsigned long long* dcomp, cudaStream_t st) {
  const int n = s->n, E = s->E, T = s->T;
  if (nc <= 0) return CB_OK;
  ScopedBuf te_(st), ef_(st), vfp_(st), vf_(st), elen_(st), scr_(st), row_(st), hist_(st), stmp_(st);
  ScopedBuf k0_(st), k1_(st), g0_(st), g1_(st), i0_(st), i1_(st);
  // mesh adjacency (built on the host at scene creation) and rest edge lengths
  CB_TRY(geo_upload(te_.b, s->geo_te, st));
  CB_TRY(geo_upload(ef_.b, s->geo_ef, st));
  CB_TRY(geo_upload(vfp_.b, s->geo_vfp, st));
  CB_TRY(geo_upload(vf_.b, s->geo_vf, st));
  CB_TRY(buf_ensure(elen_.b, sizeof(double) * (size_t)std::max(1, E), st));
  k_geo_elen<<<cb_grid(std::max(1, E)), CB_THREADS, 0, cb_count(st)>>>(E, bp<int32_t>(s->ev0), bp<int32_t>(s->ev1),
                                                                     bp<double>(s->rest), n, bp<double>(elen_.b));
  GeoMesh M{bp<int32_t>(s->tv), T, bp<int32_t>(te_.b), bp<int32_t>(ef_.b), bp<int32_t>(vfp_.b),
            bp<int32_t>(vf_.b), bp<double>(elen_.b)};
  // scratch of the persistent threads
  const int nt = std::min(((n + 31) / 32) * 32, s->n_sms * 2 * GEO_T);
  const size_t szs[9] = {sizeof(int32_t) * GEO_HV,  sizeof(double) * GEO_HV,        1 * GEO_HV,
                         sizeof(uint16_t) * GEO_VL, sizeof(int32_t) * GEO_HE,        sizeof(double) * GEO_HE,
                         sizeof(uint16_t) * GEO_EL, sizeof(double) * 10 * GEO_STACK, sizeof(int32_t) * 3 * GEO_STACK};
  size_t off[10] = {0};
  for (int k = 0; k < 9; ++k) off[k + 1] = off[k] + geo_align(szs[k] * (size_t)nt);
  CB_TRY(buf_ensure(scr_.b, off[9], st));
  char* base = (char*)scr_.b.p;
  GeoScratch S{nt,
               (int32_t*)(base + off[0]),
               (double*)(base + off[1]),
               (uint8_t*)(base + off[2]),
               (uint16_t*)(base + off[3]),
               (int32_t*)(base + off[4]),
               (double*)(base + off[5]),
               (uint16_t*)(base + off[6]),
               (double*)(base + off[7]),
               (int32_t*)(base + off[8])};
  CB_CUDA(cudaMemsetAsync(S.vkey, 0xff, szs[0] * (size_t)nt, st));
  CB_CUDA(cudaMemsetAsync(S.ekey, 0xff, szs[4] * (size_t)nt, st));
  // the (edge, vertex, g) entries: a first guess of the count, then the exact one
  uint64_t* sc = scalars(s);
  unsigned long long* cnt = (unsigned long long*)(sc + SC_GEO_COUNT);
  unsigned long long* err = (unsigned long long*)(sc + SC_GEO_ERR);
  static_assert(SC_GEO_ERR == SC_GEO_COUNT + 1, "count and error bits are adjacent");
  uint64_t cap = std::max<uint64_t>(1024, 48 * (uint64_t)n), total = 0;
  for (int run = 0; run < 2; ++run) {
    CB_TRY(buf_ensure(k0_.b, sizeof(uint64_t) * cap, st));
    CB_TRY(buf_ensure(g0_.b, sizeof(double) * cap, st));
    CB_CUDA(cudaMemsetAsync(cnt, 0, 2 * sizeof(uint64_t), st));  // count and error bits
    k_geo_ball<<<(nt + GEO_T - 1) / GEO_T, GEO_T, 0, cb_count(st)>>>(n, s->a, M, S, bp<uint64_t>(k0_.b),
                                                                    bp<double>(g0_.b), cap, cnt, err);
    CB_CUDA(cudaGetLastError());
    uint64_t h[2];
    CB_TRY(read_scalars(s, SC_GEO_COUNT, 2, h, st));
    if (h[1]) return CB_ERR_TOO_LARGE;  // a source's ball, edge list or strip exceeds the fixed capacities
    total = h[0];
    if (total <= cap) break;
    cap = total;
  }
  // sorted by (edge, vertex); rows by edge
  const int64_t m = (int64_t)total;
  if (m >= (int64_t)UINT32_MAX) return CB_ERR_TOO_LARGE;
  const size_t m1 = (size_t)std::max<int64_t>(1, m);
  CB_TRY(buf_ensure(k1_.b, sizeof(uint64_t) * m1, st));
  CB_TRY(buf_ensure(g1_.b, sizeof(double) * m1, st));
  CB_TRY(buf_ensure(i0_.b, sizeof(uint32_t) * m1, st));
  CB_TRY(buf_ensure(i1_.b, sizeof(uint32_t) * m1, st));
  const int64_t he = cbp::radix_hist_elems((int64_t)m1);
  CB_TRY(buf_ensure(hist_.b, sizeof(uint32_t) * (size_t)he, st));
  CB_TRY(buf_ensure(stmp_.b, sizeof(uint32_t) * (size_t)(cbp::scan_tmp_elems(he) + 8), st));
  const uint64_t need = (geo_mask((uint64_t)std::max(1, E) - 1) << 32) | geo_mask((uint64_t)n - 1);
  k_geo_iota<<<cb_grid((int64_t)m1), CB_THREADS, 0, cb_count(st)>>>(m, bp<uint32_t>(i0_.b));
  const int r = cbp::radix_sort<uint64_t, uint32_t, true>(bp<uint64_t>(k0_.b), bp<uint32_t>(i0_.b),
                                                          bp<uint64_t>(k1_.b), bp<uint32_t>(i1_.b), m, 0, 64,
                                                          bp<uint32_t>(hist_.b), bp<uint32_t>(stmp_.b), st, need);
  const uint64_t* key = r ? bp<uint64_t>(k1_.b) : bp<uint64_t>(k0_.b);
  k_geo_gather<<<cb_grid((int64_t)m1), CB_THREADS, 0, cb_count(st)>>>(m, r ? bp<uint32_t>(i1_.b) : bp<uint32_t>(i0_.b),
                                                                    bp<double>(g0_.b), bp<double>(g1_.b));
  const double* g = bp<double>(g1_.b);
  CB_TRY(buf_ensure(row_.b, sizeof(int64_t) * ((size_t)E + 1), st));
  k_geo_rows<<<cb_grid((int64_t)E + 1), CB_THREADS, 0, cb_count(st)>>>(E, key, m, bp<int64_t>(row_.b));
  k_geo_dbar<<<cb_grid(nc), CB_THREADS, 0, cb_count(st)>>>(nc, cand, bp<int32_t>(s->ev0), bp<int32_t>(s->ev1),
                                                           bp<int32_t>(s->tv), T, bp<int32_t>(te_.b),
                                                           bp<int32_t>(s->comp), key, g, bp<int64_t>(row_.b), s->a,
                                                           flag, dbar, dmin, dcomp);
  CB_CUDA(cudaGetLastError());
  // the buffers above are released at scope exit after the stream's work
  return CB_OK;
}
