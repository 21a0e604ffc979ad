// broad.cu -- stage (a): spatial-hash broad phase at the full activation (Sec. 3.3).
//
// Canonical result: every non-incident primitive pair whose FP64 boxes, each
// inflated by h, overlap on all three axes (closed intervals).  The hash works
// on FP32 boxes rounded outward from the FP64 ones (lo rounded down, hi up), so
// FP32 overlap is implied by FP64 overlap: the FP32 candidate stream is a
// superset.  A pair is then accepted outright when the FP32 test still passes
// after moving every FP32 bound one ulp inward (the FP64 bound lies within that
// ulp), rejected when the plain FP32 test fails, and decided on the stored FP64
// boxes otherwise.
//
// Steps: boxes + scene bounds -> cell size -> (cell, primitive) entries for
// every cell a box covers -> stable radix sort by Morton cell key -> runs of
// equal cells -> per entry, test the later entries of its run (point vs
// triangle, edge vs later edge); a pair is reported only in the cell holding
// the low corner of the two boxes' intersection (its "home" cell) -> compact
// keys -> radix sort -> canonical keys.
//
// Several scenes can share one pass (a batch): every member has its own
// box inflation and grid, and its member index sits above the 30 Morton bits
// of the cell key, so primitives of different members never meet in a cell.
#include <algorithm>
#include <cmath>

#include "prims.cuh"
#include "scene.cuh"

namespace {

struct Topo {
  int kind, n, T, E;
  const int32_t* __restrict__ ev0;
  const int32_t* __restrict__ ev1;
  const int32_t* __restrict__ tv;
};

__device__ __forceinline__ int prim_verts(const Topo& t, int q, int v[3]) {
  if (t.kind == CB_ROD) {
    v[0] = t.ev0[q];
    v[1] = t.ev1[q];
    v[2] = -1;
    return 2;
  }
  if (q < t.n) {
    v[0] = q;
    v[1] = v[2] = -1;
    return 1;
  }
  q -= t.n;
  if (q < t.T) {
    v[0] = t.tv[q];
    v[1] = t.tv[t.T + q];
    v[2] = t.tv[2 * t.T + q];
    return 3;
  }
  q -= t.T;
  v[0] = t.ev0[q];
  v[1] = t.ev1[q];
  v[2] = -1;
  return 2;
}

__device__ __forceinline__ uint32_t f2o(float f) {
  uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__host__ __device__ __forceinline__ float o2f(uint32_t o) {
  uint32_t b = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float f;
  memcpy(&f, &b, 4);
  return f;
#endif
}

// per member: [0..2] min (ordered), [3..5] max (ordered), [6..7] pad, then a double extent sum
constexpr int BOUNDS_STRIDE = 10;  // uint32 words per member (40 bytes)

__global__ void k_bounds_init(uint32_t* b, int count) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= count) return;
  uint32_t* q = b + (size_t)m * BOUNDS_STRIDE;
  for (int k = 0; k < 3; ++k) {
    q[k] = 0xffffffffu;
    q[3 + k] = 0u;
  }
  q[6] = q[7] = 0u;
  *(double*)(q + 8) = 0.0;
}

__device__ __forceinline__ int prim_member(const Topo& t, const int32_t* __restrict__ vsc, int q) {
  int v[3];
  prim_verts(t, q, v);
  return vsc[v[0]];
}

// swept: boxes of x and x + p inflated by xi / 2 (the CCD phase); else boxes
// of x inflated by a / 2 (full activation)
__global__ void k_boxes(Topo t, int np, const double* __restrict__ x, const double* __restrict__ p,
                        const MemberParams* __restrict__ mp, bool swept, const int32_t* __restrict__ vsc,
                        float4* __restrict__ box32, double* __restrict__ box64, double* __restrict__ box_raw,
                        uint32_t* bounds) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  float lo32[3] = {INFINITY, INFINITY, INFINITY}, hi32[3] = {-INFINITY, -INFINITY, -INFINITY};
  float ext = 0.f;
  int mem = -1;
  if (q < np) {
    int v[3];
    const int nv = prim_verts(t, q, v);
    mem = vsc[v[0]];
    const double h = swept ? 0.5 * mp[mem].xi : 0.5 * mp[mem].a;
    double lo[3], hi[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double mn = INFINITY, mx = -INFINITY;
      for (int a = 0; a < nv; ++a) {
        double c = x[(size_t)k * t.n + v[a]];
        mn = fmin(mn, c);
        mx = fmax(mx, c);
        if (p) {
          double c2 = xadd(c, p[(size_t)k * t.n + v[a]]);
          mn = fmin(mn, c2);
          mx = fmax(mx, c2);
        }
      }
      if (box_raw) {  // the primitive's own box (per-stencil activation inflates it by each pair's width)
        box_raw[(size_t)q * 6 + k] = mn;
        box_raw[(size_t)q * 6 + 3 + k] = mx;
      }
      lo[k] = xsub(mn, h);
      hi[k] = xadd(mx, h);
      lo32[k] = __double2float_rd(lo[k]);
      hi32[k] = __double2float_ru(hi[k]);
      box64[(size_t)q * 6 + k] = lo[k];
      box64[(size_t)q * 6 + 3 + k] = hi[k];
      ext = fmaxf(ext, hi32[k] - lo32[k]);
    }
    box32[2 * (size_t)q] = make_float4(lo32[0], lo32[1], lo32[2], 0.f);
    box32[2 * (size_t)q + 1] = make_float4(hi32[0], hi32[1], hi32[2], 0.f);
  }
  // per-member bounds and extent sums: a block reduction when the block holds
  // one member (the usual case: members occupy contiguous primitive ranges),
  // per-thread atomics at the few blocks that straddle members
  __shared__ int s_mmin, s_mmax;
  if (threadIdx.x == 0) {
    s_mmin = 0x7fffffff;
    s_mmax = -1;
  }
  __syncthreads();
  if (mem >= 0) {
    atomicMin(&s_mmin, mem);
    atomicMax(&s_mmax, mem);
  }
  __syncthreads();
  if (s_mmax < 0) return;
  if (s_mmin != s_mmax) {
    if (mem >= 0) {
      uint32_t* bq = bounds + (size_t)mem * BOUNDS_STRIDE;
      for (int k = 0; k < 3; ++k) {
        atomicMin(&bq[k], f2o(lo32[k]));
        atomicMax(&bq[3 + k], f2o(hi32[k]));
      }
      atomicAdd((double*)(bq + 8), (double)ext);
    }
    return;
  }
  __shared__ float s_lo[3][CB_THREADS / 32], s_hi[3][CB_THREADS / 32];
  __shared__ double s_ext[CB_THREADS / 32];
  double e = ext;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      lo32[k] = fminf(lo32[k], __shfl_xor_sync(0xffffffffu, lo32[k], o));
      hi32[k] = fmaxf(hi32[k], __shfl_xor_sync(0xffffffffu, hi32[k], o));
    }
    e += __shfl_xor_sync(0xffffffffu, e, o);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    for (int k = 0; k < 3; ++k) {
      s_lo[k][w] = lo32[k];
      s_hi[k][w] = hi32[k];
    }
    s_ext[w] = e;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float l[3] = {INFINITY, INFINITY, INFINITY}, hh[3] = {-INFINITY, -INFINITY, -INFINITY};
    double es = 0;
    for (int q2 = 0; q2 < CB_THREADS / 32; ++q2) {
      for (int k = 0; k < 3; ++k) {
        l[k] = fminf(l[k], s_lo[k][q2]);
        hh[k] = fmaxf(hh[k], s_hi[k][q2]);
      }
      es += s_ext[q2];
    }
    uint32_t* bq = bounds + (size_t)s_mmin * BOUNDS_STRIDE;
    for (int k = 0; k < 3; ++k) {
      atomicMin(&bq[k], f2o(l[k]));
      atomicMax(&bq[3 + k], f2o(hh[k]));
    }
    atomicAdd((double*)(bq + 8), es);
  }
}

// One thread per member: its hash grid from the bounds and extent sum of its
// inflated primitive boxes.  The cell edge is the mean box extent (times the
// tuned factor) rounded down to a quarter octave, so that summation-order
// differences in the extent sum never move it, and at least 1/1000 of the
// member's span along every axis.  cx gets the member's box centre and half
// its largest extent (the origin of the FP32 positions).
__global__ void k_grids(int M, const uint32_t* __restrict__ bounds, const MemberParams* __restrict__ mp,
                        double cell_factor, Grid* __restrict__ grids, double* __restrict__ cx) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  const uint32_t* bq = bounds + (size_t)m * BOUNDS_STRIDE;
  float lo[3], hi[3];
  bool empty = false;
  for (int k = 0; k < 3; ++k) {
    lo[k] = o2f(bq[k]);
    hi[k] = o2f(bq[3 + k]);
    if (!(hi[k] >= lo[k])) empty = true;
  }
  Grid g;
  if (empty) {
    g = Grid{0.f, 0.f, 0.f, 1.f, 1, 1, 1, 0};
    for (int k = 0; k < 4; ++k) cx[4 * m + k] = 0.0;
    grids[m] = g;
    return;
  }
  const double ext_sum = __longlong_as_double((long long)((uint64_t)bq[8] | ((uint64_t)bq[9] << 32)));
  double X = 0.0;
  for (int k = 0; k < 3; ++k) {
    cx[4 * m + k] = 0.5 * ((double)lo[k] + (double)hi[k]);
    X = fmax(X, 0.5 * ((double)hi[k] - (double)lo[k]) * (1.0 + 1e-6));
  }
  cx[4 * m + 3] = X;
  const int npm = max(1, mp[m].n_prims);
  double c = cell_factor * (ext_sum / npm);
  if (!(c > 0)) c = 1.0;
  c = exp2(floor(log2(c) * 4.0) / 4.0);
  for (int k = 0; k < 3; ++k) {
    const double span = (double)hi[k] - (double)lo[k];
    if (span / c > 1000.0) c = span / 1000.0;
  }
  g.inv = (float)(1.0 / c);
  g.ox = lo[0];
  g.oy = lo[1];
  g.oz = lo[2];
  int d3[3];
  for (int k = 0; k < 3; ++k) {
    const double span = (double)hi[k] - (double)lo[k];
    const int d = (int)floor(span * (double)g.inv) + 2;
    d3[k] = min(max(d, 1), 1024);
  }
  g.dx = d3[0];
  g.dy = d3[1];
  g.dz = d3[2];
  g.pad = 0;
  grids[m] = g;
}

__device__ __forceinline__ int cell_of(float v, float o, float inv, int dim) {
  float tt = __fmul_rn(__fsub_rn(v, o), inv);
  int c = (int)floorf(tt);
  return min(max(c, 0), dim - 1);
}

__device__ __forceinline__ uint32_t spread10(uint32_t v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}
__device__ __forceinline__ uint32_t morton(int x, int y, int z) {
  return spread10((uint32_t)x) | (spread10((uint32_t)y) << 1) | (spread10((uint32_t)z) << 2);
}
// x cell index of a Morton cell code (every third bit from bit 0)
__device__ __forceinline__ int morton_x(uint32_t m) {
  uint32_t v = m & 0x09249249u;
  v = (v ^ (v >> 2)) & 0x030C30C3u;
  v = (v ^ (v >> 4)) & 0x0300F00Fu;
  v = (v ^ (v >> 8)) & 0x030000FFu;
  v = (v ^ (v >> 16)) & 0x000003FFu;
  return (int)v;
}

// Shell cells are swept along x: within each type group of a cell, entries
// are sorted by the position of their box's lower x bound inside the cell,
// quantized to XQ_LEVELS steps.  The map is monotone (FP32 operations with
// the rounding written out, then floor and clamp), so a partner whose level
// is above the level of an entry's upper x bound lies beyond it, and so does
// every partner after it: the entry's scan stops there.
constexpr int XQ_BITS = 10, XQ_LEVELS = 1 << XQ_BITS;
constexpr int SWEEP_SHIFT = XQ_BITS + 2;  // cell code above [type group : 2][x level : XQ_BITS]
__device__ __forceinline__ uint32_t x_level(float v, const Grid& G, int cx) {
  const float tt = __fmul_rn(__fsub_rn(v, G.ox), G.inv);
  const float f = __fmul_rn(__fsub_rn(tt, (float)cx), (float)XQ_LEVELS);
  const float q = floorf(f);
  return q <= 0.f ? 0u : (q >= (float)(XQ_LEVELS - 1) ? (uint32_t)(XQ_LEVELS - 1) : (uint32_t)q);
}

__global__ void k_cell_count(Topo t, int np, const float4* __restrict__ box32, const int32_t* __restrict__ vsc,
                             const Grid* __restrict__ grids, uint32_t* __restrict__ cnt) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= np) return;
  const Grid g = grids[prim_member(t, vsc, q)];
  float4 lo = box32[2 * (size_t)q], hi = box32[2 * (size_t)q + 1];
  int nx = cell_of(hi.x, g.ox, g.inv, g.dx) - cell_of(lo.x, g.ox, g.inv, g.dx) + 1;
  int ny = cell_of(hi.y, g.oy, g.inv, g.dy) - cell_of(lo.y, g.oy, g.inv, g.dy) + 1;
  int nz = cell_of(hi.z, g.oz, g.inv, g.dz) - cell_of(lo.z, g.oz, g.inv, g.dz) + 1;
  cnt[q] = (uint32_t)(nx * ny * nz);
}

__global__ void k_cell_fill(Topo t, int np, const float4* __restrict__ box32, const int32_t* __restrict__ vsc,
                            const Grid* __restrict__ grids, const uint32_t* __restrict__ off,
                            uint64_t* __restrict__ ekey, uint32_t* __restrict__ eval, bool sweep) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= np) return;
  const int mem = prim_member(t, vsc, q);
  const Grid g = grids[mem];
  float4 lo = box32[2 * (size_t)q], hi = box32[2 * (size_t)q + 1];
  int x0 = cell_of(lo.x, g.ox, g.inv, g.dx), x1 = cell_of(hi.x, g.ox, g.inv, g.dx);
  int y0 = cell_of(lo.y, g.oy, g.inv, g.dy), y1 = cell_of(hi.y, g.oy, g.inv, g.dy);
  int z0 = cell_of(lo.z, g.oz, g.inv, g.dz), z1 = cell_of(hi.z, g.oz, g.inv, g.dz);
  uint32_t w = off[q];
  const uint64_t mbits = (uint64_t)mem << 30;
  // shells: type group (vertex 0, triangle 1, edge 2) and x level below the cell code
  const uint32_t grp = q < t.n ? 0u : (q < t.n + t.T ? 1u : 2u);
  for (int z = z0; z <= z1; ++z)
    for (int y = y0; y <= y1; ++y)
      for (int xx = x0; xx <= x1; ++xx) {
        const uint64_t cell = mbits | morton(xx, y, z);
        ekey[w] = sweep ? (cell << SWEEP_SHIFT) | ((uint64_t)grp << XQ_BITS) | x_level(lo.x, g, xx) : cell;
        eval[w] = (uint32_t)q;
        ++w;
      }
}

// boxes in entry order, so that the pair loops read their run contiguously
__global__ void k_gather_boxes(int64_t ne, const uint32_t* __restrict__ eval, const float4* __restrict__ box32,
                               float4* __restrict__ ebox) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ne) return;
  const uint32_t q = eval[i];
  ebox[2 * i] = box32[2 * (size_t)q];
  ebox[2 * i + 1] = box32[2 * (size_t)q + 1];
}

__global__ void k_run_flag(int64_t ne, const uint64_t* __restrict__ key, int shift, uint32_t* __restrict__ flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ne) return;
  flag[i] = (i == 0 || (key[i] >> shift) != (key[i - 1] >> shift)) ? 1u : 0u;
}

// run_id[i] = index of the run holding entry i; run_start[r] = first entry of run r
__global__ void k_run_start(int64_t ne, const uint32_t* __restrict__ flag, const uint32_t* __restrict__ excl,
                            uint32_t* __restrict__ run_id, uint32_t* __restrict__ run_start) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ne) return;
  uint32_t f = flag[i], e = excl[i];
  run_id[i] = e + f - 1u;
  if (f) run_start[e] = (uint32_t)i;
  if (i == ne - 1) run_start[e + f] = (uint32_t)ne;
}

// the IEEE-754 neighbours of a float towards +inf and -inf, from its bit
// pattern (a float's successor is the next integer bit pattern for x >= +0
// and the previous one for x < 0; -0 steps to the smallest subnormal; +inf
// and -inf stay where they are)
__device__ __forceinline__ float nextup(float v) {
  const int u = __float_as_int(v);
  if (u == (int)0x80000000) return __int_as_float(1);
  if (u == 0x7f800000) return v;
  return __int_as_float(u >= 0 ? u + 1 : u - 1);
}
__device__ __forceinline__ float nextdn(float v) { return -nextup(-v); }

// first index in [lo, hi) of a shell cell's run whose type group is >= g
// (the run's keys share the cell code and ascend by group, then x level)
__device__ __forceinline__ int lower_bound_group(const uint64_t* __restrict__ key, int lo, int hi, uint32_t g) {
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if ((uint32_t)((key[mid] >> XQ_BITS) & 3u) < g) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// pairs a rod entry's thread keeps from the count pass for the fill pass
// (larger counts are found again by the fill pass's tests)
constexpr int PAIR_STAGE = 32;

struct PairArgs {
  Topo t;
  int64_t ne;
  const uint64_t* __restrict__ ekey;
  const uint32_t* __restrict__ eval;
  const uint32_t* __restrict__ run_id;
  const uint32_t* __restrict__ run_start;
  const float4* __restrict__ box32;
  const float4* __restrict__ ebox;   // boxes in entry order: entry j at [2 j], [2 j + 1]
  const double* __restrict__ box64;
  const Grid* __restrict__ grids;
  int bi, bj;
  int shift;                   // bits of type group and x level below the cell code (shells: swept)
  unsigned long long* fpstat;  // count pass: [0] FP32-accepted pairs, [1] FP64-decided (may be null)
  bool canonical;              // fill pass: write canonical keys (else compact ones for the sort)
};

// An entry's partners: entries [j0, j1) of its run s..e (none for a triangle
// entry of a shell cell), the key type and the id offsets of the two sides.
struct EntryRange {
  uint32_t P, type, ibase, jbase;
  int s, e, j0, j1;
  bool none;
};

__device__ __forceinline__ EntryRange entry_range(const PairArgs& A, int64_t i) {
  const Topo& t = A.t;
  EntryRange R;
  R.P = A.eval[i];
  const uint32_t r = A.run_id[i];
  R.s = (int)A.run_start[r];
  R.e = (int)A.run_start[r + 1];
  R.ibase = R.jbase = 0;
  R.none = false;
  if (t.kind == CB_ROD) {
    R.j0 = (int)i + 1;
    R.j1 = R.e;
    R.type = CB_KEY_ROD_EE;
  } else if (R.P < (uint32_t)t.n) {
    R.j0 = lower_bound_group(A.ekey, R.s, R.e, 1u);
    R.j1 = lower_bound_group(A.ekey, R.j0, R.e, 2u);
    R.type = CB_KEY_PT;
    R.jbase = (uint32_t)t.n;
  } else if (R.P < (uint32_t)(t.n + t.T)) {
    R.j0 = R.j1 = 0;
    R.type = 0;
    R.none = true;
  } else {
    R.j0 = (int)i + 1;
    R.j1 = R.e;
    R.type = CB_KEY_EE;
    R.ibase = R.jbase = (uint32_t)(t.n + t.T);
  }
  return R;
}

// key of the pair (k1, k2) (ids already relative to their kind): canonical,
// or compact (type | k1 | k2 in bi + bj bits) for the sort
__device__ __forceinline__ uint64_t pair_key(const PairArgs& A, uint32_t type, uint32_t k1, uint32_t k2) {
  return A.canonical ? cb_key(type, k1, k2)
                     : (((uint64_t)type << (A.bi + A.bj)) | ((uint64_t)k1 << A.bj) | (uint64_t)k2);
}

// Rod cells: the pairs one entry reports, in a fixed order (the count and the
// fill pass make the same decisions).  Rod cells hold many edges (yarn
// segments crowd the cells of a knit or weave), so the m (m - 1) / 2 tests of
// a cell are shared by its m entries in round-robin order (entry a with
// a + 1, ..., a + (m - 1) / 2 mod m, and with a + m/2 for a < m/2 when m is
// even): every thread makes about (m - 1) / 2 tests instead of the first one
// m - 1 and the last none.  The count pass keeps an entry's first PAIR_STAGE
// keys (element-major, stage[k * ne + i]) and lists entries with more in ovl.
template <bool FILL>
__device__ __forceinline__ void rod_pairs_of_entry(const PairArgs& A, int64_t i, uint32_t* __restrict__ cnt,
                                                   const uint32_t* __restrict__ off, uint64_t* __restrict__ out,
                                                   uint64_t* __restrict__ stage, uint32_t* __restrict__ ovl,
                                                   unsigned int* __restrict__ novl) {
  const Topo& t = A.t;
  const EntryRange R = entry_range(A, i);
  const uint32_t P = R.P;
  const uint64_t kc = A.ekey[i] >> A.shift;
  const Grid G = A.grids[kc >> 30];
  const float4 plo = A.ebox[2 * (size_t)i], phi = A.ebox[2 * (size_t)i + 1];
  int pv[3];
  prim_verts(t, (int)P, pv);
  uint32_t count = 0, n32 = 0, n64 = 0;
  // the fill pass re-makes the count pass's decisions; never write past them
  const uint32_t c_end = FILL ? cnt[i] : 0;
  constexpr uint32_t K = PAIR_STAGE;
  const int m = R.e - R.s, a = (int)(i - R.s);
  const int jn = (m % 2 == 0 && a < m / 2) ? m / 2 : (m - 1) / 2;
  for (int jj = 0; jj < jn; ++jj) {
    int j = a + 1 + jj;
    if (j >= m) j -= m;
    j += R.s;
    const float4 qlo = A.ebox[2 * (size_t)j], qhi = A.ebox[2 * (size_t)j + 1];
    const uint32_t Q = A.eval[j];
    bool acc = false;
    if (plo.x <= qhi.x && qlo.x <= phi.x && plo.y <= qhi.y && qlo.y <= phi.y && plo.z <= qhi.z &&
        qlo.z <= phi.z) {
      // home cell: low corner of the intersection
      const uint32_t hc = morton(cell_of(fmaxf(plo.x, qlo.x), G.ox, G.inv, G.dx),
                                 cell_of(fmaxf(plo.y, qlo.y), G.oy, G.inv, G.dy),
                                 cell_of(fmaxf(plo.z, qlo.z), G.oz, G.inv, G.dz));
      if (hc == (uint32_t)(kc & 0x3fffffffull)) {
        int qv[3];
        prim_verts(t, (int)Q, qv);
        bool inc = false;
#pragma unroll
        for (int u = 0; u < 3; ++u)
#pragma unroll
          for (int b = 0; b < 3; ++b) inc |= (pv[u] >= 0 && pv[u] == qv[b]);
        if (!inc) {
          const bool sure = nextup(plo.x) <= nextdn(qhi.x) && nextup(qlo.x) <= nextdn(phi.x) &&
                            nextup(plo.y) <= nextdn(qhi.y) && nextup(qlo.y) <= nextdn(phi.y) &&
                            nextup(plo.z) <= nextdn(qhi.z) && nextup(qlo.z) <= nextdn(phi.z);
          ++n32;
          acc = true;
          if (!sure) {
            ++n64;
            const double* b1 = A.box64 + (size_t)P * 6;
            const double* b2 = A.box64 + (size_t)Q * 6;
#pragma unroll
            for (int k = 0; k < 3; ++k) acc = acc && (b1[k] <= b2[3 + k]) && (b2[k] <= b1[3 + k]);
          }
        }
      }
    }
    if (acc) {
      // the pair's key takes the lower primitive first (round-robin order)
      const bool swap = j < (int)i;
      const uint64_t key = pair_key(A, R.type, (swap ? Q : P) - R.ibase, (swap ? P : Q) - R.jbase);
      if (FILL) {
        // the pairs past the staged ones, at their place in the entry's range
        if (count >= K && count < c_end) out[(size_t)off[i] + count] = key;
      } else if (count < K) {
        stage[(size_t)count * A.ne + i] = key;
      }
      ++count;
    }
  }
  if (!FILL) {
    cnt[i] = count;
    if (count > K) ovl[atomicAdd(novl, 1u)] = (uint32_t)i;
    if (A.fpstat) {  // one atomic per converged group of lanes
      const unsigned mask = __activemask();
      const unsigned a32 = __reduce_add_sync(mask, n32), a64 = __reduce_add_sync(mask, n64);
      if ((int)(threadIdx.x & 31) == __ffs(mask) - 1) {
        if (a32) atomicAdd(&A.fpstat[0], (unsigned long long)a32);
        if (a64) atomicAdd(&A.fpstat[1], (unsigned long long)a64);
      }
    }
  }
}

// rod cells, count pass (FILL = false, one thread per entry): cnt[i] = number
// of pairs entry i reports; the fill pass (FILL = true) then runs over the
// entries listed in ovl only, writing their pairs past the staged ones
template <bool FILL>
__global__ void __launch_bounds__(CB_THREADS) k_rod_pairs(PairArgs A, uint32_t* __restrict__ cnt,
                                                          const uint32_t* __restrict__ off,
                                                          uint64_t* __restrict__ out, uint64_t* __restrict__ stage,
                                                          uint32_t* __restrict__ ovl, unsigned int* __restrict__ novl) {
  if (!FILL) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < A.ne) rod_pairs_of_entry<FILL>(A, i, cnt, off, out, stage, ovl, novl);
  } else {
    const unsigned m = *novl;
    for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < m; q += gridDim.x * blockDim.x)
      rod_pairs_of_entry<true>(A, ovl[q], cnt, off, out, stage, ovl, novl);
  }
}

// ---- shells: the pair tests spread evenly over the threads ----------------
// An entry's partner range (the swept part of its run: every triangle entry
// of its cell for a vertex entry, every later edge entry for an edge entry,
// up to the first partner whose x level lies above its own upper bound) has
// any length from 0 to thousands, so one thread per entry leaves most lanes
// of a warp idle.  Here the ranges are laid end to end: entry i owns the test
// slots [toff[i], toff[i+1]) (an exclusive scan of the lengths), slot f of
// entry i tests partner j = j0[i] + (f - toff[i]).  A warp takes 32 x
// FLAT_STEPS consecutive slots, lane l the slots with f = l (mod 32), so each
// step tests 32 neighbouring partners (coalesced box loads) and its ballot is
// one word of the hit bits.  The pairs come out in the same order as before
// (entry by entry, partners ascending), so the candidate array is unchanged.
constexpr int FLAT_STEPS = 32;
// Entries with fewer partners than this keep their hits in one word each and
// are tested warp by warp (k_pairs_short); only longer ranges are laid end
// to end, so a lane of the end-to-end pass moves to a new entry at most once
// per step.  (Thresholds of 64 and 128 partners measured the same.)
constexpr int FLAT_MIN = 32;

// entry i's first partner j0[i] and the length of its swept range: short
// ranges in slen[i], long ones in len[i] with lflag[i] = 1 (lflag[ne] = 0)
__global__ void k_flat_ranges(PairArgs A, uint32_t* __restrict__ len, uint32_t* __restrict__ lflag,
                              uint8_t* __restrict__ slen, uint32_t* __restrict__ j0s) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > A.ne) return;
  if (i == A.ne) {
    lflag[i] = 0;
    return;
  }
  const EntryRange R = entry_range(A, i);
  if (R.none) {
    len[i] = 0;
    lflag[i] = 0;
    slen[i] = 0;
    j0s[i] = 0;
    return;
  }
  const uint64_t kc = A.ekey[i] >> A.shift;
  const Grid G = A.grids[kc >> 30];
  const int cxi = morton_x((uint32_t)(kc & 0x3fffffffull));
  const uint32_t xhi = x_level(A.ebox[2 * (size_t)i + 1].x, G, cxi);
  // partners of one cell and group are sorted by x level (the key's low bits)
  int lo = R.j0, hi = R.j1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if ((uint32_t)(A.ekey[mid] & (uint64_t)(XQ_LEVELS - 1)) <= xhi) lo = mid + 1;
    else hi = mid;
  }
  const uint32_t n = (uint32_t)(lo - R.j0);
  const bool lng = n >= (uint32_t)FLAT_MIN;
  len[i] = lng ? n : 0u;
  lflag[i] = lng ? 1u : 0u;
  slen[i] = lng ? (uint8_t)0 : (uint8_t)n;
  j0s[i] = (uint32_t)R.j0;
}

// the long entries in entry order: lidx[k] = i, llen[k] = len[i] (k = lpos[i])
__global__ void k_flat_compact(int64_t ne, const uint32_t* __restrict__ lflag, const uint32_t* __restrict__ lpos,
                               const uint32_t* __restrict__ len, uint32_t* __restrict__ lidx,
                               uint32_t* __restrict__ llen) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ne || !lflag[i]) return;
  lidx[lpos[i]] = (uint32_t)i;
  llen[lpos[i]] = len[i];
}

struct FlatEntry {
  int pv[3];
  float4 plo, phi;
  uint32_t P;
  int cx, cy, cz;  // the cell's coordinates (its Morton code decoded)
  Grid G;
};

__device__ __forceinline__ void flat_load(const PairArgs& A, int64_t i, FlatEntry& E) {
  E.P = A.eval[i];
  prim_verts(A.t, (int)E.P, E.pv);
  E.plo = A.ebox[2 * (size_t)i];
  E.phi = A.ebox[2 * (size_t)i + 1];
  const uint64_t kc = A.ekey[i] >> A.shift;
  const uint32_t cell = (uint32_t)(kc & 0x3fffffffull);
  E.cx = morton_x(cell);
  E.cy = morton_x(cell >> 1);
  E.cz = morton_x(cell >> 2);
  E.G = A.grids[kc >> 30];
}

__device__ __forceinline__ bool box_overlap(const float4& plo, const float4& phi, const float4& qlo,
                                            const float4& qhi) {
  return plo.x <= qhi.x && qlo.x <= phi.x && plo.y <= qhi.y && qlo.y <= phi.y && plo.z <= qhi.z && qlo.z <= phi.z;
}

// the test of a pair whose FP32 boxes overlap: the overlap's low corner lies
// in this cell (each pair is reported by one cell), the two share no vertex;
// the FP64 boxes decide where the FP32 margins cannot
__device__ __forceinline__ bool flat_rest(const PairArgs& A, const FlatEntry& E, const float4& qlo,
                                          const float4& qhi, int j, uint32_t& n32, uint32_t& n64) {
  const Grid& G = E.G;
  if (cell_of(fmaxf(E.plo.x, qlo.x), G.ox, G.inv, G.dx) != E.cx ||
      cell_of(fmaxf(E.plo.y, qlo.y), G.oy, G.inv, G.dy) != E.cy ||
      cell_of(fmaxf(E.plo.z, qlo.z), G.oz, G.inv, G.dz) != E.cz)
    return false;
  const uint32_t Q = A.eval[j];
  int qv[3];
  prim_verts(A.t, (int)Q, qv);
  bool inc = false;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) inc |= (E.pv[a] >= 0 && E.pv[a] == qv[b]);
  if (inc) return false;
  const bool sure = nextup(E.plo.x) <= nextdn(qhi.x) && nextup(qlo.x) <= nextdn(E.phi.x) &&
                    nextup(E.plo.y) <= nextdn(qhi.y) && nextup(qlo.y) <= nextdn(E.phi.y) &&
                    nextup(E.plo.z) <= nextdn(qhi.z) && nextup(qlo.z) <= nextdn(E.phi.z);
  ++n32;
  if (sure) return true;
  ++n64;
  const double* b1 = A.box64 + (size_t)E.P * 6;
  const double* b2 = A.box64 + (size_t)Q * 6;
  bool acc = true;
#pragma unroll
  for (int k = 0; k < 3; ++k) acc = acc && (b1[k] <= b2[3 + k]) && (b2[k] <= b1[3 + k]);
  return acc;
}

// The box test is cheap, while the rest of the test (home cell, shared
// vertices, FP32 margins) is long, and a warp whose lanes disagree runs it
// for all of them.  So the end-to-end kernel splits the two: each step's box
// overlaps go to a small per-warp queue in shared memory (entry, partner,
// and the hit bit to set: word t >> 5, bit t & 31 of a per-warp array), and
// the rest of the test runs 32 queued slots at a time with every lane busy,
// the remainder at the end.  (The same split in the short-range kernel
// measured slower: its lanes already take their entries' data by shuffles.)
constexpr int FLAT_WARPS = 8;  // warps per block of k_pairs_flat
static_assert(FLAT_STEPS == 32, "one hit word per lane at the end of a chunk");

// the rest of the test for queued slots q0 .. q0 + cnt - 1, one per lane
__device__ __forceinline__ void flat_batch(const PairArgs& A, const uint32_t* qi, const uint32_t* qj,
                                           const uint16_t* qs, int q0, int cnt, uint32_t* cw, uint32_t& n32,
                                           uint32_t& n64) {
  const int lane = threadIdx.x & 31;
  if (lane >= cnt) return;
  const uint32_t i = qi[q0 + lane], j = qj[q0 + lane];
  const int sl = qs[q0 + lane];
  FlatEntry E;
  flat_load(A, i, E);
  const float4 qlo = A.ebox[2 * (size_t)j], qhi = A.ebox[2 * (size_t)j + 1];
  if (flat_rest(A, E, qlo, qhi, (int)j, n32, n64)) atomicOr(&cw[sl >> 5], 1u << (sl & 31));
}

// the whole test of entry E against partner j
__device__ __forceinline__ bool flat_test(const PairArgs& A, const FlatEntry& E, int j, uint32_t& n32,
                                          uint32_t& n64) {
  const float4 qlo = A.ebox[2 * (size_t)j], qhi = A.ebox[2 * (size_t)j + 1];
  return box_overlap(E.plo, E.phi, qlo, qhi) && flat_rest(A, E, qlo, qhi, j, n32, n64);
}

// Entries with short ranges, a warp per 32 consecutive entries: the warp
// scans their lengths (with shuffles) and lays their partners end to end, and
// each step tests 32 of those (entry, partner) slots, lane l the slot
// base + l -- its entry is the last lane whose range starts at or before the
// slot (a search over the lanes' starts), whose data the lane takes by
// shuffles.  Hit bit b of an entry's word is its partner j0 + b.
__global__ void __launch_bounds__(256) k_pairs_short(PairArgs A, const uint8_t* __restrict__ slen,
                                                     const uint32_t* __restrict__ j0s,
                                                     uint32_t* __restrict__ sbits) {
  __shared__ uint32_t sw[256];  // the hit word of each entry of the block
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int n = i < A.ne ? (int)slen[i] : 0;
  sw[threadIdx.x] = 0u;
  int inc = n;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(full, inc, o);
    if (lane >= o) inc += v;
  }
  const int ex = inc - n;                        // this entry's first slot
  const int total = __shfl_sync(full, inc, 31);  // slots of the warp's entries
  FlatEntry E{};
  int j0 = 0;
  if (n > 0) {
    flat_load(A, i, E);
    j0 = (int)j0s[i];
  }
  uint32_t n32 = 0, n64 = 0;
  __syncwarp();
  for (int base = 0; base < total; base += 32) {
    const int sl = base + lane;
    int e = 0;  // the last lane whose range starts at or before sl
#pragma unroll
    for (int bit = 16; bit > 0; bit >>= 1) {
      const int c = e + bit;
      if (__shfl_sync(full, ex, c) <= sl) e = c;
    }
    FlatEntry F;
    F.P = __shfl_sync(full, E.P, e);
    F.cx = __shfl_sync(full, E.cx, e);
    F.cy = __shfl_sync(full, E.cy, e);
    F.cz = __shfl_sync(full, E.cz, e);
#pragma unroll
    for (int k = 0; k < 3; ++k) F.pv[k] = __shfl_sync(full, E.pv[k], e);
    F.plo = make_float4(__shfl_sync(full, E.plo.x, e), __shfl_sync(full, E.plo.y, e),
                        __shfl_sync(full, E.plo.z, e), 0.f);
    F.phi = make_float4(__shfl_sync(full, E.phi.x, e), __shfl_sync(full, E.phi.y, e),
                        __shfl_sync(full, E.phi.z, e), 0.f);
    F.G.ox = __shfl_sync(full, E.G.ox, e);
    F.G.oy = __shfl_sync(full, E.G.oy, e);
    F.G.oz = __shfl_sync(full, E.G.oz, e);
    F.G.inv = __shfl_sync(full, E.G.inv, e);
    F.G.dx = __shfl_sync(full, E.G.dx, e);
    F.G.dy = __shfl_sync(full, E.G.dy, e);
    F.G.dz = __shfl_sync(full, E.G.dz, e);
    const int b = sl - __shfl_sync(full, ex, e);
    const int j = __shfl_sync(full, j0, e) + b;
    if (sl < total && flat_test(A, F, j, n32, n64)) atomicOr(&sw[(threadIdx.x & ~31) + e], 1u << b);
  }
  __syncwarp();
  if (i < A.ne) sbits[i] = sw[threadIdx.x];
  if (A.fpstat) {
    const unsigned a32 = __reduce_add_sync(full, n32), a64 = __reduce_add_sync(full, n64);
    if (lane == 0) {
      if (a32) atomicAdd(&A.fpstat[0], (unsigned long long)a32);
      if (a64) atomicAdd(&A.fpstat[1], (unsigned long long)a64);
    }
  }
}

// hit bits of slots [0, T): word w holds slots 32 w .. 32 w + 31 (grid-stride
// over chunks of FLAT_STEPS = 32 words, one warp per chunk); the queued rest
// of the test sets bits of the chunk's 32 words in shared memory
__global__ void __launch_bounds__(32 * FLAT_WARPS) k_pairs_flat(PairArgs A, const uint64_t* __restrict__ toff,
                                                                const uint32_t* __restrict__ lidx,
                                                                const uint32_t* __restrict__ j0s, uint64_t T,
                                                                uint32_t* __restrict__ bits) {
  __shared__ uint32_t s_qi[FLAT_WARPS][64], s_qj[FLAT_WARPS][64], s_cw[FLAT_WARPS][32];
  __shared__ uint16_t s_qs[FLAT_WARPS][64];
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
  const unsigned below = (1u << lane) - 1u;
  uint32_t* qi = s_qi[wb];
  uint32_t* qj = s_qj[wb];
  uint16_t* qs = s_qs[wb];
  uint32_t* cw = s_cw[wb];
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const uint64_t chunk = 32ull * FLAT_STEPS;
  const int64_t nchunks = (int64_t)((T + chunk - 1) / chunk);
  uint32_t n32 = 0, n64 = 0;
  for (int64_t ch = warp; ch < nchunks; ch += nwarps) {
    const uint64_t base = (uint64_t)ch * chunk;
    // slots of this chunk (the last one may be short), counted from base
    const uint32_t nvalid = (uint32_t)(T - base < chunk ? T - base : chunk);
    // the long entry of this lane's first slot: the last k with toff[k] <= f
    // (toff runs over the long entries, then stays at T)
    int64_t k = 0;
    {
      int64_t lo = 0, hi = A.ne + 1;
      const uint64_t fs = base + (lane < (int)nvalid ? (uint64_t)lane : (uint64_t)(nvalid - 1));
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (toff[mid] <= fs) lo = mid + 1;
        else hi = mid;
      }
      k = lo - 1;
    }
    uint32_t i = lidx[k];
    float4 plo = A.ebox[2 * (size_t)i], phi = A.ebox[2 * (size_t)i + 1];
    // the entry's end and its partner offset, relative to base (a range that
    // ends past the chunk reads as ending at the chunk's end)
    uint64_t e_end = toff[k + 1];
    uint32_t r_end = (uint32_t)(e_end - base < chunk ? e_end - base : chunk);
    int64_t jofs = (int64_t)j0s[i] - (int64_t)(toff[k] - base);
    cw[lane] = 0u;
    int qn = 0;  // queued slots (fewer than 32 between steps)
    __syncwarp();
    for (int b = 0; b < FLAT_STEPS; ++b) {
      const uint32_t sl = 32u * (uint32_t)b + (uint32_t)lane;
      bool pass = false;
      int j = 0;
      if (sl < nvalid) {
        if (sl >= r_end) {
          // every long range holds at least 32 slots: the next entry
          uint64_t e_beg;
          do {
            ++k;
            e_beg = e_end;
            e_end = toff[k + 1];
          } while (base + sl >= e_end);
          i = lidx[k];
          plo = A.ebox[2 * (size_t)i];
          phi = A.ebox[2 * (size_t)i + 1];
          r_end = (uint32_t)(e_end - base < chunk ? e_end - base : chunk);
          jofs = (int64_t)j0s[i] - (int64_t)(e_beg - base);
        }
        j = (int)(jofs + (int64_t)sl);
        pass = box_overlap(plo, phi, A.ebox[2 * (size_t)j], A.ebox[2 * (size_t)j + 1]);
      }
      const unsigned m = __ballot_sync(full, pass);
      if (pass) {
        const int at = qn + __popc(m & below);
        qi[at] = i;
        qj[at] = (uint32_t)j;
        qs[at] = (uint16_t)sl;
      }
      qn += __popc(m);
      __syncwarp();
      if (qn >= 32) {
        flat_batch(A, qi, qj, qs, qn - 32, 32, cw, n32, n64);
        qn -= 32;
        __syncwarp();  // the batch's slots are read before the next appends
      }
    }
    if (qn > 0) flat_batch(A, qi, qj, qs, 0, qn, cw, n32, n64);
    __syncwarp();
    if (32u * (uint32_t)lane < nvalid) bits[(base >> 5) + (uint64_t)lane] = cw[lane];
    __syncwarp();
  }
  if (A.fpstat) {
    const unsigned a32 = __reduce_add_sync(full, n32), a64 = __reduce_add_sync(full, n64);
    if (lane == 0) {
      if (a32) atomicAdd(&A.fpstat[0], (unsigned long long)a32);
      if (a64) atomicAdd(&A.fpstat[1], (unsigned long long)a64);
    }
  }
}

// the hit bits of slots [f0, f1) in word wd
__device__ __forceinline__ uint32_t flat_word(const uint32_t* __restrict__ bits, uint64_t wd, uint64_t f0,
                                              uint64_t f1) {
  uint32_t word = bits[wd];
  const uint64_t w0 = wd << 5;
  if (f0 > w0) word &= 0xffffffffu << (uint32_t)(f0 - w0);
  if (f1 < w0 + 32) word &= 0xffffffffu >> (uint32_t)(w0 + 32 - f1);
  return word;
}

// Slots of an entry's range from which its pairs are written by a warp
// (k_flat_emit_long) rather than by the entry's thread: shorter ranges
// would leave most of the warp's lanes without a word.
constexpr uint64_t FLAT_EMIT_WARP = 256;

// pairs per entry: the hits of its short word or of its slots; the long
// entries of FLAT_EMIT_WARP slots or more are listed (by their index among
// the long entries, in no particular order) for k_flat_emit_long
__global__ void k_flat_count(int64_t ne, const uint64_t* __restrict__ toff, const uint32_t* __restrict__ lflag,
                             const uint32_t* __restrict__ lpos, const uint32_t* __restrict__ bits,
                             const uint32_t* __restrict__ sbits, uint32_t* __restrict__ cnt,
                             uint32_t* __restrict__ vlong, unsigned int* __restrict__ nvlong) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ne) return;
  uint32_t c = __popc(sbits[i]);
  const uint64_t f0 = lflag[i] ? toff[lpos[i]] : 0, f1 = lflag[i] ? toff[lpos[i] + 1] : 0;
  if (f1 > f0)
    for (uint64_t wd = f0 >> 5; wd <= (f1 - 1) >> 5; ++wd) c += __popc(flat_word(bits, wd, f0, f1));
  cnt[i] = c;
  if (f1 > f0 && f1 - f0 >= FLAT_EMIT_WARP) vlong[atomicAdd(nvlong, 1u)] = lpos[i];
}

// entry i's pairs at off[i], partners ascending (edge-edge keys take the
// lower edge first: swept cells order edges by x, not by id)
__global__ void k_flat_emit(PairArgs A, const uint64_t* __restrict__ toff, const uint32_t* __restrict__ lflag,
                            const uint32_t* __restrict__ lpos, const uint32_t* __restrict__ j0s,
                            const uint32_t* __restrict__ bits, const uint32_t* __restrict__ sbits,
                            const uint32_t* __restrict__ cnt, const uint32_t* __restrict__ off,
                            uint64_t* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.ne || cnt[i] == 0) return;
  const uint32_t P = A.eval[i];
  const Topo& t = A.t;
  uint32_t type, ibase = 0, jbase = 0;
  if (P < (uint32_t)t.n) {
    type = CB_KEY_PT;
    jbase = (uint32_t)t.n;
  } else {
    type = CB_KEY_EE;
    ibase = jbase = (uint32_t)(t.n + t.T);
  }
  const uint64_t f0 = lflag[i] ? toff[lpos[i]] : 0, f1 = lflag[i] ? toff[lpos[i] + 1] : 0;
  const uint32_t j0 = j0s[i];
  size_t o = off[i];
  for (uint32_t word = sbits[i]; word;) {  // a short range
    const uint32_t b = (uint32_t)__ffs(word) - 1u;
    word &= word - 1u;
    const uint32_t Q = A.eval[j0 + b];
    const bool swap = type == CB_KEY_EE && Q < P;
    out[o++] = pair_key(A, type, (swap ? Q : P) - ibase, (swap ? P : Q) - jbase);
  }
  if (f1 > f0 && f1 - f0 < FLAT_EMIT_WARP) {  // a long range, not long enough for k_flat_emit_long
    for (uint64_t wd = f0 >> 5; wd <= (f1 - 1) >> 5; ++wd) {
      uint32_t word = flat_word(bits, wd, f0, f1);
      while (word) {
        const uint32_t b = (uint32_t)__ffs(word) - 1u;
        word &= word - 1u;
        const uint32_t Q = A.eval[j0 + (uint32_t)((wd << 5) + b - f0)];
        const bool swap = type == CB_KEY_EE && Q < P;
        out[o++] = pair_key(A, type, (swap ? Q : P) - ibase, (swap ? P : Q) - jbase);
      }
    }
  }
}

// The pairs of the entries with at least FLAT_EMIT_WARP slots (laid end to
// end), after their short pairs: a warp per entry, lane l taking hit word l
// of each run of 32, a warp scan of the words' hit counts placing each
// lane's pairs, so that the warp writes one contiguous run per 32 words.
// Grid-stride over the list k_flat_count made of those entries (*nvlong of
// them), so that neighbouring heavy entries go to different warps.
__global__ void __launch_bounds__(256) k_flat_emit_long(PairArgs A, const uint64_t* __restrict__ toff,
                                                        const uint32_t* __restrict__ lidx,
                                                        const uint32_t* __restrict__ vlong,
                                                        const unsigned int* __restrict__ nvlong,
                                                        const uint32_t* __restrict__ j0s,
                                                        const uint32_t* __restrict__ bits,
                                                        const uint32_t* __restrict__ sbits,
                                                        const uint32_t* __restrict__ off, uint64_t* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t nv = *nvlong;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const Topo& t = A.t;
  for (int64_t v = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); v < nv; v += nwarps) {
    const uint32_t wl = vlong[v];
    const uint64_t f0 = toff[wl], f1 = toff[wl + 1];
    const uint32_t i = lidx[wl];
    const uint32_t P = A.eval[i];
    uint32_t type, ibase = 0, jbase = 0;
    if (P < (uint32_t)t.n) {
      type = CB_KEY_PT;
      jbase = (uint32_t)t.n;
    } else {
      type = CB_KEY_EE;
      ibase = jbase = (uint32_t)(t.n + t.T);
    }
    const uint32_t j0 = j0s[i];
    size_t o = (size_t)off[i] + (size_t)__popc(sbits[i]);
    const uint64_t w_end = (f1 - 1) >> 5;
    for (uint64_t w0 = f0 >> 5; w0 <= w_end; w0 += 32) {
      const uint64_t wd = w0 + (uint64_t)lane;
      uint32_t word = wd <= w_end ? flat_word(bits, wd, f0, f1) : 0u;
      const uint32_t c = (uint32_t)__popc(word);
      uint32_t before = c;  // inclusive scan of the hit counts over the lanes
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, before, d);
        if (lane >= d) before += u;
      }
      const uint32_t total = __shfl_sync(0xffffffffu, before, 31);
      size_t q = o + before - c;
      while (word) {
        const uint32_t b = (uint32_t)__ffs(word) - 1u;
        word &= word - 1u;
        const uint32_t Q = A.eval[j0 + (uint32_t)((wd << 5) + b - f0)];
        const bool swap = type == CB_KEY_EE && Q < P;
        out[q++] = pair_key(A, type, (swap ? Q : P) - ibase, (swap ? P : Q) - jbase);
      }
      o += total;
    }
  }
}

// the staged keys of every entry to their place: entry i's first
// min(cnt[i], PAIR_STAGE) pairs at off[i]
__global__ void k_pairs_copy(int64_t ne, const uint32_t* __restrict__ cnt, const uint32_t* __restrict__ off,
                             const uint64_t* __restrict__ stage, uint64_t* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ne) return;
  const uint32_t c = min(cnt[i], (uint32_t)PAIR_STAGE);
  const size_t o = off[i];
  for (uint32_t k = 0; k < c; ++k) out[o + k] = stage[(size_t)k * ne + i];
}

__global__ void k_expand(int64_t nc, const uint64_t* __restrict__ ck, int bi, int bj, uint64_t* __restrict__ out) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nc) return;
  uint64_t c = ck[q];
  uint32_t type = (uint32_t)(c >> (bi + bj));
  uint32_t i = (uint32_t)((c >> bj) & ((1ull << bi) - 1ull));
  uint32_t j = (uint32_t)(c & ((1ull << bj) - 1ull));
  out[q] = cb_key(type, i, j);
}

}  // namespace

cb_status broad_phase(cb_scene* s, BroadWork& w, const double* x, const double* p, bool swept, bool sort_out,
                      DevBuf& out, int64_t* n_out, cudaStream_t st) {
  const int np = s->n_prims;
  const int M = s->count;
  if (np == 0) {
    *n_out = 0;
    return CB_OK;
  }
  Topo t{s->kind, s->n, s->T, s->E, bp<int32_t>(s->ev0), bp<int32_t>(s->ev1), bp<int32_t>(s->tv)};
  CB_TRY(buf_ensure(w.box32, sizeof(float4) * 2 * (size_t)np, st));
  CB_TRY(buf_ensure(w.box64, sizeof(double) * 6 * (size_t)np, st));
  // per-stencil activation: the static phase keeps the uninflated boxes for contact_filter
  const bool raw = !swept && !p && !sort_out && s->per_stencil();
  if (raw) CB_TRY(buf_ensure(w.box_raw, sizeof(double) * 6 * (size_t)np, st));
  CB_TRY(buf_ensure(w.bounds, sizeof(uint32_t) * BOUNDS_STRIDE * (size_t)M, st));
  CB_TRY(buf_ensure(w.grids, sizeof(Grid) * (size_t)M, st));
  CB_TRY(buf_ensure(w.cx, sizeof(double) * 4 * (size_t)M, st));
  uint32_t* bounds = bp<uint32_t>(w.bounds);
  k_bounds_init<<<cb_grid(M), CB_THREADS, 0, cb_count(st)>>>(bounds, M);
  k_boxes<<<cb_grid(np), CB_THREADS, 0, cb_count(st)>>>(t, np, x, p, bp<MemberParams>(s->mp), swept,
                                                       bp<int32_t>(s->vsc), bp<float4>(w.box32),
                                                       bp<double>(w.box64), raw ? bp<double>(w.box_raw) : nullptr,
                                                       bounds);
  k_grids<<<cb_grid(M), CB_THREADS, 0, cb_count(st)>>>(M, bounds, bp<MemberParams>(s->mp),
                                                      w.cell_factor > 0 ? (double)w.cell_factor : 1.0,
                                                      bp<Grid>(w.grids), bp<double>(w.cx));
  CB_CUDA(cudaGetLastError());
  const Grid* dgrids = bp<Grid>(w.grids);

  CB_TRY(buf_ensure(w.cell_cnt, sizeof(uint32_t) * (size_t)np + 16, st));
  CB_TRY(buf_ensure(w.cell_off, sizeof(uint32_t) * ((size_t)np + 1), st));
  CB_TRY(buf_ensure(w.scan_tmp, sizeof(uint64_t) * (size_t)(cbp::scan_tmp_elems(np + 1) + 8), st));
  k_cell_count<<<cb_grid(np), CB_THREADS, 0, cb_count(st)>>>(t, np, bp<float4>(w.box32), bp<int32_t>(s->vsc), dgrids,
                                                            bp<uint32_t>(w.cell_cnt));
  uint32_t* tot_dev = (uint32_t*)(scalars(s) + SC_COUNT0);
  cbp::exclusive_scan<uint32_t, uint32_t>(bp<uint32_t>(w.cell_cnt), bp<uint32_t>(w.cell_off), np,
                                          bp<uint32_t>(w.scan_tmp), tot_dev, st);
  CB_CUDA(cudaGetLastError());
  // the grids come back with the entry count (one wait): their sizes bound
  // the bits of the cell codes the sort has to look at
  CB_CUDA(cudaMemcpyAsync(s->hstage_host, w.grids.p, sizeof(Grid) * M, cudaMemcpyDeviceToHost, st));
  uint64_t hne;
  CB_TRY(read_scalars(s, SC_COUNT0, 1, &hne, st));
  int dmax = 1;
  for (int m = 0; m < M; ++m) {
    const Grid& g = ((const Grid*)s->hstage_host)[m];
    dmax = std::max({dmax, g.dx, g.dy, g.dz});
  }
  const int64_t ne = (uint32_t)hne;
  if (ne == 0) {
    *n_out = 0;
    return CB_OK;
  }
  for (int b = 0; b < 2; ++b) {
    CB_TRY(buf_ensure(w.ekey[b], sizeof(uint64_t) * (size_t)ne, st));
    CB_TRY(buf_ensure(w.eval[b], sizeof(uint32_t) * (size_t)ne, st));
  }
  int mbits = 0;
  while ((1 << mbits) < M) ++mbits;
  // shell cells are swept along x (type group and x level below the cell code)
  const bool sweep = s->kind == CB_SHELL;
  const int shift = sweep ? SWEEP_SHIFT : 0;
  if (30 + mbits + shift > 64) return CB_ERR_ARG;  // more members than the cell keys can number
  k_cell_fill<<<cb_grid(np), CB_THREADS, 0, cb_count(st)>>>(t, np, bp<float4>(w.box32), bp<int32_t>(s->vsc), dgrids,
                                                           bp<uint32_t>(w.cell_off), bp<uint64_t>(w.ekey[0]),
                                                           bp<uint32_t>(w.eval[0]), sweep);
  CB_TRY(buf_ensure(w.hist, sizeof(uint32_t) * (size_t)cbp::radix_hist_elems(ne), st));
  CB_TRY(buf_ensure(w.scan_tmp, sizeof(uint64_t) * (size_t)(cbp::scan_tmp_elems(cbp::radix_hist_elems(ne)) +
                                                             cbp::scan_tmp_elems(ne + 1) + 8),
                    st));
  // bits a cell key can hold: the Morton code of cell coordinates below
  // 2^cb (3 cb bits), the member index above bit 30, and for shells the type
  // group and x level below them (every key is shifted up by `shift`)
  int cb = 0;
  while ((1 << cb) < dmax) ++cb;
  const uint64_t need = ((((1ull << (3 * cb)) - 1ull) | (((1ull << mbits) - 1ull) << 30)) << shift) |
                        ((1ull << shift) - 1ull);
  int r = cbp::radix_sort<uint64_t, uint32_t, true>(bp<uint64_t>(w.ekey[0]), bp<uint32_t>(w.eval[0]),
                                                    bp<uint64_t>(w.ekey[1]), bp<uint32_t>(w.eval[1]), ne, 0,
                                                    30 + mbits + shift, bp<uint32_t>(w.hist), bp<uint32_t>(w.scan_tmp),
                                                    st, need);
  const uint64_t* ekey = bp<uint64_t>(w.ekey[r]);
  const uint32_t* eval = bp<uint32_t>(w.eval[r]);
  CB_TRY(buf_ensure(w.run_flag, sizeof(uint32_t) * (size_t)ne, st));
  CB_TRY(buf_ensure(w.run_id, sizeof(uint32_t) * (size_t)ne, st));
  CB_TRY(buf_ensure(w.run_start, sizeof(uint32_t) * ((size_t)ne + 2), st));
  CB_TRY(buf_ensure(w.pair_cnt, sizeof(uint32_t) * (size_t)ne, st));
  CB_TRY(buf_ensure(w.pair_off, sizeof(uint32_t) * ((size_t)ne + 1), st));
  k_run_flag<<<cb_grid(ne), CB_THREADS, 0, cb_count(st)>>>(ne, ekey, shift, bp<uint32_t>(w.run_flag));
  // exclusive scan of the flags into pair_off (used as scratch here)
  cbp::exclusive_scan<uint32_t, uint32_t>(bp<uint32_t>(w.run_flag), bp<uint32_t>(w.pair_off), ne,
                                          bp<uint32_t>(w.scan_tmp), (uint32_t*)nullptr, st);
  k_run_start<<<cb_grid(ne), CB_THREADS, 0, cb_count(st)>>>(ne, bp<uint32_t>(w.run_flag), bp<uint32_t>(w.pair_off),
                                                           bp<uint32_t>(w.run_id), bp<uint32_t>(w.run_start));
  PairArgs A;
  A.t = t;
  A.ne = ne;
  A.ekey = ekey;
  A.shift = shift;
  A.eval = eval;
  A.run_id = bp<uint32_t>(w.run_id);
  A.run_start = bp<uint32_t>(w.run_start);
  A.box32 = bp<float4>(w.box32);
  CB_TRY(buf_ensure(w.ebox, sizeof(float4) * 2 * (size_t)ne, st));
  k_gather_boxes<<<cb_grid(ne), CB_THREADS, 0, cb_count(st)>>>(ne, eval, bp<float4>(w.box32), bp<float4>(w.ebox));
  A.ebox = bp<float4>(w.ebox);
  A.box64 = bp<double>(w.box64);
  A.grids = dgrids;
  A.bi = s->bits_i;
  A.bj = s->bits_j;
  A.fpstat = nullptr;
  A.canonical = false;
  if (!swept) {
    A.fpstat = (unsigned long long*)(scalars(s) + SC_FP32_PAIRS);
    CB_CUDA(cudaMemsetAsync(A.fpstat, 0, 2 * sizeof(unsigned long long), st));
  }
  const int pb = w.pair_block;
  const bool rods = s->kind == CB_ROD;
  // keys are final from the count pass on: canonical straight out, compact for the sort
  A.canonical = !sort_out;
  unsigned int* novl = (unsigned int*)(scalars(s) + SC_NOVF);
  unsigned int* nvlong = (unsigned int*)(scalars(s) + SC_NVLONG);
  uint32_t* c = bp<uint32_t>(w.pair_cnt);
  uint64_t flat_t = 0;
  if (rods) {
    CB_TRY(buf_ensure(w.stage, sizeof(uint64_t) * PAIR_STAGE * (size_t)ne, st));
    CB_TRY(buf_ensure(w.ovl, sizeof(uint32_t) * (size_t)ne, st));
    CB_CUDA(cudaMemsetAsync(novl, 0, sizeof(unsigned int), st));
    k_rod_pairs<false><<<cb_grid(ne, pb), pb, 0, cb_count(st)>>>(A, c, nullptr, nullptr, bp<uint64_t>(w.stage),
                                                                bp<uint32_t>(w.ovl), novl);
  } else {
    // shells: the swept ranges laid end to end, tested evenly, counted per entry
    CB_TRY(buf_ensure(w.flat_len, sizeof(uint32_t) * ((size_t)ne + 1), st));
    CB_TRY(buf_ensure(w.flat_off, sizeof(uint64_t) * ((size_t)ne + 1), st));
    CB_TRY(buf_ensure(w.flat_j0, sizeof(uint32_t) * (size_t)ne, st));
    CB_TRY(buf_ensure(w.flat_slen, (size_t)ne, st));
    CB_TRY(buf_ensure(w.flat_sbits, sizeof(uint32_t) * (size_t)ne, st));
    CB_TRY(buf_ensure(w.flat_lflag, sizeof(uint32_t) * ((size_t)ne + 1), st));
    CB_TRY(buf_ensure(w.flat_lpos, sizeof(uint32_t) * ((size_t)ne + 1), st));
    CB_TRY(buf_ensure(w.flat_lidx, sizeof(uint32_t) * (size_t)ne, st));
    CB_TRY(buf_ensure(w.flat_llen, sizeof(uint32_t) * ((size_t)ne + 1), st));
    k_flat_ranges<<<cb_grid(ne + 1), CB_THREADS, 0, cb_count(st)>>>(A, bp<uint32_t>(w.flat_len),
                                                                    bp<uint32_t>(w.flat_lflag), bp<uint8_t>(w.flat_slen),
                                                                    bp<uint32_t>(w.flat_j0));
    k_pairs_short<<<cb_grid(ne, 256), 256, 0, cb_count(st)>>>(A, bp<uint8_t>(w.flat_slen), bp<uint32_t>(w.flat_j0),
                                                             bp<uint32_t>(w.flat_sbits));
    // the long entries in entry order, their ranges laid end to end
    cbp::exclusive_scan<uint32_t, uint32_t>(bp<uint32_t>(w.flat_lflag), bp<uint32_t>(w.flat_lpos), ne + 1,
                                            bp<uint32_t>(w.scan_tmp), (uint32_t*)nullptr, st);
    CB_CUDA(cudaMemsetAsync(w.flat_llen.p, 0, sizeof(uint32_t) * ((size_t)ne + 1), st));
    k_flat_compact<<<cb_grid(ne), CB_THREADS, 0, cb_count(st)>>>(ne, bp<uint32_t>(w.flat_lflag),
                                                                bp<uint32_t>(w.flat_lpos), bp<uint32_t>(w.flat_len),
                                                                bp<uint32_t>(w.flat_lidx), bp<uint32_t>(w.flat_llen));
    cbp::exclusive_scan<uint32_t, uint64_t>(bp<uint32_t>(w.flat_llen), bp<uint64_t>(w.flat_off), ne + 1,
                                            bp<uint64_t>(w.scan_tmp), scalars(s) + SC_COUNT0, st);
    CB_CUDA(cudaGetLastError());
    CB_TRY(read_scalars(s, SC_COUNT0, 1, &flat_t, st));
    CB_TRY(buf_ensure(w.flat_bits, sizeof(uint32_t) * (size_t)std::max<uint64_t>(1, (flat_t + 31) / 32), st));
    if (flat_t > 0) {
      const int64_t chunks = (int64_t)((flat_t + 32ull * FLAT_STEPS - 1) / (32ull * FLAT_STEPS));
      const int64_t g = std::min<int64_t>((chunks + FLAT_WARPS - 1) / FLAT_WARPS, (int64_t)s->n_sms * 8);
      k_pairs_flat<<<(int)g, 32 * FLAT_WARPS, 0, cb_count(st)>>>(A, bp<uint64_t>(w.flat_off), bp<uint32_t>(w.flat_lidx),
                                                    bp<uint32_t>(w.flat_j0), flat_t, bp<uint32_t>(w.flat_bits));
    }
    CB_TRY(buf_ensure(w.flat_vlong, sizeof(uint32_t) * (size_t)ne, st));
    CB_CUDA(cudaMemsetAsync(nvlong, 0, sizeof(unsigned int), st));
    k_flat_count<<<cb_grid(ne), CB_THREADS, 0, cb_count(st)>>>(ne, bp<uint64_t>(w.flat_off), bp<uint32_t>(w.flat_lflag),
                                                              bp<uint32_t>(w.flat_lpos), bp<uint32_t>(w.flat_bits),
                                                              bp<uint32_t>(w.flat_sbits), c,
                                                              bp<uint32_t>(w.flat_vlong), nvlong);
  }
  // the fill: rods move their staged keys and re-test the entries with more;
  // shells write the pairs of their hit bits
  auto pairs = [&](uint64_t* o) -> cb_status {
    const uint32_t* f = bp<uint32_t>(w.pair_off);
    if (rods) {
      uint64_t* sg = bp<uint64_t>(w.stage);
      k_pairs_copy<<<cb_grid(ne), CB_THREADS, 0, cb_count(st)>>>(ne, c, f, sg, o);
      const int g = (int)std::min<int64_t>(cb_grid(ne, pb), (int64_t)s->n_sms * 8);
      k_rod_pairs<true><<<g, pb, 0, cb_count(st)>>>(A, c, f, o, sg, bp<uint32_t>(w.ovl), novl);
    } else {
      k_flat_emit<<<cb_grid(ne), CB_THREADS, 0, cb_count(st)>>>(A, bp<uint64_t>(w.flat_off), bp<uint32_t>(w.flat_lflag),
                                                               bp<uint32_t>(w.flat_lpos), bp<uint32_t>(w.flat_j0),
                                                               bp<uint32_t>(w.flat_bits), bp<uint32_t>(w.flat_sbits),
                                                               c, f, o);
      if (flat_t > 0) {
        const int g = (int)std::min<int64_t>(cb_grid(ne, 256), (int64_t)s->n_sms * 16);
        k_flat_emit_long<<<g, 256, 0, cb_count(st)>>>(A, bp<uint64_t>(w.flat_off), bp<uint32_t>(w.flat_lidx),
                                                      bp<uint32_t>(w.flat_vlong), nvlong, bp<uint32_t>(w.flat_j0),
                                                      bp<uint32_t>(w.flat_bits), bp<uint32_t>(w.flat_sbits), f, o);
      }
    }
    return CB_OK;
  };
  cbp::exclusive_scan<uint32_t, uint32_t>(c, bp<uint32_t>(w.pair_off), ne, bp<uint32_t>(w.scan_tmp), tot_dev, st);
  CB_CUDA(cudaGetLastError());
  uint64_t hnc;
  CB_TRY(read_scalars(s, SC_COUNT0, 1, &hnc, st));
  const int64_t nc = (uint32_t)hnc;
  *n_out = nc;
  if (nc == 0) return CB_OK;
  if (!sort_out) {
    // canonical keys straight from the fill pass, in hash-cell order
    CB_TRY(buf_ensure(out, sizeof(uint64_t) * (size_t)nc, st));
    CB_TRY(pairs(bp<uint64_t>(out)));
    CB_CUDA(cudaGetLastError());
    return CB_OK;
  }
  for (int b = 0; b < 2; ++b) CB_TRY(buf_ensure(w.ckey[b], sizeof(uint64_t) * (size_t)nc, st));
  CB_TRY(pairs(bp<uint64_t>(w.ckey[0])));
  const int cbits = s->bits_i + s->bits_j + (s->kind == CB_SHELL ? 2 : 0);
  CB_TRY(buf_ensure(w.hist, sizeof(uint32_t) * (size_t)cbp::radix_hist_elems(nc), st));
  CB_TRY(buf_ensure(w.scan_tmp, sizeof(uint64_t) * (size_t)(cbp::scan_tmp_elems(cbp::radix_hist_elems(nc)) + 8),
                    st));
  int r2 = cbp::radix_sort<uint64_t, uint32_t, false>(bp<uint64_t>(w.ckey[0]), nullptr, bp<uint64_t>(w.ckey[1]),
                                                      nullptr, nc, 0, cbits, bp<uint32_t>(w.hist),
                                                      bp<uint32_t>(w.scan_tmp), st);
  CB_TRY(buf_ensure(out, sizeof(uint64_t) * (size_t)nc, st));
  k_expand<<<cb_grid(nc), CB_THREADS, 0, cb_count(st)>>>(nc, bp<uint64_t>(w.ckey[r2]), s->bits_i, s->bits_j,
                                                        bp<uint64_t>(out));
  CB_CUDA(cudaGetLastError());
  return CB_OK;
}
