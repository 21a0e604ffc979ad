// scene.cuh -- internal scene object and the launchers each stage file provides.
#pragma once
#include <vector>

#include "common.cuh"

// A device buffer remembers the allocator that made it (NULL: the library's
// own stream-ordered pool) and the byte counter of the scene it is charged to.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  const cb_allocator* alloc = nullptr;
  int64_t* charged = nullptr;
};

// Where the buffers of the current API call come from: set for the duration
// of each call that may allocate (AllocScope), read by buf_ensure.
struct AllocCtx {
  const cb_allocator* alloc = nullptr;
  int64_t* charged = nullptr;
};
AllocCtx& alloc_ctx();
struct AllocScope {
  AllocCtx saved;
  AllocScope(const cb_allocator* a, int64_t* charged) : saved(alloc_ctx()) {
    alloc_ctx().alloc = a;
    alloc_ctx().charged = charged;
  }
  ~AllocScope() { alloc_ctx() = saved; }
};

// A growable device buffer: keeps its allocation, grows by 25 % headroom.
// Allocates through the current AllocScope's allocator (or the library's
// pool) and charges the scope's counter; frees through the buffer's own
// allocator (after the stream's work is done, since a caller's allocator may
// hand the memory out again at once).
cb_status buf_ensure(DevBuf& b, size_t bytes, cudaStream_t st);
void buf_free(DevBuf& b, cudaStream_t st);

// A device buffer local to one call, released on every way out of its scope
// (error returns included).
struct ScopedBuf {
  DevBuf b;
  cudaStream_t st;
  explicit ScopedBuf(cudaStream_t s) : st(s) {}
  ~ScopedBuf() { buf_free(b, st); }
  ScopedBuf(const ScopedBuf&) = delete;
  ScopedBuf& operator=(const ScopedBuf&) = delete;
};
template <typename T>
static inline T* bp(const DevBuf& b) {
  return (T*)b.p;
}

// Per-member parameters.  A plain scene has one member; a batch (several
// scenes merged into one index space, cb_batch_create) has one per scene.
struct MemberParams {
  double xi, dhat, a, kappa;
  double dbar_min;        // 0 when nothing is filtered
  int32_t single, core_temp, filter_off, n_prims;
  // FP32 copies rounded up, for the screens' rigorous FP32 comparisons (set
  // at upload): a (1 + 1e-9) + 1e-9, dbar_min (1 + 1e-9) + 1e-9,
  // xi (1 + 1e-9) + 1e-9, xi
  float thrU32, thrF32, thrC32, xi32;
  int32_t cull_radius;    // CB_FILTER_KALDOR: rod edge pairs of one polyline this close are culled; else 0
  int32_t per_comp;       // CB_DBAR_PER_COMPONENT: class-F width from dbar_comp by component label
  double dbar_fmax;       // largest class-F width of the member (= dbar_min unless per_comp)
  int32_t loops;          // rods: the member has closed loops (backward arc-length windows to test)
  int32_t mollify;        // CB_EE_MOLLIFIER: edge-edge pairs take IPC's mollifier
  int32_t per_stencil;    // CB_PER_STENCIL: class-F candidates outside their own width are dropped
};

// Spatial-hash grid of one member.
struct Grid {
  float ox, oy, oz, inv;
  int dx, dy, dz, pad;
};

// Workspace of one broad phase (static or swept) -- reused between calls.
struct BroadWork {
  float cell_factor = 1.0f;  // hash cell edge = factor x mean primitive box extent (tuning knob)
  int pair_block = CB_THREADS;  // threads per block of the pair enumeration (tuning knob)
  DevBuf box32;       // float4 lo, float4 hi per primitive
  DevBuf box64;       // double lo[3], hi[3] per primitive
  DevBuf box_raw;     // per-stencil activation (static phase): double lo[3], hi[3] per primitive, not inflated
  DevBuf bounds;      // per member: 6 x uint32 ordered-float min/max, 2 pad, double extent sum
  DevBuf grids;       // Grid per member
  DevBuf cx;          // per member: double centre[3], X (max |coordinate - centre|)
  DevBuf cell_cnt;    // uint32 per primitive
  DevBuf cell_off;    // uint32 per primitive (+1)
  DevBuf ekey[2];     // uint64 (member << 30 | Morton cell) per entry (ping-pong); shells: shifted up by
                      // 12 bits above the entry's type group and x level in the cell
  DevBuf eval[2];     // uint32 primitive per entry
  DevBuf run_flag;    // uint32 per entry
  DevBuf run_id;      // uint32 per entry
  DevBuf run_start;   // uint32 per run (+1)
  DevBuf pair_cnt;    // uint32 per entry
  DevBuf pair_off;    // uint32 per entry (+1)
  DevBuf ebox;        // float4 lo, float4 hi per entry (boxes gathered into entry order)
  DevBuf ckey[2];     // uint64 compact candidate keys (ping-pong)
  DevBuf stage;       // uint64 [PAIR_STAGE][entries]: the count pass's first pairs of each entry
  DevBuf ovl;         // uint32 entries with more pairs than the stage holds
  DevBuf flat_len;    // shells: uint32 per entry, the length of a long swept partner range
  DevBuf flat_lflag;  // shells: uint32 per entry (+1), 1 for a long range
  DevBuf flat_lpos;   // shells: uint32 per entry (+1), its place among the long entries (scan of flat_lflag)
  DevBuf flat_lidx;   // shells: uint32 per long entry, the entry
  DevBuf flat_llen;   // shells: uint32 per long entry (+1), its range length
  DevBuf flat_vlong;  // shells: uint32, the long entries with ranges of FLAT_EMIT_WARP slots or more (any order)
  DevBuf flat_off;    // shells: uint64 per long entry (+1), its first test slot (scan of flat_llen)
  DevBuf flat_j0;     // shells: uint32 per entry, its first partner
  DevBuf flat_bits;   // shells: one hit bit per test slot
  DevBuf flat_slen;   // shells: uint8 per entry, the length of a short range (tested per entry)
  DevBuf flat_sbits;  // shells: uint32 per entry, the hits of a short range
  DevBuf scan_tmp;
  DevBuf hist;
};

struct cb_scene {
  // the caller's allocator (copied at create; has_alloc false: the library's pool)
  // and the bytes of device memory the scene holds now
  cb_allocator allocator{};
  bool has_alloc = false;
  int64_t live_bytes = 0;
  const cb_allocator* alloc_ptr() const { return has_alloc ? &allocator : nullptr; }
  int kind = 0;
  int n = 0, E = 0, T = 0, n_rods = 0;
  int n_prims = 0;     // broad-phase primitives
  int bits_i = 0, bits_j = 0;
  double xi = 0, dhat = 0, a = 0, kappa = 1;   // member 0 (plain scenes: the scene)
  int filter = CB_FILTER_DOUBLE;
  int core_temp = 1;
  double dbar_min = 0;  // +inf when nothing is filtered
  // members (1 for a plain scene)
  int count = 1;
  std::vector<MemberParams> hmp;
  DevBuf mp;            // MemberParams [count]
  DevBuf vsc;           // int32 [n] member of each vertex
  std::vector<int64_t> voff, eoff, toff;  // member offsets of vertices, edges, triangles (count+1)
  int64_t n_frest_pt = 0;                 // shells: point-triangle keys at the head of frest
  DevBuf macc;          // per member: double energy, u64 alpha bits, u64 lb bits, u64 status, double lo, hi
  void* hstage_host = nullptr;  // pinned staging (the largest per-member record x members + 256)
  cudaStream_t last_stream = nullptr;
  int device = 0;
  int n_sms = 152;      // multiprocessors of the device (caps of grid-stride launches: a few blocks per SM)
  int proj_occ[2] = {0, 0};  // resident blocks per SM of k_hess_proj<9> and <6> (0: not looked up yet)

  // topology on device
  DevBuf ev0, ev1;      // int32 [E]
  DevBuf tv;            // int32 [3][T]
  DevBuf comp;          // int32 [n]
  DevBuf rest;          // double [3][n]
  DevBuf rod_ptr;       // int32 [n_rods+1] (rods)
  // filter tables
  DevBuf S;             // double [n] rods: arc length
  DevBuf win;           // int32 [E] rods: last filtered partner edge
  DevBuf wst;           // int32 [E] rods: first partner edge of the backward window on a closed loop (-1: none)
  DevBuf rloop;         // int32 [E] rods: edge count of the edge's closed loop (0: open polyline)
  DevBuf rlast;         // int32 [E] rods: last (closing) edge of the edge's closed loop (-1: open)
  DevBuf elen2;         // double [E] squared rest length of each edge (the mollifier's threshold)
  DevBuf ruv;           // double [3][n] shells: the flat pattern (u, v, 0), when given; reference distances there
  bool geodesic = false;  // shells, CB_DBAR_GEODESIC: reference distances are geodesic distances on the rest mesh
  // ... its mesh adjacency, host copies kept until the rest filter has run: edge of (t_k, t_k+1) [T][3],
  // faces of an edge [E][2] (-1: none), faces around a vertex (CSR [n+1], [3T])
  std::vector<int32_t> geo_te, geo_ef, geo_vfp, geo_vf;
  DevBuf frest;         // uint64 shells: sorted rest-filtered keys
  DevBuf frest_dbar;    // double
  DevBuf frest_j;       // uint32 shells: the partner index j of each frest key (the rows' search keys)
  DevBuf dbar_comp;     // uint64 bits of the per-component dbar_min, by component label (n entries)
  double dbar_fmax = 0.0;  // largest per-component dbar_min (finite), or dbar_min
  int64_t n_frest = 0;
  DevBuf frow_pt;       // uint32 shells: row offsets of frest by vertex (point-triangle keys), n + 1
  DevBuf frow_ee;       // uint32 shells: row offsets of frest by edge (edge-edge keys), E + 1

  // pass state
  BroadWork bw;         // static broad phase
  BroadWork bwc;        // swept broad phase (CCD)
  DevBuf cand;          // uint64 [nc] sorted candidate keys
  int64_t n_cand = 0;
  DevBuf klass;         // uint8 [nc]
  DevBuf cand_alt, klass_alt;  // per-stencil activation: the compacted candidates before the swap
  int64_t n_dropped = 0;       // last contact_filter: class-F candidates outside their own width
  bool per_stencil() const {
    for (const MemberParams& m : hmp)
      if (m.per_stencil) return true;
    return false;
  }
  DevBuf cd;            // double [nc] distance
  DevBuf cflag;         // uint32 [nc] active flag
  DevBuf cpos;          // uint32 [nc+1] scan of flags
  DevBuf ctype;         // int8 [nc]
  DevBuf ccls;          // uint8 [nc] final class (with C)
  int64_t n_active = 0;
  DevBuf aidx;          // uint32 [na] candidate index of each active pair
  DevBuf bkey[2];       // uint64 [16 na]
  DevBuf bflag, bpos;   // uint32
  DevBuf bsr_row;       // int32 [n+1]
  DevBuf bsr_col;       // int32 [nnzb]
  DevBuf bsr_val;       // double [nnzb][9]
  DevBuf row_cnt;       // uint32 [n+1]
  int64_t nnzb = 0;
  DevBuf horder;        // uint32 active pair indices in prep order (face / line-line pairs first)
  DevBuf hmoll;         // uint8 [na] mollified edge-edge pair (CB_EE_MOLLIFIER), handled by k_moll_hess
  DevBuf mlist;         // uint32 active indices of the mollified pairs
  DevBuf hB9, hB6, hB4;  // queued reduced Hessians (packed, element-major); hB4: point-edge in its own frame
  DevBuf hslot;          // uint32 [2][na] active index of each queued matrix
  DevBuf xf, pf;         // float [3][n]: centred FP32 copies of x and of p
  DevBuf dlist;          // uint32: candidates / CCD pairs queued for the FP64 phase
  DevBuf ccd_keys;      // uint64 [nccd]
  DevBuf ccd_t;         // double [nccd]
  DevBuf ccd_cls;       // uint8 [nccd] class | 0x80 when t is exact
  DevBuf ccd_lb;        // double [nccd] lower bound of t (2 when resolved)
  DevBuf ccd_flag, ccd_pos, ccd_list;  // band selection: u64 kind counts (flag, scan), uint32 list
  DevBuf ccd_ulist;     // uint32 pairs still unresolved after the first-step pass
  int64_t n_ccd = 0;
  // lagged friction (friction_lag / friction_eval / friction_spmv)
  DevBuf fr_key;        // uint64 [nf] keys of the lagged pairs
  DevBuf fr_st;         // int4 [nf] their stencil vertices
  DevBuf fr_dat;        // double [8][nf]: lambda, beta[4], n[3] (element-major)
  DevBuf fr_hw;         // double [6][nf]: packed tangent Hessian (xx xy xz yy yz zz) of the last friction_eval
  int64_t n_fric = 0;
  double fr_mu = 0.0, fr_eps = 0.0;
  bool fr_lagged = false, fr_hw_valid = false;
  DevBuf scan_tmp;
  DevBuf hist;
  DevBuf dev_scalars;   // misc device scalars (counters, energy, alpha bits, status)

  uint64_t* h_pinned = nullptr;  // pinned host scratch (64 slots)
  int32_t status_host = 0;

  bool timing = false;
  // stage events: [2k, 2k+1] around stage k of cb_get_stage_ms, [10, 11] around
  // the Hessian kernels, [12] the end of stage (c) inside barrier_eval (the
  // active count known); cd_split: the last barrier_eval recorded [12]
  cudaEvent_t ev[13] = {};
  bool cd_split = false;
  float stage_ms[5] = {0, 0, 0, 0, 0};
  int64_t counts_filtered = 0, counts_core = 0;
  int ccd_max_iters = 0;
};

// device scalar slots (uint64 each) inside dev_scalars
enum {
  SC_COUNT0 = 0,
  SC_COUNT1 = 1,
  SC_STATUS = 2,
  SC_ENERGY = 3,
  SC_ALPHA_BITS = 4,
  SC_DBAR_MIN_BITS = 5,
  SC_ITERS = 6,
  SC_NFILT = 7,
  SC_NCORE = 8,
  SC_N9 = 9,
  SC_N6 = 10,
  SC_NLIST = 11,        // two uint32 counters: point-triangle and edge-edge pairs for the exact distance
  SC_N4 = 14,           // point-edge pairs queued in their own frame
  SC_NU = 15,           // CCD pairs left unresolved by the first step
  SC_FP32_PAIRS = 12,   // broad phase of contact_build: pairs passing the FP32 box test
  SC_FP64_DECIDED = 13, // ... of which the FP64 boxes decided
  SC_KSPLIT = 16,       // two uint32 counters: face / line-line pairs, the other active pairs
  SC_NOVF = 17,         // broad phase: entries whose pairs overflow the stage
  SC_NBK = 18,          // BSR pattern: keys left after the per-run sets of k_block_keys
  SC_FETCH = 19,        // ccd_step, exact rounds: pairs of the list handed out so far
  SC_NMOLL = 20,        // barrier_eval: mollified edge-edge pairs
  SC_GEO_COUNT = 21,    // geodesic rest filter: (edge, vertex) entries below the activation
  SC_GEO_ERR = 22,      // ... error bits of its sources (a fixed capacity exceeded)
  SC_NVLONG = 23,       // shell broad phase: entries of flat_vlong
  SC_N = 24
};
// read_scalars stages up to SC_N scalars through the pinned host scratch
static_assert(SC_N <= 64, "the scalars must fit the pinned scratch");

static inline uint64_t* scalars(cb_scene* s) { return (uint64_t*)s->dev_scalars.p; }

// per-member accumulator slots (uint64 / double each) inside macc
enum { MACC_E = 0, MACC_ALPHA = 1, MACC_LB = 2, MACC_STATUS = 3, MACC_LO = 4, MACC_HI = 5, MACC_STRIDE = 6 };

// read n uint64 device scalars into host (sync on stream)
cb_status read_scalars(cb_scene* s, int first, int count, uint64_t* out, cudaStream_t st);

// broad.cu
// Candidate pairs of x (p == nullptr) or of the sweep x -> x + p.  Boxes are
// inflated per member by a/2 (static) or xi/2 (swept = true).  Writes the
// canonical keys into *out (grown as needed), in ascending order when
// sort_out is set and otherwise in hash-cell order, and their count into
// *n_out.
cb_status broad_phase(cb_scene* s, BroadWork& w, const double* x, const double* p, bool swept, bool sort_out,
                      DevBuf& out, int64_t* n_out, cudaStream_t st);

// narrow.cu
cb_status filter_precompute(cb_scene* s, cudaStream_t st);
// geodesic.cu: the rest filter's flag / dbar / minima of the rest-broad-phase
// candidates with geodesic reference distances (CB_DBAR_GEODESIC)
cb_status geo_rest_dbar(cb_scene* s, const uint64_t* cand, int64_t nc, uint32_t* flag, double* dbar,
                        unsigned long long* dmin, unsigned long long* dcomp, cudaStream_t st);
cb_status filter_apply(cb_scene* s, cudaStream_t st);
cb_status frest_rows_build(cb_scene* s, cudaStream_t st);
// energy_only: distances and energy (no active list, gradient, Hessian or BSR)
cb_status barrier_run(cb_scene* s, const double* x, double* energy, double* grad, bool energy_only,
                      cudaStream_t st);

// ccd.cu
cb_status ccd_run(cb_scene* s, const double* x, const double* p, double* alpha, cudaStream_t st);

// narrow.cu: FP32 copy of (v - centre of the vertex's member) (cx null: no centring)
cb_status to_f32(cb_scene* s, const double* v, const double* cx, DevBuf& out, cudaStream_t st);
