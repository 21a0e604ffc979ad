/*
 * contact.h -- C ABI of the GB300 barrier-filtered contact library.
 *
 * One contact pass of a projected-Newton iteration for thickened rods (yarn
 * polylines) and shells (triangle meshes) under the IPC log barrier with
 * thickness offsets, filtered against contact locking as in
 * "Unlocking Thickness Modeling for Codimensional Contact Simulation":
 *
 *   contact_build   (a) broad phase at the full, unmodified activation  Sec. 3.3
 *   contact_filter  (b) filtered / unfiltered class of every candidate  Sec. 3.2, Eq. 1/4
 *   barrier_eval    (c) exact point-triangle / edge-edge distances,
 *                   (d) barrier energy, gradient and PSD-projected 12x12
 *                       Hessians assembled into a global gradient and a
 *                       3x3-block BSR matrix                             Eq. 2-4
 *   ccd_step        (e) conservative additive-CCD step bound with per-class
 *                       offsets                                          Sec. 3.3
 *
 * Conventions
 *   Units: millimetres.  Positions are FP64 structure-of-arrays [3][n]: all x,
 *   then all y, then all z.  Every pass buffer lives on the GPU of the scene.
 *   stream: a cudaStream_t passed as void* (NULL = legacy default stream).
 *   Calls are asynchronous on the stream unless marked "sync"; they may block
 *   briefly to read counts the next kernel launch needs.  A scene is not
 *   thread-safe: one caller, one stream at a time.
 *   Errors: argument / allocation / CUDA errors return immediately.  Device-side
 *   conditions (capacity overflow, CCD iteration limit, penetration) are
 *   recorded in the scene's status word and returned by cb_sync_status().
 *
 * Pair keys (uint64): bits 63..62 type, 61..31 index i, 30..0 index j.
 *   type 0 rod edge-edge     i < j edge ids
 *   type 1 shell point-tri   i = vertex id, j = triangle id
 *   type 2 shell edge-edge   i < j edge ids
 * Edge ids: rods -- edges (v, v+1) of each polyline in order (a closed loop's
 * closing edge (last, first) after them); shells -- the
 * unique (min, max) vertex pairs of the triangles in lexicographic order.
 * Pair lists are returned sorted by key.
 */
#ifndef CONTACT_H
#define CONTACT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CB_OK = 0,
  CB_ERR_ARG = 1,          /* invalid argument (null pointer, bad size, bad mode) */
  CB_ERR_OOM = 2,          /* device allocation failed */
  CB_ERR_CAPACITY = 3,     /* a fixed-capacity buffer overflowed; results incomplete */
  CB_ERR_PENETRATION = 4,  /* a pair is at or inside its barrier offset: energy = +inf */
  CB_ERR_DEGENERATE = 5,   /* zero reference distance between stencil primitives */
  CB_ERR_ITER_LIMIT = 6,   /* additive CCD hit its iteration cap: alpha is the last safe t */
  CB_ERR_CUDA = 7,         /* CUDA runtime error */
  CB_ERR_TOO_LARGE = 8     /* input larger than a call's fixed maximum; nothing was run */
} cb_status;

#define CB_ROD 0
#define CB_SHELL 1

/* mode flags */
#define CB_FILTER_DOUBLE 0          /* Eq. 4: filtered pairs use (offset 0, width dbar_min) */
#define CB_FILTER_SINGLE 1          /* Eq. 1: single-phase barrier, no offset */
#define CB_FILTER_OFF 2             /* control: no filtering (plain thickness barrier) */
#define CB_FILTER_KALDOR 3          /* comparison: no filtering, and rod edge pairs of one polyline at
                                       most cull_radius edges apart culled (Kaldor et al.'s culling, the
                                       paper's knot-test comparison): no barrier, no CCD constraint.
                                       Rods only. */
#define CB_FILTER_MASK 3
#define CB_THICK_PAPER_LITERAL 4    /* activation a = thickness, offset = thickness - dhat */
#define CB_NO_CORE_TEMP 8           /* disable the temporary zero offset of Sec. 3.4 */
#define CB_DBAR_PER_COMPONENT 16    /* a filtered pair's width is the dbar_min of its own component (the
                                       smallest reference distance of that component's filtered pairs)
                                       instead of the scene's */
#define CB_PER_STENCIL 64           /* per-stencil activation (Sec. 3.3 leaves it for later; the paper's
                                       hash uses the full activation): after the filter, a class-F
                                       candidate stays a candidate only if its two primitives' FP64 boxes,
                                       each inflated by half the pair's own width (dbar_min, or its
                                       component's), overlap (closed intervals).  A dropped pair is farther
                                       apart than its width, so no barrier value changes; the candidate set
                                       shrinks.  The CCD candidates are unaffected. */
#define CB_DBAR_GEODESIC 128        /* shells whose rest shape is not cut from a flat pattern (doubly curved):
                                       the reference distance of a stencil pair (Sec. 3.2's rest-domain
                                       distance; the paper leaves non-flat rest shapes to future work) is
                                       the shortest-path distance between its two primitives on the
                                       polyhedral rest mesh -- exact up to rounding, for distances below the
                                       activation a (only those decide the filter).  On a flat convex
                                       sheet, or a sheet isometric to a convex pattern, it equals the
                                       pattern distance.  Shells only, not with rest_uv, and the mesh must
                                       be a manifold (at most two faces per edge): else CB_ERR_ARG.  Each
                                       vertex's geodesic ball of radius a must hold at most 192 vertices
                                       and 384 edges, and each straight strip at most 64 open branches:
                                       else cb_scene_create returns CB_ERR_TOO_LARGE. */
#define CB_EE_MOLLIFIER 32          /* IPC's edge-edge mollifier (App. A: the paper's solver uses IPC's
                                       contact energy): an edge-edge pair's energy is m(c) kappa b with
                                       c = |e0 x e1|^2, m = -c^2/eps_x^2 + 2c/eps_x below eps_x =
                                       1e-3 |rest e0|^2 |rest e1|^2 and 1 above; derivatives by the
                                       product rule, projected with the pair's 9x9 matrix */

/* pair lists for cb_get_pairs */
#define CB_PAIRS_CANDIDATE 0        /* C: broad-phase candidates */
#define CB_PAIRS_FILTERED 1         /* candidates of class F */
#define CB_PAIRS_CORE 2             /* candidates of class C (within the offset) */
#define CB_PAIRS_ACTIVE 3           /* pairs with a non-zero barrier */
#define CB_PAIRS_CCD 4              /* CCD candidates (swept boxes) */
#define CB_PAIRS_REST_FILTERED 5    /* shells: every filtered stencil pair of the rest mesh */

typedef struct cb_scene cb_scene;

/* Device memory of a scene or batch: by default the library allocates from
 * the CUDA runtime's stream-ordered pool.  A caller that accounts for device
 * memory itself (a framework with its own caching allocator, a server that
 * admits work under a memory budget) passes an allocator instead; every
 * device buffer the scene ever holds then comes from it and goes back to it:
 *   alloc(bytes, stream, ctx) -> a DEVICE pointer of the scene's GPU, 256-byte
 *     aligned, or NULL (the call fails with CB_ERR_OOM);
 *   free(ptr, bytes, stream, ctx) -- called once the work queued on `stream`
 *     has finished (the library synchronizes the stream first), so the memory
 *     may be handed out again at once.
 * `stream` is the cudaStream_t (as void*) of the call that grows or releases
 * the buffer.  Both are called from the thread that makes the library call.
 * cb_stats.device_bytes is the total the scene holds at any moment. */
typedef struct {
  void* (*alloc)(size_t bytes, void* stream, void* ctx);
  void (*free)(void* ptr, size_t bytes, void* stream, void* ctx);
  void* ctx;
} cb_allocator;

/* Scene description.  All pointers are HOST memory, read only during
 * cb_scene_create (the library copies what it needs). */
typedef struct {
  int32_t kind;               /* CB_ROD or CB_SHELL */
  int32_t n_verts;            /* n >= 1 */
  const double* rest_xyz;     /* [3][n] reference (undeformed) positions */
  int32_t n_rods;             /* rods: number of open polylines */
  const int32_t* rod_ptr;     /* rods: [n_rods+1], polyline r = vertices [rod_ptr[r], rod_ptr[r+1]) */
  int32_t n_tris;             /* shells: T */
  const int32_t* tris;        /* shells: [3][T] vertex ids */
  double thickness;           /* offset xi (eta in the paper); rods: 2 x radius */
  double dhat;                /* barrier width; full activation a = thickness + dhat */
  double kappa;               /* barrier stiffness (energy scale); 1 if <= 0 */
  int32_t mode;               /* CB_FILTER_* | CB_THICK_PAPER_LITERAL | CB_NO_CORE_TEMP | CB_DBAR_PER_COMPONENT
                                 | CB_EE_MOLLIFIER | CB_PER_STENCIL | CB_DBAR_GEODESIC */
  int32_t cull_radius;        /* CB_FILTER_KALDOR: culling radius in edges (>= 1); else ignored */
  const uint8_t* rod_closed;  /* rods, HOST [n_rods] or NULL: 1 = closed loop (an edge from the last vertex
                                 back to the first, numbered after the polyline's others; >= 3 vertices,
                                 else CB_ERR_ARG).  Its reference distances take the shorter way round the
                                 loop, Kaldor gaps too.  NULL: every polyline open. */
  const double* rest_uv;      /* shells, HOST [2][n] or NULL: the flat pattern the shell is cut from.
                                 Reference distances (Sec. 3.2: the 2D rest-domain distance) are taken in
                                 the pattern -- the geodesic distance of a developable rest shape -- while
                                 rest_xyz keeps the 3D rest shape.  Non-NULL for rods: CB_ERR_ARG. */
} cb_scene_desc;

typedef struct {
  int64_t n_candidates;       /* |C| */
  int64_t n_filtered;         /* candidates of class F */
  int64_t n_core;             /* candidates of class C */
  int64_t n_active;
  int64_t n_ccd;              /* |C_ccd| */
  int64_t nnzb;               /* BSR blocks */
  int64_t n_rest_filtered;    /* shells: filtered stencil pairs of the rest mesh */
  double dbar_min;            /* min reference distance over locking stencils (+inf if none) */
  double offset, dhat, activation;   /* effective xi, dhat, a after the mode mapping */
  int32_t status_bits;        /* device status word: 1 capacity, 2 penetration, 4 iteration limit */
  int32_t ccd_max_iters;
  int64_t device_bytes;       /* device memory held by the scene */
  int64_t n_candidates_fp32;  /* last contact_build: non-incident pairs passing the FP32 box test
                                 (a superset of the candidates; the FP32 effect on |C| is this / n_candidates) */
  int64_t n_fp64_decided;     /* ... of which the FP32 test was not conclusive and the FP64 boxes decided */
  int64_t n_hess_face;        /* last barrier_eval: active face / line-line pairs (9x9 projection) */
  int64_t n_hess_pe_frame;    /* ... point-edge pairs projected in their own frame (3x3 + 2x2) */
  int64_t n_hess_pe;          /* ... point-edge pairs on the generic 6x6 projection */
  int64_t n_pair_overflow;    /* last broad phase of a rod scene (ccd_step's, once a pass ran it): entries
                                 with more pairs than the 32 keys the count pass stages, re-tested by the fill
                                 pass (shell scenes keep one hit bit per test and never re-test: 0) */
  int64_t n_mollified;        /* last barrier_eval with CB_EE_MOLLIFIER: edge-edge pairs below their threshold */
  int64_t n_stencil_dropped;  /* last contact_filter with CB_PER_STENCIL: filtered broad-phase pairs outside
                                 their own width, removed from the candidates */
} cb_stats;

/* Create a scene: uploads topology and rest positions, derives edges and
 * components, and precomputes the filter tables of Sec. 3.2 on the GPU
 * (rods: arc-length windows; shells: every stencil pair of the rest mesh
 * closer than the activation) and dbar_min.  allocator: NULL (the library's
 * pool) or the caller's (copied; its ctx must outlive the scene).  sync.
 * Errors: CB_ERR_ARG (bad sizes / indices, an allocator without alloc or
 * free), CB_ERR_DEGENERATE (zero reference distance), CB_ERR_OOM,
 * CB_ERR_CUDA.  *out is set only on CB_OK. */
cb_status cb_scene_create(const cb_scene_desc* desc, const cb_allocator* allocator, void* stream, cb_scene** out);

/* Release every device buffer of the scene.  sync on the scene's last stream. */
cb_status cb_scene_destroy(cb_scene* scene);

/* (a) Broad phase, Sec. 3.3: every non-incident primitive pair (shells:
 * point-triangle and edge-edge; rods: edge-edge) whose FP64 bounding boxes of
 * x, each inflated by a/2, overlap (closed intervals).  Runs an FP32 spatial
 * hash with outward-rounded boxes (a provable superset) and decides ambiguous
 * pairs in FP64.  x_dev: DEVICE [3][n] FP64, read during the call's kernels.
 * Result (scene-owned, kept in hash-cell order; the getters return it sorted
 * by key) is the input of the next three calls. */
cb_status contact_build(cb_scene* scene, const double* x_dev, void* stream);

/* (b) Barrier filter, Sec. 3.2 / Eq. 1, 4: class F for a candidate whose
 * primitives belong to one component and whose reference distance is below
 * the activation, U otherwise.  Uses the tables built at create.  With
 * CB_PER_STENCIL it then removes the class-F candidates outside their own
 * width (boxes of the last contact_build's x); this reads a count back
 * (sync). */
cb_status contact_filter(cb_scene* scene, void* stream);

/* (c)+(d) Distances, barrier, derivatives and assembly, Eq. 2-4.
 * Per candidate: exact FP64 distance d; class C (temporary zero offset,
 * Sec. 3.4) for an unfiltered pair with d <= offset; pair parameters
 * U (xi, dhat), F (0, dbar_min), C (0, a) (single mode: U (0, a)); active iff
 * y = d - xi_p < dhat_p.  For active pairs: b(y, dhat_p), its gradient and
 * the PSD projection of kappa (b'' grad d grad d^T + b' hess d).
 * energy_dev: DEVICE 1 double per member (overwritten).  grad_dev: DEVICE [3][n]
 * (overwritten).  Either may be NULL.  The BSR matrix (full symmetric, sorted
 * columns, 3x3 row-major blocks) is scene-owned: cb_get_bsr / cb_bsr_device.
 * A pair at or inside its offset sets CB_ERR_PENETRATION and energy = +inf. */
cb_status barrier_eval(cb_scene* scene, const double* x_dev, double* energy_dev, double* grad_dev,
                       void* stream);

/* (c)+(d) energy only, for the line search over the step that ccd_step
 * bounds: E = kappa sum b(y, dhat_p) over the active candidates of the last
 * contact_build / contact_filter, with the distances, classes and pair
 * parameters of barrier_eval (Eq. 2-4), and neither gradient nor Hessian.
 * Call contact_build and contact_filter at the trial positions first.
 * energy_dev: DEVICE 1 double per member (overwritten; +inf on penetration,
 * which also sets CB_ERR_PENETRATION in the status word).  Leaves no active
 * list or BSR matrix (their getters return none until the next barrier_eval).
 * Errors: CB_ERR_ARG for a NULL scene, x_dev or energy_dev. */
cb_status barrier_energy(cb_scene* scene, const double* x_dev, double* energy_dev, void* stream);

/* (e) CCD step bound, Sec. 3.3: candidates are pairs whose swept boxes (x and
 * x + p) inflated by offset/2 overlap; each is bounded by additive CCD
 * (s = 0.1, inner factor 0.9) against its class offset (U: offset; F, C: 0).
 * alpha_dev: DEVICE 1 double per member = min(1, min_p t_p) (overwritten).
 * p_dev: DEVICE [3][n] search direction. */
cb_status ccd_step(cb_scene* scene, const double* x_dev, const double* p_dev, double* alpha_dev,
                   void* stream);

/* Batch: several scenes of one kind in one pass (one launch per stage for all
 * of them).  The batch concatenates the members' vertices, edges and
 * triangles in member order (offsets: cb_batch_offsets) and keeps each
 * member's parameters, filter tables, hash grid and results separate; pairs of
 * different members are never formed.  It copies what it needs at creation:
 * members may be destroyed afterwards.  allocator: as for cb_scene_create (the
 * batch's own buffers; the members keep theirs).  Use it with the four pass calls: x, p
 * and grad are [3][N] over the concatenated vertices (N = total), and
 * energy_dev / alpha_dev receive one double per member, in member order.
 * Pair keys and the BSR matrix use the concatenated numbering.  sync.
 * Errors: CB_ERR_ARG (null members, count < 1, mixed kinds, a member that is
 * itself a batch, index overflow), CB_ERR_OOM, CB_ERR_CUDA. */
cb_status cb_batch_create(cb_scene* const* members, int32_t count, const cb_allocator* allocator, void* stream,
                          cb_scene** out);
/* Serving (no counterpart in the paper: the request loop around its pass).
 * A server holds up to `slots` resident scenes of one kind under a device
 * memory budget and advances all of them with one batched pass: one launch
 * sequence per stage for every resident scene, the batch rebuilt only when
 * the residents change.  The caller keeps ownership of the scenes: release a
 * slot before destroying its scene.
 *   cb_server_create: kind CB_ROD / CB_SHELL, slots >= 1, budget in bytes,
 *     allocator for the server's own buffers (as cb_scene_create; NULL: the
 *     library's pool).
 *   cb_batch_admit: puts a plain scene (not a batch) of the server's kind into
 *     a free slot (*slot) if the device memory charged -- every resident scene,
 *     the batch and the pass buffers as they are now, plus twice the new
 *     scene's bytes (its pass buffers and its copy in the batch) -- stays
 *     within the budget.  CB_ERR_CAPACITY: no free slot; CB_ERR_OOM: over the
 *     budget (nothing changes); CB_ERR_ARG: wrong kind, a batch, or already
 *     resident.
 *   cb_batch_release: frees a slot.
 *   cb_batch_pass: stages a-e for every resident scene.  x, p, energy, grad,
 *     alpha: HOST arrays of `slots` DEVICE pointers indexed by slot (entries
 *     of free slots are not read; energy, grad, alpha may be NULL or hold
 *     NULL entries): x[k], p[k] [3][n_k] FP64 in, energy[k], alpha[k] one
 *     double out, grad[k] [3][n_k] out -- the values cb_scene's own pass would
 *     give (summation order aside).  Asynchronous on `stream` except for the
 *     count reads of the stages; builds the batch (sync) after the residents
 *     changed.
 *   cb_server_stats: resident scenes, bytes charged now, candidates of the
 *     last pass.
 * Errors as above, plus those of the stage calls. */
typedef struct cb_server cb_server;
cb_status cb_server_create(int32_t kind, int32_t slots, int64_t hbm_budget_bytes, const cb_allocator* allocator,
                           cb_server** out);
cb_status cb_server_destroy(cb_server* server);
cb_status cb_batch_admit(cb_server* server, cb_scene* scene, int32_t* slot);
cb_status cb_batch_release(cb_server* server, int32_t slot);
cb_status cb_batch_pass(cb_server* server, const double* const* x, const double* const* p, double* const* energy,
                        double* const* grad, double* const* alpha, void* stream);
cb_status cb_server_stats(cb_server* server, int32_t* resident, int64_t* charged_bytes, int64_t* n_candidates);

/* Pre-sizes a scene's pair-list buffers -- candidates, active pairs (BSR
 * pattern keys and Hessian queues) and CCD candidates -- for the given
 * counts, so that a pass with at most those counts allocates nothing for
 * them (the broad phase's own workspace still follows its first pass).  A
 * capacity overflow can be retried after reserving more.  sync.
 * Errors: CB_ERR_ARG, CB_ERR_TOO_LARGE (a count above 2^31 - 1), CB_ERR_OOM. */
cb_status cb_scene_reserve(cb_scene* scene, int64_t n_candidates, int64_t n_ccd, int64_t n_active, void* stream);

/* HOST arrays of count+1 entries: first vertex / edge / triangle of each
 * member in the batch numbering (a plain scene reports one member). */
cb_status cb_batch_offsets(cb_scene* scene, int64_t* vert_offsets, int64_t* edge_offsets, int64_t* tri_offsets);
/* members of a scene (1 for a plain scene) */
int32_t cb_member_count(cb_scene* scene);

/* sync getters.  Each copies to HOST buffers of capacity `cap` elements and
 * writes the full count to *count (CB_ERR_CAPACITY if cap is too small). */
cb_status cb_get_pairs(cb_scene* scene, int32_t which, uint64_t* keys, int64_t cap, int64_t* count);
/* shells: the rest-filtered stencil pairs (the filtered set F of Sec. 3.2) in key order and their
 * reference distances dbar; either output may be NULL.  Rods: CB_ERR_ARG. */
cb_status cb_get_rest_filter(cb_scene* scene, uint64_t* keys, double* dbar, int64_t cap, int64_t* count);
/* active pairs in key order: key, distance, class (0 U, 1 F, 2 C), distance type */
cb_status cb_get_active(cb_scene* scene, uint64_t* keys, double* d, uint8_t* klass, int8_t* dtype,
                        int64_t cap, int64_t* count);
/* per CCD candidate (key order): t_p and class.  The step bound needs only
 * the minimum, so pairs that provably cannot attain it are not iterated: for
 * them t holds a lower bound of t_p (their first additive-CCD step).  Bit 0x80
 * of the class byte marks an exact t_p; the low bits are 0 U, 1 F, 2 C. */
cb_status cb_get_ccd(cb_scene* scene, uint64_t* keys, double* t, uint8_t* klass, int64_t cap,
                     int64_t* count);
/* BSR: row_ptr [n+1], col [nnzb], val [nnzb][9] */
cb_status cb_get_bsr(cb_scene* scene, int32_t* row_ptr, int32_t* col, double* val, int64_t cap,
                     int64_t* nnzb);
/* device pointers of the scene-owned BSR (valid until the next barrier_eval) */
cb_status cb_bsr_device(cb_scene* scene, const int32_t** row_ptr, const int32_t** col,
                        const double** val, int64_t* nnzb);
/* y = (H + shift I) v with H the BSR matrix of the last barrier_eval (the
 * product of a Newton driver's conjugate-gradient solve; App. A).
 * v_dev, y_dev: DEVICE [3][n] FP64, distinct buffers.  Asynchronous.
 * After barrier_energy (no BSR) H counts as zero.
 * Errors: CB_ERR_ARG for a NULL scene / vector, v_dev == y_dev, or a scene
 * with no barrier_eval / barrier_energy yet. */
cb_status cb_bsr_spmv(cb_scene* scene, const double* v_dev, double* y_dev, double shift, void* stream);
/* Lagged friction on the active pairs (App. A: the paper's solver uses IPC's
 * contact and friction energies; this is IPC's lagged friction potential on
 * the pairs the filtered barrier makes active).
 *
 * friction_lag: records, for every active pair of the last barrier_eval
 * (which must have run at x_lag_dev -- barrier_energy keeps no active list),
 * the normal force lambda = -kappa b'(d - xi_p; dhat_p) >= 0 with the pair's
 * own offset and width (Eq. 2-4), the closest-point weights beta[4] of its
 * distance type (w(v) = sum_a beta_a v_a: first primitive's closest point
 * minus the second's) and the normal n = w(x_lag) / |w(x_lag)|.  mu >= 0 is
 * the friction coefficient, eps > 0 the sliding displacement (mm) below
 * which f0 is smoothed.  Single scenes only (CB_ERR_ARG for a batch).
 *
 * friction_eval: ADDS D(x) = sum_k mu lambda_k f0(|(I - n n^T) w(x - x_lag)|)
 * to energy_dev[0] and, when grad_dev is not NULL, its gradient to grad_dev
 * ([3][n]) and keeps each pair's 3x3 tangent Hessian (PSD by construction,
 * no projection) for friction_spmv.  f0(y) = -y^3/(3 eps^2) + y^2/eps +
 * eps/3 for y < eps, y otherwise.  CB_ERR_ARG before friction_lag.
 *
 * friction_spmv: y_dev += H_f v_dev (v_dev, y_dev: DEVICE [3][n], distinct),
 * H_f the friction Hessian of the last friction_eval with a gradient
 * (CB_ERR_ARG if there was none).
 *
 * cb_get_friction (sync): the lagged pairs in the order of the lists above:
 * keys [nf]; dat [8][nf] = lambda, beta[4], n[3] (element-major); hw [6][nf]
 * = packed Hessians (xx xy xz yy yz zz) of the last friction_eval with a
 * gradient.  Any of the three may be NULL; CB_ERR_CAPACITY if cap < nf.
 * All pointers of the first three calls are DEVICE pointers read or written
 * by kernels on `stream`. */
cb_status friction_lag(cb_scene* scene, const double* x_lag_dev, double mu, double eps, void* stream);
cb_status friction_eval(cb_scene* scene, const double* x_dev, const double* x_lag_dev, double* energy_dev,
                        double* grad_dev, void* stream);
cb_status friction_spmv(cb_scene* scene, const double* v_dev, double* y_dev, void* stream);
cb_status cb_get_friction(cb_scene* scene, uint64_t* keys, double* dat, double* hw, int64_t cap,
                          int64_t* count);
cb_status cb_get_stats(cb_scene* scene, cb_stats* stats);
/* sync: first device-side condition since the last call (then cleared) */
cb_status cb_sync_status(cb_scene* scene);

/* Per-stage device times in milliseconds of the last calls (CUDA events):
 * [0] contact_build, [1] contact_filter, [2] barrier_eval, [3] ccd_step,
 * [4] barrier_eval Hessian kernel alone.  sync. */
cb_status cb_get_stage_ms(cb_scene* scene, float* ms5);
/* The same times and the two parts of barrier_eval, `count` floats (HOST):
 * [0..4] as cb_get_stage_ms, [5] stage (c) -- FP32 screen, exact distances,
 * classes and the active set (Eq. 2-4, Sec. 3.4) -- and [6] stage (d) --
 * compaction, BSR pattern, barrier derivatives, PSD projection, assembly;
 * [5] + [6] = [2].  [5] and [6] are 0 after a barrier_energy or a pass with no
 * candidates; entries past 7 are 0.  sync.  Errors: CB_ERR_ARG. */
cb_status cb_get_stage_times(cb_scene* scene, float* ms, int32_t count);
/* Tuning knobs of a broad phase (no counterpart in the paper; no result
 * depends on them, only speed).  phase 0: contact_build's broad phase, 1:
 * ccd_step's swept broad phase.  cell_factor in (0, 64]: hash cell edge =
 * factor x the members' mean primitive box extent (rounded to a quarter
 * octave; default 1).  pair_block: threads per block of the pair enumeration,
 * 64, 128 or 256 (default 256).  A batch starts from its first member's
 * settings.  Errors: CB_ERR_ARG. */
cb_status cb_set_tuning(cb_scene* scene, int32_t phase, float cell_factor, int32_t pair_block);
cb_status cb_get_tuning(cb_scene* scene, int32_t phase, float* cell_factor, int32_t* pair_block);
/* enable (1) / disable (0) the stage events; default off */
cb_status cb_set_timing(cb_scene* scene, int32_t on);

const char* cb_status_str(cb_status s);
/* process-wide number of CUDA kernels the library has launched so far */
int64_t cb_kernel_launches(void);
/* Diagnostic (no counterpart in the paper): measured fused-multiply-add
 * throughput of the current GPU in TFLOP/s (2 flops per FMA), fp64 = 1 for
 * double, 0 for float; `blocks` blocks of 256 threads, `iters` x 8 FMA each.
 * Used as the roofline denominator of the FP64-bound kernels.  sync. */
cb_status cb_measure_fma_tflops(int32_t fp64, int32_t blocks, int32_t iters, double* tflops);
/* library version string */
const char* cb_version(void);

/* Step bound of an explicit stencil list that allocates no device memory.
 * No counterpart in the paper: it is ccd_step's additive CCD (same s, inner
 * factor, iteration cap and arithmetic) for callers that cannot allocate
 * device memory while they run it -- a solver that has handed its whole
 * device budget to its own pool, or a time-critical loop in which an
 * allocation or a free could stall the device.  The only memory it uses is a
 * fixed scratch array of the library, 8 MiB + 256 bytes per device, set aside
 * when the library's code is loaded onto the device.
 *   x_dev, p_dev  DEVICE [3][n_verts] FP64 positions and search direction.
 *   stencils_dev  DEVICE [n_stencils][4] int32 vertex ids: point-triangle
 *                 (p, t0, t1, t2) or edge-edge (a0, a1, b0, b1).
 *   is_ee_dev     DEVICE [n_stencils] uint8: 1 edge-edge, 0 point-triangle.
 *   offset_dev    DEVICE [n_stencils] FP64 offset the step keeps (>= 0).
 *   alpha_dev     DEVICE 1 double: min(1, min_p t_p) (overwritten).
 *   flags_dev     DEVICE 1 uint32 (overwritten): CB_DEV conditions 2
 *                 (penetration: a stencil at or inside its offset, t_p = 0),
 *                 4 (iteration limit) and CB_NOALLOC_BAD_STENCIL (a vertex id
 *                 outside [0, n_verts), a negative or non-finite offset, or a
 *                 non-finite position or displacement: that stencil is
 *                 skipped and does not bound alpha -- check the flag).
 * The caller owns every buffer; each must be memory of the current device
 * (or managed memory), else CB_ERR_ARG before any work.  The call is
 * asynchronous on `stream`, which must belong to the current device.
 * n_stencils = 0 gives alpha = 1.  More than CB_NOALLOC_MAX_STENCILS stencils
 * return CB_ERR_TOO_LARGE before any work; split the list and take the
 * minimum.  The first call on each device looks up the scratch address and may
 * make the CUDA runtime load the library's code onto that device: make it
 * before any stream capture.  The address is kept for the life of the
 * process: do not use this call on a device after cudaDeviceReset there.  All calls on one device share the scratch:
 * calls that overlap in time on one device (several streams or host threads)
 * race and give wrong results.  Errors: CB_ERR_ARG, CB_ERR_TOO_LARGE,
 * CB_ERR_CUDA. */
#define CB_NOALLOC_MAX_STENCILS (1 << 20)
#define CB_NOALLOC_BAD_STENCIL 8u
cb_status ccd_step_noalloc(const double* x_dev, const double* p_dev, int32_t n_verts, const int32_t* stencils_dev,
                           const uint8_t* is_ee_dev, const double* offset_dev, int64_t n_stencils,
                           double* alpha_dev, uint32_t* flags_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif
