// api.cu -- C ABI of the contact library: scene lifetime, the four pass calls,
// getters.  Host code only orchestrates; every stage runs in the kernels of
// broad.cu, narrow.cu and ccd.cu.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "scene.cuh"

#include <atomic>
static std::atomic<long long> g_launches{0};
long long cb_launch_counter_add() { return g_launches.fetch_add(1, std::memory_order_relaxed) + 1; }

AllocCtx& alloc_ctx() {
  static thread_local AllocCtx ctx;
  return ctx;
}

cb_status buf_ensure(DevBuf& b, size_t bytes, cudaStream_t st) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return CB_OK;
  buf_free(b, st);
  const size_t want = bytes + bytes / 4 + 256;
  const AllocCtx& c = alloc_ctx();
  if (c.alloc) {
    void* p = c.alloc->alloc(want, (void*)st, c.alloc->ctx);
    if (!p) return CB_ERR_OOM;
    if ((uintptr_t)p & 255u) {  // every buffer must be 256-byte aligned (vector loads of any width)
      fprintf(stderr, "contact: the caller's allocator returned a pointer that is not 256-byte aligned\n");
      c.alloc->free(p, want, (void*)st, c.alloc->ctx);
      return CB_ERR_OOM;
    }
    b.p = p;
  } else if (cudaMallocAsync(&b.p, want, st) != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return CB_ERR_OOM;
  }
  b.bytes = want;
  b.alloc = c.alloc;
  b.charged = c.charged;
  if (b.charged) *b.charged += (int64_t)want;
  return CB_OK;
}

void buf_free(DevBuf& b, cudaStream_t st) {
  if (b.p) {
    if (b.alloc) {
      // the caller's allocator may reuse the memory as soon as it has it back
      cudaStreamSynchronize(st);
      b.alloc->free(b.p, b.bytes, (void*)st, b.alloc->ctx);
    } else {
      cudaFreeAsync(b.p, st);
    }
    if (b.charged) *b.charged -= (int64_t)b.bytes;
  }
  b.p = nullptr;
  b.bytes = 0;
  b.alloc = nullptr;
  b.charged = nullptr;
}

cb_status read_scalars(cb_scene* s, int first, int count, uint64_t* out, cudaStream_t st) {
  CB_CUDA(cudaMemcpyAsync(s->h_pinned, scalars(s) + first, sizeof(uint64_t) * count, cudaMemcpyDeviceToHost, st));
  CB_CUDA(cudaStreamSynchronize(st));
  memcpy(out, s->h_pinned, sizeof(uint64_t) * count);
  return CB_OK;
}

static int bits_needed(int64_t max_value) {
  int b = 1;
  while ((1ll << b) <= max_value) ++b;
  return b;
}

template <typename T>
static cb_status upload(DevBuf& b, const T* h, size_t count, cudaStream_t st) {
  CB_TRY(buf_ensure(b, sizeof(T) * std::max<size_t>(count, 1), st));
  if (count) CB_CUDA(cudaMemcpyAsync(b.p, h, sizeof(T) * count, cudaMemcpyHostToDevice, st));
  return CB_OK;
}

static void scene_release(cb_scene* s) {
  cudaStream_t st = s->last_stream;
  DevBuf* bufs[] = {&s->ev0, &s->ev1, &s->tv, &s->comp, &s->rest, &s->rod_ptr, &s->S, &s->win, &s->wst,
                    &s->rloop, &s->rlast, &s->elen2, &s->hmoll, &s->mlist, &s->ruv, &s->frest,
                    &s->frest_dbar, &s->frest_j, &s->frow_pt, &s->frow_ee, &s->dbar_comp, &s->cand, &s->klass, &s->cand_alt, &s->klass_alt, &s->cd, &s->cflag, &s->cpos, &s->ctype, &s->ccls, &s->aidx,
                    &s->bkey[0], &s->bkey[1], &s->bflag, &s->bpos, &s->bsr_row, &s->bsr_col, &s->bsr_val,
                    &s->row_cnt, &s->hB9, &s->hB6, &s->hB4, &s->hslot, &s->horder, &s->xf, &s->pf, &s->dlist, &s->mp, &s->vsc, &s->macc, &s->ccd_keys, &s->ccd_t, &s->ccd_cls, &s->ccd_lb, &s->ccd_flag, &s->ccd_pos, &s->ccd_list, &s->ccd_ulist, &s->scan_tmp, &s->hist,
                    &s->fr_key, &s->fr_st, &s->fr_dat, &s->fr_hw, &s->dev_scalars};
  for (DevBuf* b : bufs) buf_free(*b, st);
  for (BroadWork* w : {&s->bw, &s->bwc}) {
    DevBuf* wb[] = {&w->grids, &w->cx, &w->box32,   &w->box64,  &w->box_raw, &w->bounds,   &w->cell_cnt, &w->cell_off, &w->ekey[0], &w->ekey[1],
                    &w->eval[0], &w->eval[1], &w->run_flag, &w->run_id,   &w->run_start, &w->pair_cnt,
                    &w->pair_off, &w->ebox, &w->ckey[0], &w->ckey[1],  &w->stage, &w->ovl, &w->scan_tmp, &w->hist,
                    &w->flat_len, &w->flat_off, &w->flat_j0, &w->flat_bits, &w->flat_slen, &w->flat_sbits,
                    &w->flat_lflag, &w->flat_lpos, &w->flat_lidx, &w->flat_llen, &w->flat_vlong};
    for (DevBuf* b : wb) buf_free(*b, st);
  }
  cudaStreamSynchronize(st);
  if (s->h_pinned) cudaFreeHost(s->h_pinned);
  if (s->hstage_host) cudaFreeHost(s->hstage_host);
  for (auto& e : s->ev)
    if (e) cudaEventDestroy(e);
  delete s;
}

// --- device helpers for scene / batch set-up -------------------------------
__global__ void k_offset_copy(int32_t* __restrict__ dst, const int32_t* __restrict__ src, int64_t n, int32_t add) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[i] + add;
}
// as k_offset_copy, negative entries (markers) copied unchanged
__global__ void k_offset_copy_nonneg(int32_t* __restrict__ dst, const int32_t* __restrict__ src, int64_t n,
                                     int32_t add) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[i] >= 0 ? src[i] + add : src[i];
}
__global__ void k_comp_copy(int32_t* __restrict__ dst, const int32_t* __restrict__ src, int64_t n, int32_t add_lbl,
                            int32_t add_v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[i] >= 0 ? src[i] + add_lbl : src[i] - add_v;
}
__global__ void k_fill_i32(int32_t* __restrict__ dst, int64_t n, int32_t v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = v;
}
// pair keys of a member -> keys of the batch (indices shifted)
__global__ void k_key_shift(uint64_t* __restrict__ dst, const uint64_t* __restrict__ src, int64_t n, uint32_t add_i,
                            uint32_t add_j) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const uint64_t k = src[q];
  dst[q] = cb_key(cb_key_type(k), cb_key_i(k) + add_i, cb_key_j(k) + add_j);
}
// number of keys below `bound` in a sorted array (one thread)
__global__ void k_lower_bound(const uint64_t* __restrict__ a, int64_t n, uint64_t bound, uint64_t* out) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (a[mid] < bound) lo = mid + 1;
    else hi = mid;
  }
  *out = (uint64_t)lo;
}

static cb_status alloc_members(cb_scene* s, cudaStream_t st) {
  const int M = s->count;
  CB_TRY(buf_ensure(s->mp, sizeof(MemberParams) * (size_t)M, st));
  CB_TRY(buf_ensure(s->macc, sizeof(unsigned long long) * MACC_STRIDE * (size_t)M, st));
  CB_CUDA(cudaMemsetAsync(s->macc.p, 0, sizeof(unsigned long long) * MACC_STRIDE * (size_t)M, st));
  // per member: the largest record staged through it (member parameters,
  // the CCD accumulators)
  const size_t per = std::max(sizeof(MemberParams), sizeof(unsigned long long) * MACC_STRIDE);
  if (cudaMallocHost(&s->hstage_host, per * (size_t)M + 256) != cudaSuccess) return CB_ERR_OOM;
  return CB_OK;
}

static float float_up(double v) {
  float f = (float)v;
  if ((double)f < v) f = std::nextafter(f, INFINITY);
  return f;
}

static cb_status upload_members(cb_scene* s, cudaStream_t st) {
  for (MemberParams& m : s->hmp) {
    m.thrU32 = float_up(m.a * (1.0 + 1e-9) + 1e-9);
    m.thrF32 = float_up(std::max(m.dbar_min, m.dbar_fmax) * (1.0 + 1e-9) + 1e-9);
    m.thrC32 = float_up(m.xi * (1.0 + 1e-9) + 1e-9);
    m.xi32 = float_up(m.xi);
  }
  memcpy(s->hstage_host, s->hmp.data(), sizeof(MemberParams) * s->hmp.size());
  CB_CUDA(cudaMemcpyAsync(s->mp.p, s->hstage_host, sizeof(MemberParams) * s->hmp.size(), cudaMemcpyHostToDevice, st));
  CB_CUDA(cudaStreamSynchronize(st));
  return CB_OK;
}

template <typename T>
static cb_status dl(std::vector<T>& h, const DevBuf& b, int64_t count, cudaStream_t st) {
  h.resize((size_t)count);
  if (count) CB_CUDA(cudaMemcpyAsync(h.data(), b.p, sizeof(T) * (size_t)count, cudaMemcpyDeviceToHost, st));
  return CB_OK;
}

extern "C" {

int64_t cb_kernel_launches(void) { return (int64_t)g_launches.load(std::memory_order_relaxed); }

const char* cb_version(void) { return "gb300-contact 0.1 (sm_103a)"; }

const char* cb_status_str(cb_status st) {
  switch (st) {
    case CB_OK: return "ok";
    case CB_ERR_ARG: return "invalid argument";
    case CB_ERR_OOM: return "device allocation failed";
    case CB_ERR_CAPACITY: return "buffer capacity exceeded";
    case CB_ERR_PENETRATION: return "pair at or inside its barrier offset";
    case CB_ERR_DEGENERATE: return "zero reference distance between stencil primitives";
    case CB_ERR_ITER_LIMIT: return "additive CCD iteration limit reached";
    case CB_ERR_CUDA: return "CUDA runtime error";
    case CB_ERR_TOO_LARGE: return "input larger than the call's fixed maximum";
  }
  return "unknown status";
}

cb_status cb_scene_create(const cb_scene_desc* d, const cb_allocator* allocator, void* stream, cb_scene** out) {
  if (!d || !out || !d->rest_xyz || d->n_verts < 1) return CB_ERR_ARG;
  if (allocator && (!allocator->alloc || !allocator->free)) return CB_ERR_ARG;
  if (d->kind != CB_ROD && d->kind != CB_SHELL) return CB_ERR_ARG;
  if (!(d->dhat > 0.0) || !(d->thickness >= 0.0) || !std::isfinite(d->thickness) || !std::isfinite(d->dhat))
    return CB_ERR_ARG;
  const int fm = d->mode & CB_FILTER_MASK;
  if (d->mode & ~(CB_FILTER_MASK | CB_THICK_PAPER_LITERAL | CB_NO_CORE_TEMP | CB_DBAR_PER_COMPONENT |
                  CB_EE_MOLLIFIER | CB_PER_STENCIL | CB_DBAR_GEODESIC))
    return CB_ERR_ARG;
  if (fm == CB_FILTER_KALDOR && (d->kind != CB_ROD || d->cull_radius < 1)) return CB_ERR_ARG;
  if (d->rest_uv && d->kind != CB_SHELL) return CB_ERR_ARG;
  const bool geodesic = (d->mode & CB_DBAR_GEODESIC) != 0;
  if (geodesic && (d->kind != CB_SHELL || d->rest_uv)) return CB_ERR_ARG;
  const int n = d->n_verts;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int32_t> e0, e1, comp(n), rloop, rlast;
  std::vector<int32_t> tris;
  int T = 0;
  if (d->kind == CB_ROD) {
    if (d->n_rods < 1 || !d->rod_ptr) return CB_ERR_ARG;
    for (int r = 0; r < d->n_rods; ++r)
      if (d->rod_ptr[r] < 0 || d->rod_ptr[r + 1] < d->rod_ptr[r] || d->rod_ptr[r + 1] > n) return CB_ERR_ARG;
    for (int v = 0; v < n; ++v) comp[v] = -1 - v;
    for (int r = 0; r < d->n_rods; ++r) {
      const int p0 = d->rod_ptr[r], p1 = d->rod_ptr[r + 1];
      const bool closed = d->rod_closed && d->rod_closed[r];
      if (closed && p1 - p0 < 3) return CB_ERR_ARG;  // a loop needs three vertices
      for (int v = p0; v < p1; ++v) comp[v] = r;
      const int first = (int)e0.size();
      for (int v = p0; v + 1 < p1; ++v) {
        e0.push_back(v);
        e1.push_back(v + 1);
      }
      if (closed) {  // the closing edge, after the polyline's others
        e0.push_back(p1 - 1);
        e1.push_back(p0);
      }
      const int ne = (int)e0.size() - first;
      for (int k = 0; k < ne; ++k) {
        rloop.push_back(closed ? ne : 0);
        rlast.push_back(closed ? first + ne - 1 : -1);
      }
    }
  } else {
    T = d->n_tris;
    if (T < 0 || (T > 0 && !d->tris)) return CB_ERR_ARG;
    tris.assign(d->tris, d->tris + 3 * (size_t)T);
    std::vector<uint64_t> ek;
    ek.reserve(3 * (size_t)T);
    for (int t = 0; t < T; ++t) {
      int a = tris[t], b = tris[T + t], c = tris[2 * T + t];
      if (a < 0 || b < 0 || c < 0 || a >= n || b >= n || c >= n || a == b || b == c || a == c) return CB_ERR_ARG;
      int vv[3] = {a, b, c};
      for (int k = 0; k < 3; ++k) {
        int p = vv[k], q = vv[(k + 1) % 3];
        ek.push_back((uint64_t)std::min(p, q) * (uint64_t)n + (uint64_t)std::max(p, q));
      }
    }
    std::sort(ek.begin(), ek.end());
    ek.erase(std::unique(ek.begin(), ek.end()), ek.end());
    for (uint64_t k : ek) {
      e0.push_back((int32_t)(k / n));
      e1.push_back((int32_t)(k % n));
    }
    std::vector<int32_t> parent(n);
    std::iota(parent.begin(), parent.end(), 0);
    auto find = [&](int i) {
      while (parent[i] != i) {
        parent[i] = parent[parent[i]];
        i = parent[i];
      }
      return i;
    };
    for (size_t k = 0; k < e0.size(); ++k) {
      int ra = find(e0[k]), rb = find(e1[k]);
      if (ra != rb) parent[std::max(ra, rb)] = std::min(ra, rb);
    }
    for (int v = 0; v < n; ++v) comp[v] = find(v);
  }
  const int E = (int)e0.size();
  // geodesic reference distances: the mesh adjacency (a manifold: at most two faces per edge)
  std::vector<int32_t> geo_te, geo_ef, geo_vfp, geo_vf;
  if (geodesic) {
    auto edge_id = [&](int p, int q) {
      const uint64_t k = (uint64_t)std::min(p, q) * (uint64_t)n + (uint64_t)std::max(p, q);
      int lo = 0, hi = E;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((uint64_t)e0[mid] * (uint64_t)n + (uint64_t)e1[mid] < k) lo = mid + 1;
        else hi = mid;
      }
      return lo;
    };
    geo_te.resize(3 * (size_t)T);
    geo_ef.assign(2 * (size_t)E, -1);
    geo_vfp.assign((size_t)n + 1, 0);
    geo_vf.resize(3 * (size_t)T);
    for (int t = 0; t < T; ++t)
      for (int k = 0; k < 3; ++k) {
        const int e = edge_id(tris[(size_t)k * T + t], tris[(size_t)((k + 1) % 3) * T + t]);
        geo_te[3 * (size_t)t + k] = e;
        if (geo_ef[2 * (size_t)e] < 0) geo_ef[2 * (size_t)e] = t;
        else if (geo_ef[2 * (size_t)e + 1] < 0) geo_ef[2 * (size_t)e + 1] = t;
        else return CB_ERR_ARG;  // an edge of three faces: no geodesic distance
        ++geo_vfp[(size_t)tris[(size_t)k * T + t] + 1];
      }
    for (int v = 0; v < n; ++v) geo_vfp[(size_t)v + 1] += geo_vfp[v];
    std::vector<int32_t> fill(geo_vfp.begin(), geo_vfp.end() - 1);
    for (int t = 0; t < T; ++t)
      for (int k = 0; k < 3; ++k) geo_vf[(size_t)fill[tris[(size_t)k * T + t]]++] = t;
  }
  cb_scene* s = new cb_scene();
  if (allocator) {
    s->allocator = *allocator;
    s->has_alloc = true;
  }
  AllocScope scope(s->alloc_ptr(), &s->live_bytes);
  s->kind = d->kind;
  s->n = n;
  s->E = E;
  s->T = T;
  s->n_rods = d->kind == CB_ROD ? d->n_rods : 0;
  s->n_prims = d->kind == CB_ROD ? E : n + T + E;
  if (d->kind == CB_ROD) {
    s->bits_i = s->bits_j = bits_needed(std::max(E - 1, 1));
  } else {
    s->bits_i = bits_needed(std::max(std::max(n, E) - 1, 1));
    s->bits_j = bits_needed(std::max(std::max(T, E) - 1, 1));
  }
  if (s->bits_i > 31 || s->bits_j > 31) {
    delete s;
    return CB_ERR_ARG;
  }
  s->filter = fm;
  s->core_temp = (d->mode & CB_NO_CORE_TEMP) ? 0 : 1;
  if (d->mode & CB_THICK_PAPER_LITERAL) {
    s->a = d->thickness;
    s->xi = d->thickness - d->dhat;
    if (s->xi < 0.0) {
      delete s;
      return CB_ERR_ARG;
    }
  } else {
    s->xi = d->thickness;
    s->a = d->thickness + d->dhat;
  }
  s->dhat = d->dhat;
  s->kappa = d->kappa > 0.0 ? d->kappa : 1.0;
  s->geodesic = geodesic;
  s->geo_te.swap(geo_te);
  s->geo_ef.swap(geo_ef);
  s->geo_vfp.swap(geo_vfp);
  s->geo_vf.swap(geo_vf);
  s->last_stream = st;
  cudaGetDevice(&s->device);
  cudaDeviceGetAttribute(&s->n_sms, cudaDevAttrMultiProcessorCount, s->device);
  if (s->n_sms < 1) s->n_sms = 1;
  s->count = 1;
  s->hmp.assign(1, MemberParams{s->xi, s->dhat, s->a, s->kappa, 0.0, fm == CB_FILTER_SINGLE ? 1 : 0, s->core_temp,
                                (fm == CB_FILTER_OFF || fm == CB_FILTER_KALDOR) ? 1 : 0, s->n_prims});
  s->hmp[0].cull_radius = fm == CB_FILTER_KALDOR ? d->cull_radius : 0;
  s->hmp[0].per_comp = (d->mode & CB_DBAR_PER_COMPONENT) ? 1 : 0;
  s->hmp[0].mollify = (d->mode & CB_EE_MOLLIFIER) ? 1 : 0;
  s->hmp[0].per_stencil = (d->mode & CB_PER_STENCIL) ? 1 : 0;
  s->hmp[0].loops = 0;
  for (int32_t lc : rloop) s->hmp[0].loops |= lc > 0 ? 1 : 0;
  s->voff = {0, (int64_t)n};
  s->eoff = {0, (int64_t)E};
  s->toff = {0, (int64_t)T};
  cb_status rc = CB_OK;
  auto fail = [&](cb_status e) {
    scene_release(s);
    return e;
  };
  if ((rc = alloc_members(s, st)) != CB_OK) return fail(rc);
  if ((rc = buf_ensure(s->vsc, sizeof(int32_t) * (size_t)n, st)) != CB_OK) return fail(rc);
  if (cudaMemsetAsync(s->vsc.p, 0, sizeof(int32_t) * (size_t)n, st) != cudaSuccess) return fail(CB_ERR_CUDA);
  if (cudaMallocHost((void**)&s->h_pinned, 64 * sizeof(uint64_t)) != cudaSuccess) return fail(CB_ERR_OOM);
  if ((rc = buf_ensure(s->dev_scalars, SC_N * sizeof(uint64_t), st)) != CB_OK) return fail(rc);
  if (cudaMemsetAsync(s->dev_scalars.p, 0, SC_N * sizeof(uint64_t), st) != cudaSuccess) return fail(CB_ERR_CUDA);
  if ((rc = upload(s->ev0, e0.data(), e0.size(), st)) != CB_OK) return fail(rc);
  if ((rc = upload(s->ev1, e1.data(), e1.size(), st)) != CB_OK) return fail(rc);
  {
    // squared rest length of every edge (the edge-edge mollifier's threshold)
    std::vector<double> l2(e0.size());
    for (size_t k = 0; k < e0.size(); ++k) {
      double acc = 0.0;
      for (int c = 0; c < 3; ++c) {
        const double dv = d->rest_xyz[(size_t)c * n + e1[k]] - d->rest_xyz[(size_t)c * n + e0[k]];
        acc += dv * dv;
      }
      l2[k] = acc;
    }
    if ((rc = upload(s->elen2, l2.data(), l2.size(), st)) != CB_OK) return fail(rc);
  }
  if ((rc = upload(s->tv, tris.data(), tris.size(), st)) != CB_OK) return fail(rc);
  if ((rc = upload(s->comp, comp.data(), comp.size(), st)) != CB_OK) return fail(rc);
  if ((rc = upload(s->rest, d->rest_xyz, 3 * (size_t)n, st)) != CB_OK) return fail(rc);
  if (d->rest_uv) {  // the pattern as (u, v, 0): the rest-filter precompute runs on it
    std::vector<double> uv3(3 * (size_t)n, 0.0);
    std::memcpy(uv3.data(), d->rest_uv, sizeof(double) * 2 * (size_t)n);
    if ((rc = upload(s->ruv, uv3.data(), uv3.size(), st)) != CB_OK) return fail(rc);
  }
  if (d->kind == CB_ROD && (rc = upload(s->rod_ptr, d->rod_ptr, (size_t)d->n_rods + 1, st)) != CB_OK) return fail(rc);
  if (d->kind == CB_ROD && (rc = upload(s->rloop, rloop.data(), rloop.size(), st)) != CB_OK) return fail(rc);
  if (d->kind == CB_ROD && (rc = upload(s->rlast, rlast.data(), rlast.size(), st)) != CB_OK) return fail(rc);
  if (d->kind == CB_ROD && (rc = buf_ensure(s->frest, 16, st)) != CB_OK) return fail(rc);
  if (d->kind == CB_SHELL && (rc = buf_ensure(s->win, 16, st)) != CB_OK) return fail(rc);
  if (d->kind == CB_SHELL && (rc = buf_ensure(s->wst, 16, st)) != CB_OK) return fail(rc);
  if (d->kind == CB_SHELL && (rc = buf_ensure(s->rloop, 16, st)) != CB_OK) return fail(rc);
  for (auto& e : s->ev)
    if (cudaEventCreate(&e) != cudaSuccess) return fail(CB_ERR_CUDA);
  // the rest broad phase reads the member parameters (box inflation, primitive count)
  if ((rc = upload_members(s, st)) != CB_OK) return fail(rc);
  if ((rc = filter_precompute(s, st)) != CB_OK) return fail(rc);
  // the adjacency served the geodesic rest filter only
  std::vector<int32_t>().swap(s->geo_te);
  std::vector<int32_t>().swap(s->geo_ef);
  std::vector<int32_t>().swap(s->geo_vfp);
  std::vector<int32_t>().swap(s->geo_vf);
  s->hmp[0].dbar_min = std::isfinite(s->dbar_min) ? s->dbar_min : 0.0;
  s->hmp[0].dbar_fmax = s->hmp[0].per_comp && std::isfinite(s->dbar_fmax) ? s->dbar_fmax : s->hmp[0].dbar_min;
  if ((rc = upload_members(s, st)) != CB_OK) return fail(rc);
  if (s->kind == CB_SHELL && s->n_frest > 0) {
    k_lower_bound<<<1, 1, 0, cb_count(st)>>>(bp<uint64_t>(s->frest), s->n_frest, (uint64_t)CB_KEY_EE << 62,
                                             scalars(s) + SC_COUNT1);
    uint64_t h;
    if ((rc = read_scalars(s, SC_COUNT1, 1, &h, st)) != CB_OK) return fail(rc);
    s->n_frest_pt = (int64_t)h;
  }
  if ((rc = frest_rows_build(s, st)) != CB_OK) return fail(rc);
  if (cudaStreamSynchronize(st) != cudaSuccess) return fail(CB_ERR_CUDA);
  *out = s;
  return CB_OK;
}

cb_status cb_batch_create(cb_scene* const* members, int32_t count, const cb_allocator* allocator, void* stream,
                          cb_scene** out) {
  if (!members || count < 1 || !out) return CB_ERR_ARG;
  if (allocator && (!allocator->alloc || !allocator->free)) return CB_ERR_ARG;
  for (int m = 0; m < count; ++m)
    if (!members[m] || members[m]->count != 1 || members[m]->kind != members[0]->kind) return CB_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cb_scene* b = new cb_scene();
  if (allocator) {
    b->allocator = *allocator;
    b->has_alloc = true;
  }
  AllocScope scope(b->alloc_ptr(), &b->live_bytes);
  b->kind = members[0]->kind;
  b->count = count;
  b->last_stream = st;
  for (int ph = 0; ph < 2; ++ph) {
    BroadWork& dst = ph ? b->bwc : b->bw;
    const BroadWork& src = ph ? members[0]->bwc : members[0]->bw;
    dst.cell_factor = src.cell_factor;
    dst.pair_block = src.pair_block;
  }
  cudaGetDevice(&b->device);
  cudaDeviceGetAttribute(&b->n_sms, cudaDevAttrMultiProcessorCount, b->device);
  if (b->n_sms < 1) b->n_sms = 1;
  b->voff.assign(count + 1, 0);
  b->eoff.assign(count + 1, 0);
  b->toff.assign(count + 1, 0);
  std::vector<int64_t> roff(count + 1, 0);
  int64_t nf = 0, nf_pt = 0;
  for (int m = 0; m < count; ++m) {
    const cb_scene* s = members[m];
    b->voff[m + 1] = b->voff[m] + s->n;
    b->eoff[m + 1] = b->eoff[m] + s->E;
    b->toff[m + 1] = b->toff[m] + s->T;
    roff[m + 1] = roff[m] + s->n_rods;
    b->hmp.push_back(s->hmp[0]);
    nf += s->n_frest;
    nf_pt += s->n_frest_pt;
  }
  if (b->voff[count] > 0x7fffffff || b->eoff[count] > 0x7fffffff || b->toff[count] > 0x7fffffff) {
    delete b;
    return CB_ERR_ARG;
  }
  b->n = (int)b->voff[count];
  b->E = (int)b->eoff[count];
  b->T = (int)b->toff[count];
  b->n_rods = (int)roff[count];
  b->n_prims = b->kind == CB_ROD ? b->E : b->n + b->T + b->E;
  if (b->kind == CB_ROD) {
    b->bits_i = b->bits_j = bits_needed(std::max(b->E - 1, 1));
  } else {
    b->bits_i = bits_needed(std::max(std::max(b->n, b->E) - 1, 1));
    b->bits_j = bits_needed(std::max(std::max(b->T, b->E) - 1, 1));
  }
  const MemberParams& m0 = b->hmp[0];
  b->xi = m0.xi;
  b->dhat = m0.dhat;
  b->a = m0.a;
  b->kappa = m0.kappa;
  b->filter = m0.cull_radius > 0 ? CB_FILTER_KALDOR
                                 : (m0.filter_off ? CB_FILTER_OFF : (m0.single ? CB_FILTER_SINGLE : CB_FILTER_DOUBLE));
  b->core_temp = m0.core_temp;
  b->dbar_min = INFINITY;
  for (int m = 0; m < count; ++m)
    if (std::isfinite(members[m]->dbar_min)) b->dbar_min = std::min(b->dbar_min, members[m]->dbar_min);
  cb_status rc = CB_OK;
  auto fail = [&](cb_status e) {
    scene_release(b);
    return e;
  };
  if (cudaMallocHost((void**)&b->h_pinned, 64 * sizeof(uint64_t)) != cudaSuccess) return fail(CB_ERR_OOM);
  if ((rc = buf_ensure(b->dev_scalars, SC_N * sizeof(uint64_t), st)) != CB_OK) return fail(rc);
  if (cudaMemsetAsync(b->dev_scalars.p, 0, SC_N * sizeof(uint64_t), st) != cudaSuccess) return fail(CB_ERR_CUDA);
  if ((rc = alloc_members(b, st)) != CB_OK) return fail(rc);
  if ((rc = buf_ensure(b->ev0, sizeof(int32_t) * (size_t)std::max(1, b->E), st)) != CB_OK) return fail(rc);
  if ((rc = buf_ensure(b->ev1, sizeof(int32_t) * (size_t)std::max(1, b->E), st)) != CB_OK) return fail(rc);
  if ((rc = buf_ensure(b->tv, sizeof(int32_t) * 3 * (size_t)std::max(1, b->T), st)) != CB_OK) return fail(rc);
  if ((rc = buf_ensure(b->comp, sizeof(int32_t) * (size_t)b->n, st)) != CB_OK) return fail(rc);
  if ((rc = buf_ensure(b->vsc, sizeof(int32_t) * (size_t)b->n, st)) != CB_OK) return fail(rc);
  if ((rc = buf_ensure(b->win, sizeof(int32_t) * (size_t)std::max(1, b->E), st)) != CB_OK) return fail(rc);
  if ((rc = buf_ensure(b->wst, sizeof(int32_t) * (size_t)std::max(1, b->E), st)) != CB_OK) return fail(rc);
  if ((rc = buf_ensure(b->elen2, sizeof(double) * (size_t)std::max(1, b->E), st)) != CB_OK) return fail(rc);
  if ((rc = buf_ensure(b->rloop, sizeof(int32_t) * (size_t)std::max(1, b->E), st)) != CB_OK) return fail(rc);
  if ((rc = buf_ensure(b->frest, sizeof(uint64_t) * (size_t)std::max<int64_t>(1, nf), st)) != CB_OK) return fail(rc);
  int64_t wpt = 0, wee = nf_pt;
  for (int m = 0; m < count; ++m) {
    const cb_scene* s = members[m];
    const int32_t vo = (int32_t)b->voff[m], eo = (int32_t)b->eoff[m], to = (int32_t)b->toff[m];
    if (s->E > 0) {
      k_offset_copy<<<cb_grid(s->E), CB_THREADS, 0, cb_count(st)>>>(bp<int32_t>(b->ev0) + eo, bp<int32_t>(s->ev0),
                                                                     s->E, vo);
      k_offset_copy<<<cb_grid(s->E), CB_THREADS, 0, cb_count(st)>>>(bp<int32_t>(b->ev1) + eo, bp<int32_t>(s->ev1),
                                                                     s->E, vo);
      CB_CUDA(cudaMemcpyAsync(bp<double>(b->elen2) + eo, s->elen2.p, sizeof(double) * (size_t)s->E,
                              cudaMemcpyDeviceToDevice, st));
      if (b->kind == CB_ROD) {
        k_offset_copy<<<cb_grid(s->E), CB_THREADS, 0, cb_count(st)>>>(bp<int32_t>(b->win) + eo,
                                                                       bp<int32_t>(s->win), s->E, eo);
        // wst: -1 (no backward window) stays -1; rloop: counts, no offset
        k_offset_copy_nonneg<<<cb_grid(s->E), CB_THREADS, 0, cb_count(st)>>>(bp<int32_t>(b->wst) + eo,
                                                                              bp<int32_t>(s->wst), s->E, eo);
        k_offset_copy<<<cb_grid(s->E), CB_THREADS, 0, cb_count(st)>>>(bp<int32_t>(b->rloop) + eo,
                                                                       bp<int32_t>(s->rloop), s->E, 0);
      }
    }
    for (int k = 0; k < 3 && s->T > 0; ++k)
      k_offset_copy<<<cb_grid(s->T), CB_THREADS, 0, cb_count(st)>>>(
          bp<int32_t>(b->tv) + (size_t)k * b->T + to, bp<int32_t>(s->tv) + (size_t)k * s->T, s->T, vo);
    const int32_t lbl = b->kind == CB_ROD ? (int32_t)roff[m] : vo;
    k_comp_copy<<<cb_grid(s->n), CB_THREADS, 0, cb_count(st)>>>(bp<int32_t>(b->comp) + vo, bp<int32_t>(s->comp),
                                                                 s->n, lbl, vo);
    k_fill_i32<<<cb_grid(s->n), CB_THREADS, 0, cb_count(st)>>>(bp<int32_t>(b->vsc) + vo, s->n, m);
    if (b->kind == CB_SHELL && s->n_frest > 0) {
      if (s->n_frest_pt > 0)
        k_key_shift<<<cb_grid(s->n_frest_pt), CB_THREADS, 0, cb_count(st)>>>(
            bp<uint64_t>(b->frest) + wpt, bp<uint64_t>(s->frest), s->n_frest_pt, (uint32_t)vo, (uint32_t)to);
      const int64_t nee = s->n_frest - s->n_frest_pt;
      if (nee > 0)
        k_key_shift<<<cb_grid(nee), CB_THREADS, 0, cb_count(st)>>>(bp<uint64_t>(b->frest) + wee,
                                                                    bp<uint64_t>(s->frest) + s->n_frest_pt, nee,
                                                                    (uint32_t)eo, (uint32_t)eo);
      wpt += s->n_frest_pt;
      wee += nee;
    }
  }
  if (cudaGetLastError() != cudaSuccess) return fail(CB_ERR_CUDA);
  b->n_frest = b->kind == CB_SHELL ? nf : 0;
  b->n_frest_pt = nf_pt;
  // per-component dbar_min of the members, at the batch's component labels
  // (rods: polyline index + the member's first polyline; shells: vertex id + vertex offset)
  if ((rc = buf_ensure(b->dbar_comp, sizeof(unsigned long long) * (size_t)std::max(1, b->n), st)) != CB_OK)
    return fail(rc);
  for (int m = 0; m < count; ++m) {
    const cb_scene* s = members[m];
    const size_t cnt = b->kind == CB_ROD ? (size_t)s->n_rods : (size_t)s->n;
    const size_t lbl = b->kind == CB_ROD ? (size_t)roff[m] : (size_t)b->voff[m];
    if (cnt && cudaMemcpyAsync(bp<unsigned long long>(b->dbar_comp) + lbl, s->dbar_comp.p,
                               sizeof(unsigned long long) * cnt, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return fail(CB_ERR_CUDA);
  }
  if ((rc = frest_rows_build(b, st)) != CB_OK) return fail(rc);
  for (auto& e : b->ev)
    if (cudaEventCreate(&e) != cudaSuccess) return fail(CB_ERR_CUDA);
  if ((rc = upload_members(b, st)) != CB_OK) return fail(rc);
  if (cudaStreamSynchronize(st) != cudaSuccess) return fail(CB_ERR_CUDA);
  *out = b;
  return CB_OK;
}

cb_status cb_batch_offsets(cb_scene* s, int64_t* vert_offsets, int64_t* edge_offsets, int64_t* tri_offsets) {
  if (!s) return CB_ERR_ARG;
  for (int m = 0; m <= s->count; ++m) {
    if (vert_offsets) vert_offsets[m] = s->voff[m];
    if (edge_offsets) edge_offsets[m] = s->eoff[m];
    if (tri_offsets) tri_offsets[m] = s->toff[m];
  }
  return CB_OK;
}

int32_t cb_member_count(cb_scene* s) { return s ? s->count : 0; }

cb_status cb_scene_destroy(cb_scene* s) {
  if (!s) return CB_ERR_ARG;
  scene_release(s);
  return CB_OK;
}

static void stage_begin(cb_scene* s, int k, cudaStream_t st) {
  if (s->timing) cudaEventRecord(s->ev[2 * k], st);
}
static void stage_end(cb_scene* s, int k, cudaStream_t st) {
  if (s->timing) cudaEventRecord(s->ev[2 * k + 1], st);
}

cb_status contact_build(cb_scene* s, const double* x, void* stream) {
  if (!s || !x) return CB_ERR_ARG;
  AllocScope scope(s->alloc_ptr(), &s->live_bytes);
  cudaStream_t st = (cudaStream_t)stream;
  s->last_stream = st;
  stage_begin(s, 0, st);
  cb_status r = broad_phase(s, s->bw, x, nullptr, false, false, s->cand, &s->n_cand, st);
  stage_end(s, 0, st);
  s->n_active = 0;
  return r;
}

cb_status contact_filter(cb_scene* s, void* stream) {
  if (!s) return CB_ERR_ARG;
  AllocScope scope(s->alloc_ptr(), &s->live_bytes);
  cudaStream_t st = (cudaStream_t)stream;
  s->last_stream = st;
  stage_begin(s, 1, st);
  cb_status r = filter_apply(s, st);
  stage_end(s, 1, st);
  return r;
}

cb_status barrier_eval(cb_scene* s, const double* x, double* energy, double* grad, void* stream) {
  if (!s || !x) return CB_ERR_ARG;
  AllocScope scope(s->alloc_ptr(), &s->live_bytes);
  cudaStream_t st = (cudaStream_t)stream;
  s->last_stream = st;
  stage_begin(s, 2, st);
  cb_status r = barrier_run(s, x, energy, grad, false, st);
  stage_end(s, 2, st);
  return r;
}

cb_status barrier_energy(cb_scene* s, const double* x, double* energy, void* stream) {
  if (!s || !x || !energy) return CB_ERR_ARG;
  AllocScope scope(s->alloc_ptr(), &s->live_bytes);
  cudaStream_t st = (cudaStream_t)stream;
  s->last_stream = st;
  stage_begin(s, 2, st);
  cb_status r = barrier_run(s, x, energy, nullptr, true, st);
  stage_end(s, 2, st);
  return r;
}

cb_status ccd_step(cb_scene* s, const double* x, const double* p, double* alpha, void* stream) {
  if (!s || !x || !p) return CB_ERR_ARG;
  AllocScope scope(s->alloc_ptr(), &s->live_bytes);
  cudaStream_t st = (cudaStream_t)stream;
  s->last_stream = st;
  stage_begin(s, 3, st);
  cb_status r = ccd_run(s, x, p, alpha, st);
  stage_end(s, 3, st);
  return r;
}

cb_status cb_set_tuning(cb_scene* s, int32_t phase, float cell_factor, int32_t pair_block) {
  if (!s || (phase != 0 && phase != 1) || !(cell_factor > 0.0f) || !(cell_factor <= 64.0f)) return CB_ERR_ARG;
  if (pair_block != 64 && pair_block != 128 && pair_block != 256) return CB_ERR_ARG;
  BroadWork& w = phase ? s->bwc : s->bw;
  w.cell_factor = cell_factor;
  w.pair_block = pair_block;
  return CB_OK;
}

cb_status cb_get_tuning(cb_scene* s, int32_t phase, float* cell_factor, int32_t* pair_block) {
  if (!s || (phase != 0 && phase != 1)) return CB_ERR_ARG;
  const BroadWork& w = phase ? s->bwc : s->bw;
  if (cell_factor) *cell_factor = w.cell_factor;
  if (pair_block) *pair_block = w.pair_block;
  return CB_OK;
}

cb_status cb_set_timing(cb_scene* s, int32_t on) {
  if (!s) return CB_ERR_ARG;
  s->timing = on != 0;
  return CB_OK;
}

cb_status cb_get_stage_ms(cb_scene* s, float* ms) {
  if (!s || !ms) return CB_ERR_ARG;
  CB_CUDA(cudaStreamSynchronize(s->last_stream));
  for (int k = 0; k < 4; ++k) {
    ms[k] = 0.f;
    if (s->timing) cudaEventElapsedTime(&ms[k], s->ev[2 * k], s->ev[2 * k + 1]);
  }
  ms[4] = 0.f;
  if (s->timing && s->n_active > 0) cudaEventElapsedTime(&ms[4], s->ev[10], s->ev[11]);
  cudaGetLastError();
  return CB_OK;
}

cb_status cb_get_stage_times(cb_scene* s, float* ms, int32_t count) {
  if (!s || !ms || count < 0) return CB_ERR_ARG;
  float all[7] = {0, 0, 0, 0, 0, 0, 0};
  CB_TRY(cb_get_stage_ms(s, all));
  if (s->timing && s->cd_split) {
    cudaEventElapsedTime(&all[5], s->ev[4], s->ev[12]);
    cudaEventElapsedTime(&all[6], s->ev[12], s->ev[5]);
    cudaGetLastError();
  }
  for (int k = 0; k < count && k < 7; ++k) ms[k] = all[k];
  for (int k = 7; k < count; ++k) ms[k] = 0.f;
  return CB_OK;
}

// Ascending order of 64-bit keys on the host (the pass keeps its pair lists
// in hash-cell order; the getters return them sorted): LSD radix sort of
// (key, original index) with 16-bit digits, skipping digits that are equal
// in every key.  idx (optional) receives the original positions.
static void sort_keys(std::vector<uint64_t>& keys, std::vector<uint32_t>* idx) {
  const size_t n = keys.size();
  std::vector<uint32_t> ix(n), ix2(idx ? n : 0);
  for (size_t i = 0; i < n; ++i) ix[i] = (uint32_t)i;
  if (n < 2) {
    if (idx) idx->swap(ix);
    return;
  }
  uint64_t all_or = 0, all_and = ~0ull;
  for (uint64_t k : keys) {
    all_or |= k;
    all_and &= k;
  }
  const uint64_t varying = all_or & ~all_and;
  std::vector<uint64_t> k2(n);
  std::vector<size_t> cnt(65537);
  for (int sh = 0; sh < 64; sh += 16) {
    if (((varying >> sh) & 0xffffull) == 0) continue;
    std::fill(cnt.begin(), cnt.end(), 0);
    for (size_t i = 0; i < n; ++i) ++cnt[((keys[i] >> sh) & 0xffff) + 1];
    for (size_t d = 1; d < cnt.size(); ++d) cnt[d] += cnt[d - 1];
    for (size_t i = 0; i < n; ++i) {
      const size_t o = cnt[(keys[i] >> sh) & 0xffff]++;
      k2[o] = keys[i];
      if (idx) ix2[o] = ix[i];
    }
    keys.swap(k2);
    if (idx) ix.swap(ix2);
  }
  if (idx) idx->swap(ix);
}

cb_status cb_get_pairs(cb_scene* s, int32_t which, uint64_t* keys, int64_t cap, int64_t* count) {
  if (!s || !count) return CB_ERR_ARG;
  cudaStream_t st = s->last_stream;
  std::vector<uint64_t> k;
  std::vector<uint8_t> c;
  std::vector<uint32_t> ai;
  std::vector<uint64_t> res;
  switch (which) {
    case CB_PAIRS_CANDIDATE: CB_TRY(dl(res, s->cand, s->n_cand, st)); break;
    case CB_PAIRS_FILTERED:
      CB_TRY(dl(k, s->cand, s->n_cand, st));
      CB_TRY(dl(c, s->klass, s->n_cand, st));
      CB_CUDA(cudaStreamSynchronize(st));
      for (size_t i = 0; i < k.size(); ++i)
        if (c[i] == 1) res.push_back(k[i]);
      break;
    case CB_PAIRS_CORE:
      CB_TRY(dl(k, s->cand, s->n_cand, st));
      CB_TRY(dl(c, s->ccls, s->n_cand, st));
      CB_CUDA(cudaStreamSynchronize(st));
      for (size_t i = 0; i < k.size(); ++i)
        if (c[i] == 2) res.push_back(k[i]);
      break;
    case CB_PAIRS_ACTIVE:
      CB_TRY(dl(k, s->cand, s->n_cand, st));
      CB_TRY(dl(ai, s->aidx, s->n_active, st));
      CB_CUDA(cudaStreamSynchronize(st));
      for (uint32_t a : ai) res.push_back(k[a]);
      break;
    case CB_PAIRS_CCD: CB_TRY(dl(res, s->ccd_keys, s->n_ccd, st)); break;
    case CB_PAIRS_REST_FILTERED:
      if (s->kind == CB_SHELL) CB_TRY(dl(res, s->frest, s->n_frest, st));
      break;
    default: return CB_ERR_ARG;
  }
  CB_CUDA(cudaStreamSynchronize(st));
  *count = (int64_t)res.size();
  if ((int64_t)res.size() > cap) return CB_ERR_CAPACITY;
  if (keys && !res.empty()) {
    sort_keys(res, nullptr);
    memcpy(keys, res.data(), res.size() * sizeof(uint64_t));
  }
  return CB_OK;
}

cb_status cb_get_rest_filter(cb_scene* s, uint64_t* keys, double* dbar, int64_t cap, int64_t* count) {
  if (!s || !count || s->kind != CB_SHELL) return CB_ERR_ARG;
  cudaStream_t st = s->last_stream;
  *count = s->n_frest;
  if (s->n_frest > cap) return CB_ERR_CAPACITY;
  if (s->n_frest > 0 && keys)
    CB_CUDA(cudaMemcpyAsync(keys, s->frest.p, sizeof(uint64_t) * (size_t)s->n_frest, cudaMemcpyDeviceToHost, st));
  if (s->n_frest > 0 && dbar)
    CB_CUDA(cudaMemcpyAsync(dbar, s->frest_dbar.p, sizeof(double) * (size_t)s->n_frest, cudaMemcpyDeviceToHost, st));
  CB_CUDA(cudaStreamSynchronize(st));
  return CB_OK;
}

cb_status cb_get_active(cb_scene* s, uint64_t* keys, double* dd, uint8_t* klass, int8_t* dtype, int64_t cap,
                        int64_t* count) {
  if (!s || !count) return CB_ERR_ARG;
  cudaStream_t st = s->last_stream;
  *count = s->n_active;
  if (s->n_active > cap) return CB_ERR_CAPACITY;
  std::vector<uint64_t> k;
  std::vector<uint32_t> ai;
  std::vector<double> d;
  std::vector<uint8_t> c;
  std::vector<int8_t> t;
  CB_TRY(dl(k, s->cand, s->n_cand, st));
  CB_TRY(dl(ai, s->aidx, s->n_active, st));
  CB_TRY(dl(d, s->cd, s->n_cand, st));
  CB_TRY(dl(c, s->ccls, s->n_cand, st));
  CB_TRY(dl(t, s->ctype, s->n_cand, st));
  CB_CUDA(cudaStreamSynchronize(st));
  std::vector<uint64_t> ak(ai.size());
  for (size_t q = 0; q < ai.size(); ++q) ak[q] = k[ai[q]];
  std::vector<uint32_t> order;
  sort_keys(ak, &order);
  for (size_t q = 0; q < ai.size(); ++q) {
    const uint32_t src = ai[order[q]];
    if (keys) keys[q] = ak[q];
    if (dd) dd[q] = d[src];
    if (klass) klass[q] = c[src];
    if (dtype) dtype[q] = t[src];
  }
  return CB_OK;
}

cb_status cb_get_ccd(cb_scene* s, uint64_t* keys, double* t, uint8_t* klass, int64_t cap, int64_t* count) {
  if (!s || !count) return CB_ERR_ARG;
  cudaStream_t st = s->last_stream;
  *count = s->n_ccd;
  if (s->n_ccd > cap) return CB_ERR_CAPACITY;
  if (s->n_ccd) {
    std::vector<uint64_t> k;
    std::vector<double> tt;
    std::vector<uint8_t> cc;
    CB_TRY(dl(k, s->ccd_keys, s->n_ccd, st));
    if (t) CB_TRY(dl(tt, s->ccd_t, s->n_ccd, st));
    if (klass) CB_TRY(dl(cc, s->ccd_cls, s->n_ccd, st));
    CB_CUDA(cudaStreamSynchronize(st));
    std::vector<uint32_t> order;
    sort_keys(k, &order);
    for (size_t q = 0; q < k.size(); ++q) {
      if (keys) keys[q] = k[q];
      if (t) t[q] = tt[order[q]];
      if (klass) klass[q] = cc[order[q]];
    }
  }
  return CB_OK;
}

cb_status cb_get_bsr(cb_scene* s, int32_t* row_ptr, int32_t* col, double* val, int64_t cap, int64_t* nnzb) {
  if (!s || !nnzb) return CB_ERR_ARG;
  cudaStream_t st = s->last_stream;
  *nnzb = s->nnzb;
  if (s->nnzb > cap) return CB_ERR_CAPACITY;
  if (row_ptr) CB_CUDA(cudaMemcpyAsync(row_ptr, s->bsr_row.p, 4 * ((size_t)s->n + 1), cudaMemcpyDeviceToHost, st));
  if (s->nnzb) {
    if (col) CB_CUDA(cudaMemcpyAsync(col, s->bsr_col.p, 4 * (size_t)s->nnzb, cudaMemcpyDeviceToHost, st));
    if (val) CB_CUDA(cudaMemcpyAsync(val, s->bsr_val.p, 72 * (size_t)s->nnzb, cudaMemcpyDeviceToHost, st));
  }
  CB_CUDA(cudaStreamSynchronize(st));
  return CB_OK;
}

cb_status cb_bsr_device(cb_scene* s, const int32_t** row_ptr, const int32_t** col, const double** val,
                        int64_t* nnzb) {
  if (!s) return CB_ERR_ARG;
  if (row_ptr) *row_ptr = (const int32_t*)s->bsr_row.p;
  if (col) *col = (const int32_t*)s->bsr_col.p;
  if (val) *val = (const double*)s->bsr_val.p;
  if (nnzb) *nnzb = s->nnzb;
  return CB_OK;
}

cb_status cb_get_stats(cb_scene* s, cb_stats* o) {
  if (!s || !o) return CB_ERR_ARG;
  uint64_t h[SC_N];
  CB_TRY(read_scalars(s, 0, SC_N, h, s->last_stream));
  memset(o, 0, sizeof(*o));
  o->n_candidates = s->n_cand;
  o->n_filtered = (int64_t)h[SC_NFILT];
  o->n_core = (int64_t)h[SC_NCORE];
  o->n_active = s->n_active;
  o->n_ccd = s->n_ccd;
  o->nnzb = s->nnzb;
  o->n_rest_filtered = s->n_frest;
  o->dbar_min = s->dbar_min;
  o->offset = s->xi;
  o->dhat = s->dhat;
  o->activation = s->a;
  o->status_bits = (int32_t)h[SC_STATUS];
  o->ccd_max_iters = (int32_t)h[SC_ITERS];
  o->n_candidates_fp32 = (int64_t)h[SC_FP32_PAIRS];
  o->n_fp64_decided = (int64_t)h[SC_FP64_DECIDED];
  o->n_hess_face = (int64_t)(uint32_t)h[SC_N9];
  o->n_hess_pe_frame = (int64_t)(uint32_t)h[SC_N4];
  o->n_hess_pe = (int64_t)(uint32_t)h[SC_N6];
  o->n_pair_overflow = (int64_t)(uint32_t)h[SC_NOVF];
  o->n_mollified = (int64_t)(uint32_t)h[SC_NMOLL];
  o->n_stencil_dropped = s->n_dropped;
  o->device_bytes = s->live_bytes;
  return CB_OK;
}

cb_status cb_sync_status(cb_scene* s) {
  if (!s) return CB_ERR_ARG;
  uint64_t h;
  CB_TRY(read_scalars(s, SC_STATUS, 1, &h, s->last_stream));
  uint64_t zero = 0;
  CB_CUDA(cudaMemcpyAsync(scalars(s) + SC_STATUS, &zero, 8, cudaMemcpyHostToDevice, s->last_stream));
  CB_CUDA(cudaStreamSynchronize(s->last_stream));
  if (h & CB_DEV_CAPACITY) return CB_ERR_CAPACITY;
  if (h & CB_DEV_PENETRATION) return CB_ERR_PENETRATION;
  if (h & CB_DEV_ITER_LIMIT) return CB_ERR_ITER_LIMIT;
  return CB_OK;
}

}  // extern "C"
