// server.cu -- serving entry points of the C ABI: a set of resident scenes of
// one kind, admitted into slots under a device-memory budget, advanced
// together by one batched pass (one launch sequence per stage for all of
// them), and the pre-sizing of a scene's pass buffers.  Host orchestration
// only: the pass itself is the batch's four stage calls.
#include <algorithm>
#include <cstring>
#include <vector>

#include "scene.cuh"

struct cb_server {
  int kind = CB_SHELL;
  int slots = 0;
  int64_t budget = 0;
  cb_allocator allocator{};
  bool has_alloc = false;
  std::vector<cb_scene*> resident;   // per slot (nullptr: free)
  cb_scene* batch = nullptr;         // the batch over the resident scenes, in slot order
  std::vector<int> members;          // slots of the batch's members, in member order
  bool stale = true;                 // membership changed since the batch was built
  DevBuf x, p, energy, grad, alpha;  // the batch's concatenated pass buffers
  int64_t live_bytes = 0;            // device bytes of those buffers
  cudaStream_t last_stream = nullptr;
  const cb_allocator* alloc_ptr() const { return has_alloc ? &allocator : nullptr; }
};

namespace {

// device memory the server is charged now: every resident scene, the batch
// and the pass buffers
int64_t charged_bytes(const cb_server* sv) {
  int64_t b = sv->live_bytes;
  for (const cb_scene* s : sv->resident)
    if (s) b += s->live_bytes;
  if (sv->batch && !sv->stale) b += sv->batch->live_bytes;
  return b;
}

void drop_batch(cb_server* sv) {
  if (sv->batch) {
    cb_scene_destroy(sv->batch);
    sv->batch = nullptr;
  }
  sv->members.clear();
}

}  // namespace

cb_status cb_server_create(int32_t kind, int32_t slots, int64_t hbm_budget_bytes, const cb_allocator* allocator,
                           cb_server** out) {
  if (!out || (kind != CB_ROD && kind != CB_SHELL) || slots < 1 || hbm_budget_bytes < 0) return CB_ERR_ARG;
  if (allocator && (!allocator->alloc || !allocator->free)) return CB_ERR_ARG;
  cb_server* sv = new cb_server();
  sv->kind = kind;
  sv->slots = slots;
  sv->budget = hbm_budget_bytes;
  if (allocator) {
    sv->allocator = *allocator;
    sv->has_alloc = true;
  }
  sv->resident.assign((size_t)slots, nullptr);
  *out = sv;
  return CB_OK;
}

cb_status cb_server_destroy(cb_server* sv) {
  if (!sv) return CB_ERR_ARG;
  drop_batch(sv);
  for (DevBuf* b : {&sv->x, &sv->p, &sv->energy, &sv->grad, &sv->alpha}) buf_free(*b, sv->last_stream);
  delete sv;
  return CB_OK;
}

cb_status cb_batch_admit(cb_server* sv, cb_scene* scene, int32_t* slot) {
  if (!sv || !scene || !slot || scene->count != 1 || scene->kind != sv->kind) return CB_ERR_ARG;
  for (const cb_scene* s : sv->resident)
    if (s == scene) return CB_ERR_ARG;  // already resident
  int free_slot = -1;
  for (int k = 0; k < sv->slots && free_slot < 0; ++k)
    if (!sv->resident[k]) free_slot = k;
  if (free_slot < 0) return CB_ERR_CAPACITY;
  // the scene as it stands, and as much again for its pass buffers and its
  // copy in the batch
  if (charged_bytes(sv) + 2 * scene->live_bytes > sv->budget) return CB_ERR_OOM;
  sv->resident[free_slot] = scene;
  sv->stale = true;
  *slot = free_slot;
  return CB_OK;
}

cb_status cb_batch_release(cb_server* sv, int32_t slot) {
  if (!sv || slot < 0 || slot >= sv->slots || !sv->resident[slot]) return CB_ERR_ARG;
  sv->resident[slot] = nullptr;
  sv->stale = true;
  return CB_OK;
}

cb_status cb_batch_pass(cb_server* sv, const double* const* x, const double* const* p, double* const* energy,
                        double* const* grad, double* const* alpha, void* stream) {
  if (!sv || !x || !p) return CB_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int> order;
  for (int k = 0; k < sv->slots; ++k)
    if (sv->resident[k]) {
      if (!x[k] || !p[k]) return CB_ERR_ARG;
      order.push_back(k);
    }
  if (order.empty()) return CB_OK;
  AllocScope scope(sv->alloc_ptr(), &sv->live_bytes);
  sv->last_stream = st;
  if (sv->stale || !sv->batch) {
    drop_batch(sv);
    std::vector<cb_scene*> ms;
    for (int k : order) ms.push_back(sv->resident[k]);
    CB_TRY(cb_batch_create(ms.data(), (int32_t)ms.size(), sv->alloc_ptr(), stream, &sv->batch));
    sv->members = order;
    sv->stale = false;
  }
  cb_scene* b = sv->batch;
  const int M = b->count;
  const size_t N = (size_t)b->n;
  CB_TRY(buf_ensure(sv->x, sizeof(double) * 3 * std::max<size_t>(N, 1), st));
  CB_TRY(buf_ensure(sv->p, sizeof(double) * 3 * std::max<size_t>(N, 1), st));
  CB_TRY(buf_ensure(sv->grad, sizeof(double) * 3 * std::max<size_t>(N, 1), st));
  CB_TRY(buf_ensure(sv->energy, sizeof(double) * (size_t)M, st));
  CB_TRY(buf_ensure(sv->alpha, sizeof(double) * (size_t)M, st));
  // gather: member m's [3][n_m] rows into the batch's [3][N] at its offset
  for (int m = 0; m < M; ++m) {
    const int k = sv->members[m];
    const size_t nm = (size_t)(b->voff[m + 1] - b->voff[m]), o = (size_t)b->voff[m];
    if (nm == 0) continue;
    CB_CUDA(cudaMemcpy2DAsync(bp<double>(sv->x) + o, N * sizeof(double), x[k], nm * sizeof(double),
                              nm * sizeof(double), 3, cudaMemcpyDeviceToDevice, st));
    CB_CUDA(cudaMemcpy2DAsync(bp<double>(sv->p) + o, N * sizeof(double), p[k], nm * sizeof(double),
                              nm * sizeof(double), 3, cudaMemcpyDeviceToDevice, st));
  }
  CB_TRY(contact_build(b, bp<double>(sv->x), stream));
  CB_TRY(contact_filter(b, stream));
  CB_TRY(barrier_eval(b, bp<double>(sv->x), bp<double>(sv->energy), bp<double>(sv->grad), stream));
  CB_TRY(ccd_step(b, bp<double>(sv->x), bp<double>(sv->p), bp<double>(sv->alpha), stream));
  // scatter the members' results to the caller's buffers
  for (int m = 0; m < M; ++m) {
    const int k = sv->members[m];
    const size_t nm = (size_t)(b->voff[m + 1] - b->voff[m]), o = (size_t)b->voff[m];
    if (energy && energy[k])
      CB_CUDA(cudaMemcpyAsync(energy[k], bp<double>(sv->energy) + m, sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (alpha && alpha[k])
      CB_CUDA(cudaMemcpyAsync(alpha[k], bp<double>(sv->alpha) + m, sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (grad && grad[k] && nm > 0)
      CB_CUDA(cudaMemcpy2DAsync(grad[k], nm * sizeof(double), bp<double>(sv->grad) + o, N * sizeof(double),
                                nm * sizeof(double), 3, cudaMemcpyDeviceToDevice, st));
  }
  return CB_OK;
}

cb_status cb_server_stats(cb_server* sv, int32_t* resident, int64_t* charged_bytes_out, int64_t* n_candidates) {
  if (!sv) return CB_ERR_ARG;
  int r = 0;
  for (const cb_scene* s : sv->resident) r += s != nullptr;
  if (resident) *resident = r;
  if (charged_bytes_out) *charged_bytes_out = charged_bytes(sv);
  if (n_candidates) *n_candidates = sv->batch && !sv->stale ? sv->batch->n_cand : 0;
  return CB_OK;
}

cb_status cb_scene_reserve(cb_scene* s, int64_t n_candidates, int64_t n_ccd, int64_t n_active, void* stream) {
  if (!s || n_candidates < 0 || n_ccd < 0 || n_active < 0) return CB_ERR_ARG;
  if (n_candidates > 0x7fffffffLL || n_ccd > 0x7fffffffLL || n_active > 0x7fffffffLL) return CB_ERR_TOO_LARGE;
  AllocScope scope(s->alloc_ptr(), &s->live_bytes);
  cudaStream_t st = (cudaStream_t)stream;
  s->last_stream = st;
  const size_t nc = (size_t)std::max<int64_t>(1, n_candidates), nq = (size_t)std::max<int64_t>(1, n_ccd),
               na = (size_t)std::max<int64_t>(1, n_active);
  // candidates and their per-pair data (broad phase, filter, stage c)
  CB_TRY(buf_ensure(s->cand, sizeof(uint64_t) * nc, st));
  CB_TRY(buf_ensure(s->klass, nc, st));
  CB_TRY(buf_ensure(s->cd, sizeof(double) * nc, st));
  CB_TRY(buf_ensure(s->ctype, nc, st));
  CB_TRY(buf_ensure(s->ccls, nc, st));
  CB_TRY(buf_ensure(s->cflag, sizeof(uint32_t) * nc, st));
  CB_TRY(buf_ensure(s->cpos, sizeof(uint32_t) * (nc + 1), st));
  CB_TRY(buf_ensure(s->dlist, sizeof(uint32_t) * std::max(nc, nq), st));
  // active pairs (stage d): compaction, BSR pattern keys, Hessian queues
  CB_TRY(buf_ensure(s->aidx, sizeof(uint32_t) * na, st));
  for (int k = 0; k < 2; ++k) CB_TRY(buf_ensure(s->bkey[k], sizeof(uint64_t) * 16 * na, st));
  CB_TRY(buf_ensure(s->bflag, sizeof(uint32_t) * 16 * na, st));
  CB_TRY(buf_ensure(s->bpos, sizeof(uint32_t) * (16 * na + 1), st));
  CB_TRY(buf_ensure(s->horder, sizeof(uint32_t) * na, st));
  CB_TRY(buf_ensure(s->hB9, sizeof(double) * 45 * na, st));
  CB_TRY(buf_ensure(s->hB6, sizeof(double) * 21 * na, st));
  CB_TRY(buf_ensure(s->hB4, sizeof(double) * 19 * na, st));
  CB_TRY(buf_ensure(s->hslot, sizeof(uint32_t) * 3 * na, st));
  // CCD candidates (stage e)
  CB_TRY(buf_ensure(s->ccd_keys, sizeof(uint64_t) * nq, st));
  CB_TRY(buf_ensure(s->ccd_t, sizeof(double) * nq, st));
  CB_TRY(buf_ensure(s->ccd_cls, nq, st));
  CB_TRY(buf_ensure(s->ccd_lb, sizeof(double) * nq, st));
  CB_TRY(buf_ensure(s->ccd_flag, sizeof(unsigned long long) * nq, st));
  CB_TRY(buf_ensure(s->ccd_pos, sizeof(unsigned long long) * (nq + 1), st));
  CB_TRY(buf_ensure(s->ccd_list, sizeof(uint32_t) * nq, st));
  CB_TRY(buf_ensure(s->ccd_ulist, sizeof(uint32_t) * nq, st));
  return CB_OK;
}
