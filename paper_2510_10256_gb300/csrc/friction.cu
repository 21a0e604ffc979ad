// friction.cu -- lagged friction on the barrier's active pairs.  The paper's
// solver pairs the contact barrier with IPC's friction (App. A); this is
// IPC's lagged friction potential on the pairs the filtered barrier makes
// active, so the filter's reduced widths carry over to the normal forces.
//
// Lagged, per active pair k of the last barrier_eval (positions x^t):
//   lambda_k = -kappa b'(d_k - xi_p; dhat_p) >= 0      (normal force, Eq. 2-4)
//   beta_k   = closest-point weights of the pair's distance type, so that
//              w(v) = sum_a beta_a v_a is the first primitive's closest point
//              minus the second's
//   n_k      = w(x^t) / |w(x^t)|
// At x:  u = (I - n n^T) w(x - x^t),  y = |u|,  D = sum_k mu lambda f0(y), with
//   f0(y) = -y^3/(3 eps^2) + y^2/eps + eps/3 below eps and y above, f1 = f0';
//   grad on point a:  beta_a mu lambda (f1(y)/y) u
//   Hessian block (a, b):  beta_a beta_b H,
//   H = mu lambda ((f1(y)/y) P + (f1'(y) y - f1(y))/y^3 u u^T),  P = I - n n^T,
// whose eigenvalues (mu lambda f1' along u, mu lambda f1/y across it, 0 along
// n) are all >= 0: no projection.  The Hessian is kept per pair (3x3 H and
// the weights) and applied matrix-free (friction_spmv).
#include <cmath>

#include "pairs.cuh"
#include "scene.cuh"

namespace {

// closest-point weights of a stencil for its distance type, from the
// coordinates R relative to the first point (types as in geometry.cuh)
__device__ void closest_weights(bool ee, int ty, const d3 (&R)[4], double (&b)[4]) {
  b[0] = b[1] = b[2] = b[3] = 0.0;
  auto dot = [](d3 a, d3 c) { return a.x * c.x + a.y * c.y + a.z * c.z; };
  auto dif = [](d3 a, d3 c) { return mk3(a.x - c.x, a.y - c.y, a.z - c.z); };
  if (!ee) {
    if (ty <= 2) {
      b[0] = 1.0;
      b[1 + ty] = -1.0;
    } else if (ty <= 5) {
      const int i = ty == 3 ? 0 : (ty == 4 ? 1 : 2), j = ty == 3 ? 1 : (ty == 4 ? 2 : 0);
      const d3 e = dif(R[1 + j], R[1 + i]);
      const double t = dot(dif(R[0], R[1 + i]), e) / dot(e, e);
      b[0] = 1.0;
      b[1 + i] = -(1.0 - t);
      b[1 + j] = -t;
    } else {
      const d3 u = dif(R[2], R[1]), v = dif(R[3], R[1]), w = dif(R[0], R[1]);
      const double uu = dot(u, u), uv = dot(u, v), vv = dot(v, v), wu = dot(w, u), wv = dot(w, v);
      const double det = uu * vv - uv * uv;
      const double s1 = (wu * vv - wv * uv) / det, s2 = (uu * wv - uv * wu) / det;
      b[0] = 1.0;
      b[1] = -(1.0 - s1 - s2);
      b[2] = -s1;
      b[3] = -s2;
    }
    return;
  }
  if (ty <= 3) {
    b[ty >> 1] = 1.0;
    b[2 + (ty & 1)] = -1.0;
  } else if (ty <= 5) {
    const d3 e = dif(R[3], R[2]);
    const double t = dot(dif(R[ty - 4], R[2]), e) / dot(e, e);
    b[ty - 4] = 1.0;
    b[2] = -(1.0 - t);
    b[3] = -t;
  } else if (ty <= 7) {
    const d3 e = dif(R[1], R[0]);
    const double s = dot(dif(R[ty - 4], R[0]), e) / dot(e, e);
    b[0] = 1.0 - s;
    b[1] = s;
    b[ty - 4] = -1.0;
  } else {
    // a0 + s u - (b0 + t v) orthogonal to u and v
    const d3 u = dif(R[1], R[0]), v = dif(R[3], R[2]), r = dif(R[2], R[0]);
    const double uu = dot(u, u), uv = dot(u, v), vv = dot(v, v), ru = dot(r, u), rv = dot(r, v);
    const double det = uv * uv - uu * vv;
    const double s = (uv * rv - ru * vv) / det, t = (uu * rv - uv * ru) / det;
    b[0] = 1.0 - s;
    b[1] = s;
    b[2] = -(1.0 - t);
    b[3] = -t;
  }
}

struct FricLagArgs {
  int64_t na;
  const uint32_t* __restrict__ aidx;
  const uint64_t* __restrict__ cand;
  const int8_t* __restrict__ ctype;
  const uint8_t* __restrict__ ccls;
  const double* __restrict__ cd;
  const int32_t* __restrict__ ev0;
  const int32_t* __restrict__ ev1;
  const int32_t* __restrict__ tv;
  int T, n;
  const int32_t* __restrict__ vsc;
  const MemberParams* __restrict__ mp;
  const int32_t* __restrict__ comp;
  const unsigned long long* __restrict__ dbar_comp;
  const double* __restrict__ x;
  uint64_t* __restrict__ key;
  int4* __restrict__ stn;
  double* __restrict__ dat;  // [8][na]
};

// one thread per active pair: lambda, beta, n at the lagged positions
__global__ void k_fric_lag(FricLagArgs A) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= A.na) return;
  const uint32_t c = A.aidx[a];
  const uint64_t key = A.cand[c];
  const Stencil s = stencil_of(key, A.ev0, A.ev1, A.tv, A.T);
  const PassParams P = member_pass(A.mp[A.vsc[s.v[0]]]);
  double xi_p, dh_p;
  pair_params(P, A.ccls[c], f_width(P, A.dbar_comp, A.comp, s.v[0]), xi_p, dh_p);
  double b, b1, b2;
  barrier_b012(A.cd[c] - xi_p, dh_p, b, b1, b2);
  const double lam = -P.kappa * b1;
  d3 R[4];
  const d3 X0 = load3(A.x, A.n, s.v[0]);
  for (int i = 0; i < 4; ++i) {
    const d3 X = load3(A.x, A.n, s.v[i]);
    R[i] = mk3(X.x - X0.x, X.y - X0.y, X.z - X0.z);
  }
  double be[4];
  closest_weights(s.ee, A.ctype[c], R, be);
  double wx = 0.0, wy = 0.0, wz = 0.0;
  for (int i = 1; i < 4; ++i) {
    wx += be[i] * R[i].x;
    wy += be[i] * R[i].y;
    wz += be[i] * R[i].z;
  }
  const double ww = wx * wx + wy * wy + wz * wz;
  const double iw = ww > 0.0 ? 1.0 / sqrt(ww) : 0.0;  // no normal (and no friction) at zero distance
  A.key[a] = key;
  A.stn[a] = make_int4(s.v[0], s.v[1], s.v[2], s.v[3]);
  const int64_t m = A.na;
  A.dat[a] = iw > 0.0 ? lam : 0.0;
  for (int i = 0; i < 4; ++i) A.dat[(1 + i) * m + a] = be[i];
  A.dat[5 * m + a] = wx * iw;
  A.dat[6 * m + a] = wy * iw;
  A.dat[7 * m + a] = wz * iw;
}

struct FricEvalArgs {
  int64_t nf;
  int n;
  double mu, eps;
  const int4* __restrict__ stn;
  const double* __restrict__ dat;
  const double* __restrict__ x;
  const double* __restrict__ xl;
  double* __restrict__ energy;  // [1], added to
  double* __restrict__ grad;    // [3][n], added to (null: energy only)
  double* __restrict__ hw;      // [6][nf] (written with the gradient)
};

__device__ __forceinline__ void pair_sliding(const FricEvalArgs& A, int64_t k, int4& v, double (&be)[4], double& c,
                                             double (&nn)[3], double (&u)[3], double& y) {
  const int64_t m = A.nf;
  v = A.stn[k];
  c = A.mu * A.dat[k];
  for (int i = 0; i < 4; ++i) be[i] = A.dat[(1 + i) * m + k];
  for (int j = 0; j < 3; ++j) nn[j] = A.dat[(5 + j) * m + k];
  const int vv[4] = {v.x, v.y, v.z, v.w};
  double w[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 3; ++j) {
      const size_t o = (size_t)j * A.n + vv[i];
      w[j] += be[i] * (A.x[o] - A.xl[o]);
    }
  const double wn = w[0] * nn[0] + w[1] * nn[1] + w[2] * nn[2];
  for (int j = 0; j < 3; ++j) u[j] = w[j] - wn * nn[j];
  y = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
}

// one thread per lagged pair: energy (warp-summed, one atomic per warp),
// gradient scatter and the pair's tangent Hessian
__global__ void k_fric_eval(FricEvalArgs A) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double e = 0.0;
  if (k < A.nf) {
    int4 v;
    double be[4], c, nn[3], u[3], y;
    pair_sliding(A, k, v, be, c, nn, u, y);
    const double eps = A.eps, ie = 1.0 / eps;
    const bool stick = y < eps;
    e = c * (stick ? (-y * y * y * (ie * ie) / 3.0 + y * y * ie + eps / 3.0) : y);
    if (A.grad) {
      const double q = stick ? 2.0 * ie - y * (ie * ie) : 1.0 / y;       // f1(y) / y
      const double k2 = y > 0.0 ? (stick ? -(ie * ie) / y : -1.0 / (y * y * y)) : 0.0;  // (f1' y - f1) / y^3
      const int vv[4] = {v.x, v.y, v.z, v.w};
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 3; ++j) {
          const double g = be[i] * c * q * u[j];
          if (g != 0.0) atomicAdd(&A.grad[(size_t)j * A.n + vv[i]], g);
        }
      // H = c (q (I - n n^T) + k2 u u^T), packed xx xy xz yy yz zz
      const int64_t m = A.nf;
      const int ii[6] = {0, 0, 0, 1, 1, 2}, jj[6] = {0, 1, 2, 1, 2, 2};
      for (int t = 0; t < 6; ++t) {
        const int i = ii[t], j = jj[t];
        A.hw[t * m + k] = c * (q * ((i == j ? 1.0 : 0.0) - nn[i] * nn[j]) + k2 * u[i] * u[j]);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
  if ((threadIdx.x & 31) == 0 && e != 0.0) atomicAdd(A.energy, e);
}

// y += H_f v, one thread per lagged pair: wv = sum_a beta_a v_a, r = H wv,
// y_a += beta_a r
__global__ void k_fric_spmv(int64_t nf, int n, const int4* __restrict__ stn, const double* __restrict__ dat,
                            const double* __restrict__ hw, const double* __restrict__ v, double* __restrict__ y) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nf) return;
  const int4 s = stn[k];
  const int vv[4] = {s.x, s.y, s.z, s.w};
  double be[4];
  for (int i = 0; i < 4; ++i) be[i] = dat[(1 + i) * nf + k];
  double w[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 3; ++j) w[j] += be[i] * v[(size_t)j * n + vv[i]];
  const double h00 = hw[k], h01 = hw[nf + k], h02 = hw[2 * nf + k], h11 = hw[3 * nf + k], h12 = hw[4 * nf + k],
               h22 = hw[5 * nf + k];
  const double r[3] = {h00 * w[0] + h01 * w[1] + h02 * w[2], h01 * w[0] + h11 * w[1] + h12 * w[2],
                       h02 * w[0] + h12 * w[1] + h22 * w[2]};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 3; ++j) {
      const double t = be[i] * r[j];
      if (t != 0.0) atomicAdd(&y[(size_t)j * n + vv[i]], t);
    }
}

}  // namespace

extern "C" cb_status friction_lag(cb_scene* s, const double* x_lag, double mu, double eps, void* stream) {
  if (!s || !x_lag || !(mu >= 0.0) || !(eps > 0.0) || s->count != 1) return CB_ERR_ARG;
  AllocScope scope(s->alloc_ptr(), &s->live_bytes);
  cudaStream_t st = (cudaStream_t)stream;
  s->last_stream = st;
  const int64_t na = s->n_active;
  s->n_fric = na;
  s->fr_mu = mu;
  s->fr_eps = eps;
  s->fr_lagged = true;
  s->fr_hw_valid = false;
  if (na == 0) return CB_OK;
  CB_TRY(buf_ensure(s->fr_key, sizeof(uint64_t) * (size_t)na, st));
  CB_TRY(buf_ensure(s->fr_st, sizeof(int4) * (size_t)na, st));
  CB_TRY(buf_ensure(s->fr_dat, sizeof(double) * 8 * (size_t)na, st));
  CB_TRY(buf_ensure(s->fr_hw, sizeof(double) * 6 * (size_t)na, st));
  FricLagArgs A;
  A.na = na;
  A.aidx = bp<uint32_t>(s->aidx);
  A.cand = bp<uint64_t>(s->cand);
  A.ctype = bp<int8_t>(s->ctype);
  A.ccls = bp<uint8_t>(s->ccls);
  A.cd = bp<double>(s->cd);
  A.ev0 = bp<int32_t>(s->ev0);
  A.ev1 = bp<int32_t>(s->ev1);
  A.tv = bp<int32_t>(s->tv);
  A.T = s->T;
  A.n = s->n;
  A.vsc = bp<int32_t>(s->vsc);
  A.mp = bp<MemberParams>(s->mp);
  A.comp = bp<int32_t>(s->comp);
  A.dbar_comp = bp<unsigned long long>(s->dbar_comp);
  A.x = x_lag;
  A.key = bp<uint64_t>(s->fr_key);
  A.stn = bp<int4>(s->fr_st);
  A.dat = bp<double>(s->fr_dat);
  k_fric_lag<<<cb_grid(na), CB_THREADS, 0, cb_count(st)>>>(A);
  CB_CUDA(cudaGetLastError());
  return CB_OK;
}

extern "C" cb_status friction_eval(cb_scene* s, const double* x, const double* x_lag, double* energy, double* grad,
                                   void* stream) {
  if (!s || !x || !x_lag || !energy || !s->fr_lagged) return CB_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  s->last_stream = st;
  if (s->n_fric == 0) {
    if (grad) s->fr_hw_valid = true;
    return CB_OK;
  }
  FricEvalArgs A;
  A.nf = s->n_fric;
  A.n = s->n;
  A.mu = s->fr_mu;
  A.eps = s->fr_eps;
  A.stn = bp<int4>(s->fr_st);
  A.dat = bp<double>(s->fr_dat);
  A.x = x;
  A.xl = x_lag;
  A.energy = energy;
  A.grad = grad;
  A.hw = bp<double>(s->fr_hw);
  k_fric_eval<<<cb_grid(A.nf), CB_THREADS, 0, cb_count(st)>>>(A);
  CB_CUDA(cudaGetLastError());
  if (grad) s->fr_hw_valid = true;
  return CB_OK;
}

extern "C" cb_status friction_spmv(cb_scene* s, const double* v, double* y, void* stream) {
  if (!s || !v || !y || v == y || !s->fr_hw_valid) return CB_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  s->last_stream = st;
  if (s->n_fric == 0) return CB_OK;
  k_fric_spmv<<<cb_grid(s->n_fric), CB_THREADS, 0, cb_count(st)>>>(s->n_fric, s->n, bp<int4>(s->fr_st),
                                                                    bp<double>(s->fr_dat), bp<double>(s->fr_hw), v,
                                                                    y);
  CB_CUDA(cudaGetLastError());
  return CB_OK;
}

extern "C" cb_status cb_get_friction(cb_scene* s, uint64_t* keys, double* dat, double* hw, int64_t cap,
                                     int64_t* count) {
  if (!s || !count || !s->fr_lagged) return CB_ERR_ARG;
  const int64_t nf = s->n_fric;
  *count = nf;
  if (nf == 0) return CB_OK;
  if ((keys || dat || hw) && cap < nf) return CB_ERR_CAPACITY;
  if (hw && !s->fr_hw_valid) return CB_ERR_ARG;
  cudaStream_t st = s->last_stream;
  if (keys) CB_CUDA(cudaMemcpyAsync(keys, s->fr_key.p, sizeof(uint64_t) * (size_t)nf, cudaMemcpyDeviceToHost, st));
  if (dat) CB_CUDA(cudaMemcpyAsync(dat, s->fr_dat.p, sizeof(double) * 8 * (size_t)nf, cudaMemcpyDeviceToHost, st));
  if (hw) CB_CUDA(cudaMemcpyAsync(hw, s->fr_hw.p, sizeof(double) * 6 * (size_t)nf, cudaMemcpyDeviceToHost, st));
  CB_CUDA(cudaStreamSynchronize(st));
  return CB_OK;
}
