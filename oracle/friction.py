"""Lagged friction on the barrier's active pairs -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
leg may import this module.  It shares no code with the CUDA path.

The paper's solver takes IPC's contact and friction energies (App. A,
Implementation Details); this is IPC's lagged friction potential restated on
the pairs the filtered barrier makes active, in plain FP64 numpy, one pair
at a time.

Lagged quantities, per active pair k at the lagged positions x^t (the
positions of the barrier pass the pairs come from):
  lambda_k  = -kappa b'(d_k - xi_k; dhat_k) >= 0, the pair's normal force
              (b' = db/dy of the barrier of Eq. 2-4 at the pair's own offset
              and width, as the barrier pass uses them)
  beta_k    = the closest-point weights of the pair's distance type:
              w(v) = sum_a beta_a v_a is the first primitive's closest point
              minus the second's (sum_a beta_a = 0)
  n_k       = w(x^t) / |w(x^t)|, the contact normal
At positions x, with the tangent projector P = I - n n^T:
  u_k = P w(x - x^t),  y_k = |u_k|
  D(x) = sum_k mu lambda_k f0(y_k)
  f0(y) = -y^3 / (3 eps^2) + y^2 / eps + eps / 3  for y < eps,  y otherwise
  f1 = f0' = -y^2 / eps^2 + 2 y / eps  for y < eps,  1 otherwise
  grad on point a of pair k:   beta_a mu lambda (f1(y) / y) u
  Hessian block (a, b):        beta_a beta_b H_k,
  H_k = mu lambda ( (f1(y) / y) P + (f1'(y) y - f1(y)) / y^3  u u^T )
H_k has eigenvalues mu lambda f1'(y) along u, mu lambda f1(y) / y across
it in the tangent plane and 0 along n, all >= 0, so it needs no projection.

Pins: tests/test_oracle_friction.py (closed forms, finite differences,
invariants, brute-force closest points).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import KLASS_F, KLASS_U, PT, barrier, key_parts, stencils, topology


def f0(y, eps):
    """Smoothed sliding magnitude: C^1 at eps, f0(0) = eps / 3."""
    y = np.asarray(y, np.float64)
    return np.where(y < eps, -y ** 3 / (3.0 * eps * eps) + y * y / eps + eps / 3.0, y)


def f1(y, eps):
    y = np.asarray(y, np.float64)
    return np.where(y < eps, -y * y / (eps * eps) + 2.0 * y / eps, 1.0)


def f1_over_y(y, eps):
    """f1(y) / y, finite at y = 0 (2 / eps)."""
    y = np.asarray(y, np.float64)
    return np.where(y < eps, 2.0 / eps - y / (eps * eps), 1.0 / np.maximum(y, 1e-300))


def df1(y, eps):
    y = np.asarray(y, np.float64)
    return np.where(y < eps, 2.0 * (eps - y) / (eps * eps), 0.0)


def _seg_param(q, a, b):
    """parameter t of the projection of q onto the line a + t (b - a)"""
    e = b - a
    return float(np.dot(q - a, e) / np.dot(e, e))


def closest_weights(is_ee: bool, x12, type_: int) -> np.ndarray:
    """beta of a stencil (4 points: p, t0, t1, t2 or a0, a1, b0, b1) for its
    distance type (the types of the distance routine: PT 0-2 point-point,
    3-5 point-edge (t0t1, t1t2, t2t0), 6 face; EE 0-3 point-point (a0b0,
    a0b1, a1b0, a1b1), 4-7 point-edge (a0-b, a1-b, b0-a, b1-a), 8 line-line).
    Coordinates are taken relative to the first point."""
    X = np.asarray(x12, np.float64).reshape(4, 3)
    X = X - X[0]
    b = np.zeros(4)
    if not is_ee:
        p, t0, t1, t2 = X
        if type_ in (0, 1, 2):
            b[0], b[1 + type_] = 1.0, -1.0
        elif type_ in (3, 4, 5):
            i, j = ((0, 1), (1, 2), (2, 0))[type_ - 3]
            t = _seg_param(p, X[1 + i], X[1 + j])
            b[0], b[1 + i], b[1 + j] = 1.0, -(1.0 - t), -t
        else:
            u, v, w = t1 - t0, t2 - t0, p - t0
            G = np.array([[u @ u, u @ v], [u @ v, v @ v]])
            s1, s2 = np.linalg.solve(G, np.array([w @ u, w @ v]))
            b[:] = (1.0, -(1.0 - s1 - s2), -s1, -s2)
        return b
    a0, a1, b0, b1 = X
    if type_ in (0, 1, 2, 3):
        ia, ib = ((0, 2), (0, 3), (1, 2), (1, 3))[type_]
        b[ia], b[ib] = 1.0, -1.0
    elif type_ in (4, 5):
        t = _seg_param(X[type_ - 4], b0, b1)
        b[type_ - 4], b[2], b[3] = 1.0, -(1.0 - t), -t
    elif type_ in (6, 7):
        s = _seg_param(X[type_ - 4], a0, a1)
        b[0], b[1], b[type_ - 4] = 1.0 - s, s, -1.0
    else:
        u, v, r = a1 - a0, b1 - b0, b0 - a0
        # a0 + s u - (b0 + t v) orthogonal to u and v
        G = np.array([[u @ u, -(u @ v)], [u @ v, -(v @ v)]])
        s, t = np.linalg.solve(G, np.array([r @ u, r @ v]))
        b[:] = (1.0 - s, s, -(1.0 - t), -t)
    return b


def active_params(res, scene, mode: str = "double"):
    """Offset xi_p and width dhat_p of each active pair of a pass: class U
    keeps (xi, dhat) (Eq. 4), class F has no offset and the width dbar_min
    (its component's when the pass was per component), class C no offset
    and the full activation a; single mode (Eq. 1) has offset 0 and width a
    outside class F."""
    xi, dhat = float(scene.thickness), float(scene.dhat)
    a = xi + dhat
    act = res.active
    kl = res.klass[act]
    fw = res.fwidth[act] if res.fwidth is not None else np.full(kl.size, res.dbar_min)
    single = mode == "single"
    xi_p = np.where((kl == KLASS_U) & (not single), xi, 0.0)
    dh_p = np.where(kl == KLASS_F, fw, np.where((kl == KLASS_U) & (not single), dhat, a))
    return xi_p, dh_p


@dataclass
class FrictionLag:
    keys: np.ndarray     # active keys of the lagged pass, in its order
    st: np.ndarray       # (m, 4) stencil vertices
    lam: np.ndarray      # (m,) normal force
    beta: np.ndarray     # (m, 4) closest-point weights
    nrm: np.ndarray      # (m, 3) contact normal
    mu: float
    eps: float


def lag(scene, res, x_lag, mu: float, eps: float, mode: str = "double", topo=None) -> FrictionLag:
    """Lagged quantities of every active pair of `res` (a pass at x_lag)."""
    topo = topo or topology(scene)
    x = np.asarray(x_lag, np.float64)
    keys = res.C[res.active]
    st = stencils(topo, keys)
    ty, _, _ = key_parts(keys)
    dt = res.dtype[res.active]
    d = res.d[res.active]
    xi_p, dh_p = active_params(res, scene, mode)
    m = keys.size
    lam = np.zeros(m)
    beta = np.zeros((m, 4))
    nrm = np.zeros((m, 3))
    for k in range(m):
        _, b1, _ = barrier(d[k] - xi_p[k], dh_p[k])
        lam[k] = -float(scene.kappa) * b1
        x12 = x[:, st[k]].T
        beta[k] = closest_weights(bool(ty[k] != PT), x12, int(dt[k]))
        w = beta[k] @ (x12 - x12[0])
        nrm[k] = w / np.linalg.norm(w)
    return FrictionLag(keys, st, lam, beta, nrm, float(mu), float(eps))


@dataclass
class FrictionEval:
    energy: float
    pair_energy: np.ndarray   # (m,)
    grad: np.ndarray          # (3, n)
    grad_abs: np.ndarray      # (3, n) sum of |contributions| (tolerance scale)
    Hw: np.ndarray            # (m, 3, 3) per-pair tangent Hessian H_k
    y: np.ndarray             # (m,) sliding magnitude


def evaluate(L: FrictionLag, x, x_lag) -> FrictionEval:
    """Friction energy, gradient and per-pair Hessians at x."""
    x = np.asarray(x, np.float64)
    xl = np.asarray(x_lag, np.float64)
    n = x.shape[1]
    m = L.keys.size
    dx = x - xl
    grad = np.zeros((3, n))
    gabs = np.zeros((3, n))
    Hw = np.zeros((m, 3, 3))
    e = np.zeros(m)
    y = np.zeros(m)
    for k in range(m):
        w = dx[:, L.st[k]] @ L.beta[k]
        nk = L.nrm[k]
        P = np.eye(3) - np.outer(nk, nk)
        u = P @ w
        yk = float(np.linalg.norm(u))
        y[k] = yk
        c = L.mu * L.lam[k]
        e[k] = c * float(f0(yk, L.eps))
        q = float(f1_over_y(yk, L.eps))
        gk = c * q * u
        for a in range(4):
            grad[:, L.st[k, a]] += L.beta[k, a] * gk
            gabs[:, L.st[k, a]] += np.abs(L.beta[k, a] * gk)
        if yk > 0.0:
            coef = (float(df1(yk, L.eps)) * yk - float(f1(yk, L.eps))) / yk ** 3
            Hw[k] = c * (q * P + coef * np.outer(u, u))
        else:
            Hw[k] = c * q * P
    return FrictionEval(float(np.sum(e)), e, grad, gabs, Hw, y)


def hessian_dense(L: FrictionLag, Hw, n: int) -> np.ndarray:
    """The friction Hessian as a dense (3n, 3n) matrix, coordinate-major
    (index c * n + v), for small problems."""
    H = np.zeros((3 * n, 3 * n))
    for k in range(L.keys.size):
        for a in range(4):
            for b in range(4):
                blk = L.beta[k, a] * L.beta[k, b] * Hw[k]
                va, vb = L.st[k, a], L.st[k, b]
                for i in range(3):
                    for j in range(3):
                        H[i * n + va, j * n + vb] += blk[i, j]
    return H


def hessian_matvec(L: FrictionLag, Hw, v) -> np.ndarray:
    """H v for v of shape (3, n), pair by pair."""
    v = np.asarray(v, np.float64)
    out = np.zeros_like(v)
    for k in range(L.keys.size):
        wv = v[:, L.st[k]] @ L.beta[k]
        r = Hw[k] @ wv
        for a in range(4):
            out[:, L.st[k, a]] += L.beta[k, a] * r
    return out
