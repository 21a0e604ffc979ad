"""High-precision evidence for the gradient / Hessian tolerance floor.

The parity tolerance of a gradient or BSR entry is 1e-9 times its scale: the
sum over contributing pairs of max(|contribution|, f_p x the pair's largest
entry), f_p = max(1e-4, 5e-7 kappa_p), kappa_p = max(1, d / (dhat_p - y)).
The kappa term exists because near the activation the barrier's derivatives
(Eq. 2, evaluated at y = d - xi_p: b' ~ (dhat - y)^2, b'' ~ (dhat - y)) turn
a relative rounding u of the computed distance d into relative errors of
about 2 u kappa_p in the pair's gradient and u kappa_p in its Hessian; the
floor's 5e-7 covers about one ulp of d (2.2e-16) on either side of a
comparison, times the gradient's 2 kappa_p.  These tests pin that reading
against a 40-digit reference that differentiates the whole pair energy
kappa b(d(x) - xi, dhat) numerically in mpmath (no chain rule, no typed
distance derivatives) and projects with mpmath's symmetric eigensolver:

* the oracle's FP64 gradient, Hessian and PSD projection of one pair agree
  with the reference within the tolerance, from y / (dhat - y) = 1 up to
  1e7 (kappa_p up to 2e8);
* the floor is not wider than FP64 needs: relative to the pair's largest
  entry, the oracle's own gradient error reaches a good fraction of what the
  floor grants once kappa_p >= 2e5, and so does the change of the exact
  gradient when d moves by one unit in its last place -- while the fixed
  floor alone (1e-13 of the pair norm) would reject both.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2510_10256_gb300 import scenes as S

mp = pytest.importorskip("mpmath").mp

XI, DHAT = 0.2, 0.01


def _rotation(seed):
    rng = np.random.default_rng(seed)
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    return q * np.sign(np.diag(r))


def _scene(kind, kap, seed):
    """One stencil pair at y = dhat kap / (1 + kap) beyond the offset (so
    y / (dhat - y) = kap), in a random orientation; coordinates rounded to
    FP64 (the exact distance of the rounded points is what the reference
    uses).  kind 'ee': two single-segment rods crossing; 'pt': a point over
    a triangle's interior."""
    y = DHAT * kap / (1.0 + kap)
    D = XI + y
    R = _rotation(seed)
    c = np.array([0.3, -0.2, 0.1])
    if kind == "ee":
        P = np.array([[-0.07, 0.0, 0.0], [0.05, 0.01, 0.0], [0.01, -0.06, D], [-0.02, 0.08, D]])
        x = (P @ R.T + c).T.copy()
        return S.Scene("rod", x.copy(), x.copy(), np.zeros_like(x), XI, DHAT,
                       rod_ptr=np.array([0, 2, 4], np.int32), name="ee_pair")
    P = np.array([[0.01, 0.02, D], [-0.1, -0.1, 0.0], [0.12, -0.08, 0.0], [-0.01, 0.13, 0.0],
                  [0.5, 0.5, 3.0]])
    x = (P @ R.T + c).T.copy()
    # a lone point (vertex 0) over a triangle (1, 2, 3); vertex 4 is a far-away
    # single triangle corner so the point has a triangle of its own
    tris = np.array([[1, 0, 4], [2, 4, 0], [3, 4, 4]], np.int32)
    tris = np.array([[1], [2], [3]], np.int32)
    return S.Scene("shell", x.copy(), x.copy(), np.zeros_like(x), XI, DHAT, tris=tris, name="pt_pair")


def _mp_energy(kind, X):
    """kappa b(d - xi, dhat) of the pair at mp coordinates X (12 values:
    4 points), d the interior distance (the type the oracle reports)."""
    p = [mp.matrix(X[3 * k:3 * k + 3]) for k in range(4)]

    def cross(a, b):
        return mp.matrix([a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]])

    def dot(a, b):
        return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]
    if kind == "ee":
        n = cross(p[1] - p[0], p[3] - p[2])
        d = abs(dot(p[2] - p[0], n)) / mp.sqrt(dot(n, n))
    else:
        n = cross(p[2] - p[1], p[3] - p[1])
        d = abs(dot(p[0] - p[1], n)) / mp.sqrt(dot(n, n))
    y = d - XI
    dh = mp.mpf(DHAT)
    return -(y - dh) ** 2 * mp.log(y / dh), d


def _reference(kind, x12):
    """Gradient, Hessian and PSD-projected Hessian of the pair energy, 40
    digits, by numerical differentiation at 60 working digits."""
    with mp.workdps(60):
        X = [mp.mpf(float(v)) for v in x12]
        f = lambda *v: _mp_energy(kind, list(v))[0]
        g = [mp.diff(f, X, tuple(1 if k == i else 0 for k in range(12))) for i in range(12)]
        H = mp.matrix(12, 12)
        for i in range(12):
            for j in range(i, 12):
                o = [0] * 12
                o[i] += 1
                o[j] += 1
                H[i, j] = H[j, i] = mp.diff(f, X, tuple(o))
        ev, Q = mp.eigsy(H)
        Hp = mp.matrix(12, 12)
        for k in range(12):
            if ev[k] > 0:
                for i in range(12):
                    for j in range(12):
                        Hp[i, j] += ev[k] * Q[i, k] * Q[j, k]
        d = _mp_energy(kind, X)[1]
        cv = lambda M, r, c: np.array([[float(M[i, j]) for j in range(c)] for i in range(r)])
        return np.array([float(v) for v in g]), cv(H, 12, 12), cv(Hp, 12, 12), d


def _oracle(sc, project):
    r = O.contact_pass(sc, project=project, ccd=False)
    assert r.active.sum() == 1 and r.C.size == 1
    st = O.stencils(O.topology(sc), r.C)[0]
    n = sc.n
    H = np.zeros((12, 12))
    Habs = np.zeros((12, 12))
    for q in range(r.bsr_col.size):
        row = int(np.searchsorted(r.bsr_row_ptr, q, side="right") - 1)
        a, b = list(st).index(row), list(st).index(int(r.bsr_col[q]))
        H[3 * a:3 * a + 3, 3 * b:3 * b + 3] = r.bsr_val[q]
        Habs[3 * a:3 * a + 3, 3 * b:3 * b + 3] = r.bsr_abs[q]
    g = np.array([r.grad[c, st[k]] for k in range(4) for c in range(3)])
    gabs = np.array([r.grad_abs[c, st[k]] for k in range(4) for c in range(3)])
    x12 = np.array([sc.x[c, st[k]] for k in range(4) for c in range(3)])
    return r, g, gabs, H, Habs, x12


def _kappa_d(d):
    return d / (DHAT - (d - XI))


def _floor_factor(kap_d):
    return max(1e-4, 5e-7 * max(1.0, kap_d))


CASES = [(k, s) for k in (1.0, 1e2, 1e4, 7e4, 1e6, 1e7) for s in (3, 11)]


@pytest.mark.parametrize("kind", ["ee", "pt"])
@pytest.mark.parametrize("kap,seed", CASES)
def test_oracle_within_floor_of_high_precision(kind, kap, seed):
    sc = _scene(kind, kap, seed=seed)
    r, g, gabs, H, Habs, x12 = _oracle(sc, project=False)
    assert int(r.dtype[0]) == (8 if kind == "ee" else 6), r.dtype  # interior edge-edge / face
    g_ref, H_ref, Hp_ref, d_ref = _reference(kind, x12)
    d = float(d_ref)
    assert (d - XI) / (DHAT - (d - XI)) == pytest.approx(kap, rel=1e-6)
    # the oracle's own scale is the one the floor defines
    hmax = np.abs(H_ref).max()
    assert np.all(Habs >= _floor_factor(_kappa_d(d)) * hmax * (1 - 1e-6))
    # unprojected Hessian and gradient: within the parity tolerance of the exact values
    assert np.all(np.abs(H - H_ref) <= 1e-9 * Habs + 1e-30), float((np.abs(H - H_ref) / Habs).max())
    assert np.all(np.abs(g - g_ref) <= 1e-9 * gabs + 1e-30), float((np.abs(g - g_ref) / gabs).max())
    # projected Hessian: the same scale (taken before projection)
    r, g, gabs, Hp, Hpabs, _ = _oracle(sc, project=True)
    assert np.all(np.abs(Hp - Hp_ref) <= 1e-9 * Hpabs + 1e-30), float((np.abs(Hp - Hp_ref) / Hpabs).max())


def _ulp_change(kind, x12, d0):
    """max |g(d (1 + u)) - g(d)| over the gradient entries, the second
    primitive moved along the pair's normal by one ulp of d."""
    u = 2.0 ** -52
    P = x12.reshape(4, 3)
    if kind == "ee":
        nrm = np.cross(P[1] - P[0], P[3] - P[2])
        move = [2, 3]
    else:
        nrm = np.cross(P[2] - P[1], P[3] - P[1])
        move = [1, 2, 3]
    nrm /= np.linalg.norm(nrm)
    with mp.workdps(60):
        step = mp.mpf(float(d0)) * u
        X = [mp.mpf(float(v)) for v in x12]
        sgn = 1.0 if float(np.dot(P[move[0]] - P[0], nrm)) < 0 else -1.0
        Xs = list(X)
        for k in move:
            for c in range(3):
                Xs[3 * k + c] = X[3 * k + c] - sgn * step * mp.mpf(float(nrm[c]))
        f = lambda *v: _mp_energy(kind, list(v))[0]
        dg = 0.0
        for i in range(12):
            o = tuple(1 if k == i else 0 for k in range(12))
            dg = max(dg, float(abs(mp.diff(f, Xs, o) - mp.diff(f, X, o))))
    return dg


@pytest.mark.parametrize("kind", ["ee", "pt"])
def test_floor_is_not_wider_than_fp64_needs(kind):
    """Relative to the pair's largest gradient entry, against the tolerance
    the floor grants (1e-9 f_p): (i) the oracle's own FP64 error (largest
    over two geometries) reaches at least a tenth of it at y / (dhat - y) =
    1e4 .. 1e6, and exceeds the fixed floor's 1e-13; (ii) a one-ulp move of
    d changes the exact gradient by between a twentieth of it and all of
    it."""
    for kap in (1e4, 7e4, 1e6):
        worst = 0.0
        for seed in (3, 11):
            sc = _scene(kind, kap, seed=seed)
            _, g, _, _, _, x12 = _oracle(sc, project=False)
            g0, _, _, d0 = _reference(kind, x12)
            gmax = np.abs(g0).max()
            granted = 1e-9 * _floor_factor(_kappa_d(float(d0)))
            err = np.abs(g - g0).max() / gmax
            assert err > 1e-13, (kap, err)
            worst = max(worst, err / granted)
            if seed == 3:
                rel = _ulp_change(kind, x12, d0) / gmax
                assert granted / 20.0 <= rel <= granted, (kap, rel, granted)
        assert worst >= 0.1, (kap, worst)
