"""Pins of the lagged-friction oracle (oracle/friction.py) against what the
mathematics fixes: the closed forms of f0 / f1, the closest-point weights
against the independent typed distance routine and the orthogonality that
defines a closest point, finite differences of the energy and gradient, and
the invariants of the potential (value eps / 3 per pair and zero gradient at
the lagged state, no change under a rigid translation or a motion along the
normals, PSD Hessians)."""
import numpy as np
import pytest

import oracle as O
import oracle.friction as Fr
from paper_2510_10256_gb300 import scenes as S


def test_f0_f1_closed_forms():
    eps = 0.3
    assert Fr.f0(0.0, eps) == pytest.approx(eps / 3.0, rel=1e-15)
    assert Fr.f0(eps, eps) == pytest.approx(eps, rel=1e-15)     # continuous at eps
    assert Fr.f1(eps, eps) == pytest.approx(1.0, rel=1e-15)     # C^1 at eps
    assert Fr.df1(eps, eps) == 0.0
    assert Fr.f1_over_y(0.0, eps) == pytest.approx(2.0 / eps, rel=1e-15)
    assert Fr.f0(2.0, eps) == 2.0 and Fr.f1(2.0, eps) == 1.0
    h = 1e-6
    for y in (0.01, 0.1, 0.2, 0.29, 0.5, 1.7):
        fd0 = (Fr.f0(y + h, eps) - Fr.f0(y - h, eps)) / (2 * h)
        fd1 = (Fr.f1(y + h, eps) - Fr.f1(y - h, eps)) / (2 * h)
        assert abs(fd0 - Fr.f1(y, eps)) < 1e-8
        assert abs(fd1 - Fr.df1(y, eps)) < 1e-7
        assert Fr.f1_over_y(y, eps) == pytest.approx(Fr.f1(y, eps) / y, rel=1e-14)
    # monotone, and f1 in [0, 1]
    ys = np.linspace(0, 1, 101)
    assert np.all(np.diff(Fr.f0(ys, eps)) > 0)
    assert np.all((Fr.f1(ys, eps) >= 0) & (Fr.f1(ys, eps) <= 1))


@pytest.mark.parametrize("is_ee,types", [(False, range(7)), (True, range(9))])
def test_closest_weights_are_closest_points(is_ee, types):
    """For every type: the weights are affine on each primitive (+1 / -1),
    |w| equals the independent typed distance of the C routine, and w is
    orthogonal to the directions the type leaves free (face, edge or line
    directions) -- the conditions that define the typed closest points."""
    rng = np.random.default_rng(21)
    for _ in range(20):
        X = rng.normal(size=(4, 3))
        for ty in types:
            b = Fr.closest_weights(is_ee, X, ty)
            first = b[:1] if not is_ee else b[:2]
            second = b[1:] if not is_ee else b[2:]
            assert abs(first.sum() - 1.0) < 1e-12 and abs(second.sum() + 1.0) < 1e-12
            w = b @ (X - X[0])
            d_typed = _typed_distance(is_ee, X, ty)
            assert abs(np.linalg.norm(w) - d_typed) <= 1e-12 * max(1.0, d_typed)
            for dvec in _free_directions(is_ee, X, ty):
                assert abs(w @ dvec) <= 1e-11 * np.linalg.norm(dvec) * max(1.0, np.linalg.norm(w))


def _typed_distance(is_ee, X, ty):
    """d of a fixed type from the C routine's gradient: d is translation
    invariant and 1-homogeneous in the coordinates relative to the first
    point, so d = grad d . (x - x0) (Euler)."""
    g, _ = O.distance_derivs(is_ee, X, ty)
    R = (X - X[0]).reshape(-1)
    return float(g @ R)


def _free_directions(is_ee, X, ty):
    if not is_ee:
        p, t0, t1, t2 = X
        if ty in (0, 1, 2):
            return []
        if ty in (3, 4, 5):
            i, j = ((0, 1), (1, 2), (2, 0))[ty - 3]
            return [X[1 + j] - X[1 + i]]
        return [t1 - t0, t2 - t0]
    a0, a1, b0, b1 = X
    if ty in (0, 1, 2, 3):
        return []
    if ty in (4, 5):
        return [b1 - b0]
    if ty in (6, 7):
        return [a1 - a0]
    return [a1 - a0, b1 - b0]


def test_closest_weights_brute_force_tiny():
    """Face and line-line weights against a brute-force search of the
    parameter plane (grid, then a finer grid around the best point)."""
    rng = np.random.default_rng(4)
    for is_ee, ty in ((False, 6), (True, 8)):
        X = rng.normal(size=(4, 3))
        b = Fr.closest_weights(is_ee, X, ty)
        if not is_ee:
            s_ref = (-b[2], -b[3])
            f = lambda s, t: np.linalg.norm(X[0] - (X[1] + s * (X[2] - X[1]) + t * (X[3] - X[1])))
        else:
            s_ref = (b[1], -b[3])
            f = lambda s, t: np.linalg.norm(X[0] + s * (X[1] - X[0]) - X[2] - t * (X[3] - X[2]))
        c, span = np.array([0.0, 0.0]), 8.0
        for _ in range(12):
            g = np.linspace(-span, span, 41)
            vals = np.array([[f(c[0] + s, c[1] + t) for t in g] for s in g])
            i, j = np.unravel_index(np.argmin(vals), vals.shape)
            c = c + np.array([g[i], g[j]])
            span /= 8.0
        assert np.allclose(c, s_ref, atol=1e-8), (c, s_ref)


@pytest.fixture(scope="module")
def lagged():
    sc = S.tiny_shell(3)
    res = O.contact_pass(sc, ccd=False)
    assert res.active.sum() > 20
    L = Fr.lag(sc, res, sc.x, mu=0.3, eps=2e-3)
    return sc, res, L


def test_lambda_is_the_normal_force(lagged):
    """lambda = -kappa b' at the pair's own offset and width: the pair
    energies of the pass are kappa b at the same parameters, and lambda is
    minus their derivative in d (central differences)."""
    sc, res, L = lagged
    xi_p, dh_p = Fr.active_params(res, sc)
    d = res.d[res.active]
    k = float(sc.kappa)
    for m in range(L.keys.size):
        b, _, _ = O.barrier(d[m] - xi_p[m], dh_p[m])
        assert k * b == pytest.approx(res.pair_energy[m], rel=1e-12, abs=1e-300)
        h = 1e-7 * d[m]
        bp = O.barrier(d[m] + h - xi_p[m], dh_p[m])[0]
        bm = O.barrier(d[m] - h - xi_p[m], dh_p[m])[0]
        assert L.lam[m] == pytest.approx(-k * (bp - bm) / (2 * h), rel=1e-5)
    assert np.all(L.lam > 0)
    # the normal is the unit vector between the closest points, |w| = d
    for m in range(L.keys.size):
        X = sc.x[:, L.st[m]].T
        w = L.beta[m] @ (X - X[0])
        assert abs(np.linalg.norm(w) - d[m]) <= 1e-12 * d[m]


def test_value_and_gradient_at_the_lagged_state(lagged):
    sc, res, L = lagged
    ev = Fr.evaluate(L, sc.x, sc.x)
    assert ev.energy == pytest.approx(float(np.sum(L.mu * L.lam * L.eps / 3.0)), rel=1e-14)
    assert np.all(ev.grad == 0.0)


def test_rigid_translation_and_normal_motion(lagged):
    sc, res, L = lagged
    base = Fr.evaluate(L, sc.x, sc.x).energy
    xt = sc.x + np.array([0.3, -0.2, 0.7])[:, None]
    ev = Fr.evaluate(L, xt, sc.x)
    assert ev.energy == pytest.approx(base, rel=1e-12)
    assert np.max(np.abs(ev.grad)) < 1e-9 * np.max(L.mu * L.lam)
    # one pair alone: moving its first primitive along the normal does not slide
    m = int(np.argmax(L.lam))
    Lk = Fr.FrictionLag(L.keys[m:m + 1], L.st[m:m + 1], L.lam[m:m + 1], L.beta[m:m + 1], L.nrm[m:m + 1],
                        L.mu, L.eps)
    x2 = sc.x.copy()
    first = [0] if L.keys[m] >> np.uint64(62) == np.uint64(O.PT) else [0, 1]
    for a in first:
        x2[:, L.st[m, a]] += 0.01 * L.nrm[m]
    ev2 = Fr.evaluate(Lk, x2, sc.x)
    assert ev2.y[0] < 1e-15 and ev2.energy == pytest.approx(Lk.mu * Lk.lam[0] * Lk.eps / 3.0, rel=1e-12)


def test_gradient_and_hessian_by_finite_differences(lagged):
    """Central differences of the energy along random directions match the
    gradient; of the gradient they match the Hessian product.  The state is
    moved so that pairs sit on both sides of eps (sticking and sliding)."""
    sc, res, L = lagged
    rng = np.random.default_rng(8)
    x = sc.x + rng.normal(0.0, 2e-3, size=sc.x.shape)
    ev = Fr.evaluate(L, x, sc.x)
    assert np.any(ev.y < L.eps) and np.any(ev.y > L.eps)
    h = 1e-7
    for _ in range(4):
        v = rng.normal(size=sc.x.shape)
        ep = Fr.evaluate(L, x + h * v, sc.x)
        em = Fr.evaluate(L, x - h * v, sc.x)
        fd = (ep.energy - em.energy) / (2 * h)
        an = float(np.sum(ev.grad * v))
        assert abs(fd - an) <= 1e-6 * float(np.sum(np.abs(ev.grad) * np.abs(v))) + 1e-12, (fd, an)
        fdg = (ep.grad - em.grad) / (2 * h)
        Hv = Fr.hessian_matvec(L, ev.Hw, v)
        La = Fr.FrictionLag(L.keys, L.st, L.lam, np.abs(L.beta), L.nrm, L.mu, L.eps)
        scale = Fr.hessian_matvec(La, np.abs(ev.Hw), np.abs(v))   # sum of |terms|
        assert np.all(np.abs(fdg - Hv) <= 1e-5 * scale + 1e-10), np.max(np.abs(fdg - Hv) / (scale + 1e-300))


def test_hessian_is_psd_and_matvec_matches_dense(lagged):
    sc, res, L = lagged
    rng = np.random.default_rng(9)
    x = sc.x + rng.normal(0.0, 2e-3, size=sc.x.shape)
    ev = Fr.evaluate(L, x, sc.x)
    for H in ev.Hw:
        w = np.linalg.eigvalsh(H)
        assert w.min() >= -1e-12 * max(1.0, np.abs(w).max())
        # the normal is a null direction of the tangent Hessian
    for m in range(L.keys.size):
        assert np.linalg.norm(ev.Hw[m] @ L.nrm[m]) <= 1e-12 * max(1.0, np.abs(ev.Hw[m]).max())
    n = sc.n
    Hd = Fr.hessian_dense(L, ev.Hw, n)
    assert np.allclose(Hd, Hd.T, atol=1e-14 * np.abs(Hd).max())
    assert np.linalg.eigvalsh(Hd).min() >= -1e-10 * np.abs(Hd).max()
    v = rng.normal(size=(3, n))
    assert np.allclose(Hd @ v.reshape(-1), Fr.hessian_matvec(L, ev.Hw, v).reshape(-1),
                       atol=1e-12 * np.abs(Hd).max())


def test_sliding_energy_grows_at_rate_mu_lambda(lagged):
    """Past eps the potential is mu lambda y: its derivative in y is the
    Coulomb bound mu lambda."""
    sc, res, L = lagged
    m = int(np.argmax(L.lam))
    Lk = Fr.FrictionLag(L.keys[m:m + 1], L.st[m:m + 1], L.lam[m:m + 1], L.beta[m:m + 1], L.nrm[m:m + 1],
                        L.mu, L.eps)
    t = np.cross(L.nrm[m], [1.0, 0.0, 0.0])
    t /= np.linalg.norm(t)
    first = [0] if L.keys[m] >> np.uint64(62) == np.uint64(O.PT) else [0, 1]
    def energy(s):
        x2 = sc.x.copy()
        for a in first:
            x2[:, L.st[m, a]] += s * t
        return Fr.evaluate(Lk, x2, sc.x).energy
    s0, h = 5 * L.eps, 1e-6
    assert (energy(s0 + h) - energy(s0 - h)) / (2 * h) == pytest.approx(L.mu * L.lam[m], rel=1e-6)
