"""Pins for the barrier (Eq. 2-3), the distance derivatives and the PSD
projection used by projected Newton."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))


def test_barrier_closed_values():
    g = GOLD["barrier_half_width"]
    b, b1, b2 = O.barrier(g["y"], g["dhat"])
    assert b == pytest.approx(g["b"], rel=1e-15)
    assert b1 == pytest.approx(g["b1"], rel=1e-15)
    assert b2 == pytest.approx(g["b2"], rel=1e-15)


def test_barrier_offset_closed_value():
    # Eq. 3: b(d, a, eta) = b(d - eta, a - eta)
    g = GOLD["barrier_offset"]
    b, _, _ = O.barrier(g["d"] - g["eta"], g["a"] - g["eta"])
    assert b == pytest.approx(g["b"], rel=1e-9)


@pytest.mark.parametrize("dh", [1.0, 0.05, 0.01, 0.3535])
def test_barrier_c2_at_activation(dh):
    assert O.barrier(dh, dh) == (0.0, 0.0, 0.0)
    assert O.barrier(1.5 * dh, dh) == (0.0, 0.0, 0.0)
    # one-sided approach to the activation: all three go to zero
    b, b1, b2 = O.barrier(dh * (1 - 1e-6), dh)
    assert abs(b) < 1e-17 * max(1, dh ** 2) and abs(b1) < 1e-10 and abs(b2) < 1e-4 / dh


@pytest.mark.parametrize("dh", [1.0, 0.05, 0.0123])
def test_barrier_derivatives_fd(dh):
    for y in dh * np.array([0.05, 0.2, 0.5, 0.77, 0.95]):
        h = 1e-6 * dh
        b, b1, b2 = O.barrier(y, dh)
        bp, b1p, _ = O.barrier(y + h, dh)
        bm, b1m, _ = O.barrier(y - h, dh)
        assert b1 == pytest.approx((bp - bm) / (2 * h), rel=1e-6, abs=1e-12)
        assert b2 == pytest.approx((b1p - b1m) / (2 * h), rel=1e-6, abs=1e-9)


def test_barrier_diverges_at_offset():
    vals = [O.barrier(y, 1.0)[0] for y in (1e-2, 1e-4, 1e-8, 1e-16)]
    assert all(b2 > b1 for b1, b2 in zip(vals, vals[1:]))
    assert vals[-1] > 30.0
    assert all(O.barrier(y, 1.0)[1] < 0 for y in (1e-3, 0.5, 0.99))   # repulsive


def _stencil_of_type(is_ee, want, rng, tries=20000):
    for _ in range(tries):
        x = rng.normal(size=12)
        d, ty = O.distance(is_ee, x)
        if ty == want and d > 0.2:
            return x, d
    raise RuntimeError("type not reached")


@pytest.mark.parametrize("is_ee,ty", [(False, t) for t in range(7)] + [(True, t) for t in range(9)])
def test_distance_derivatives_fd(is_ee, ty):
    rng = np.random.default_rng(11 + 17 * ty + 100 * is_ee)
    for _ in range(3):
        x, d = _stencil_of_type(is_ee, ty, rng)
        g, H = O.distance_derivs(is_ee, x, ty)
        L = np.abs(x).max()
        h = 1e-6 * L
        # first derivatives of d from the distance routine itself (type is stable
        # under a tiny step away from region boundaries)
        for i in range(12):
            xp, xm = x.copy(), x.copy()
            xp[i] += h
            xm[i] -= h
            dp, tp = O.distance(is_ee, xp)
            dm, tm = O.distance(is_ee, xm)
            assert tp == ty and tm == ty
            assert g[i] == pytest.approx((dp - dm) / (2 * h), rel=1e-6, abs=1e-8)
            gp, _ = O.distance_derivs(is_ee, xp, ty)
            gm, _ = O.distance_derivs(is_ee, xm, ty)
            fd = (gp - gm) / (2 * h)
            assert np.allclose(H[i], fd, rtol=1e-5, atol=1e-6 * max(1.0, np.abs(H).max()))
        # translation invariance: gradient sums to zero per axis, Hessian rows too
        assert np.allclose(g.reshape(4, 3).sum(0), 0, atol=1e-12)
        assert np.allclose(H.reshape(12, 4, 3).sum(1), 0, atol=1e-9 * max(1.0, np.abs(H).max()))
        assert np.allclose(H, H.T, atol=1e-12 * max(1.0, np.abs(H).max()))


@pytest.mark.parametrize("seed", range(20))
def test_psd_projection_vs_eigh(seed):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(12, 12))
    A = A + A.T
    if seed % 3 == 0:
        A[:, :3] = 0.0
        A[:3, :] = 0.0                        # rank-deficient, like PP/PE stencils
    P, ev, sweeps = O.psd_project(A)
    w, V = np.linalg.eigh(A)
    ref = (V * np.maximum(w, 0)) @ V.T
    scale = np.abs(A).max()
    assert np.abs(P - ref).max() <= 1e-12 * scale * 12
    assert np.sort(ev) == pytest.approx(w, abs=1e-12 * scale * 12)
    assert sweeps < 50
    # idempotent and PSD
    P2, _, _ = O.psd_project(P)
    assert np.abs(P2 - P).max() <= 1e-12 * scale * 12
    assert np.linalg.eigvalsh(P).min() >= -1e-12 * scale * 12


def test_psd_projection_keeps_psd_input():
    rng = np.random.default_rng(5)
    B = rng.normal(size=(12, 6))
    A = B @ B.T
    P, _, _ = O.psd_project(A)
    assert np.abs(P - A).max() <= 1e-13 * np.abs(A).max() * 12


def test_psd_projection_of_barrier_hessian():
    """H = b'' grad grad^T + b' hess(d) of a real stencil is indefinite (b' < 0,
    hess(d) PSD for point-point), and the projection clamps exactly the negative
    part: for point-point it leaves b'' grad grad^T."""
    x = np.array([0, 0, 0, 0.3, 0.1, 0.05, 5, 5, 5, 6, 5, 5.0])   # PP(p, t0) region
    d, ty = O.distance(False, x)
    assert ty == 0
    g, Hd = O.distance_derivs(False, x, ty)
    b, b1, b2 = O.barrier(d - 0.0, 0.5)
    H = b2 * np.outer(g, g) + b1 * Hd
    P, ev, _ = O.psd_project(H)
    assert ev.min() < 0
    assert np.allclose(P, b2 * np.outer(g, g), atol=1e-12 * np.abs(H).max())
