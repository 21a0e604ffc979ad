"""Pins of the oracle's edge-edge mollifier (IPC's, which the paper's solver
takes with the contact energy, App. A): on two single-edge rods crossing at
angle theta and height h, the pair's energy is m(s) times the plain
barrier's, with s = sin^2(theta) / 1e-3 (c = |e0 x e1|^2 = L^4 sin^2 theta,
eps_x = 1e-3 L^4) and m(s) = (2 - s) s below 1, 1 above; it vanishes for
parallel edges and is continuous at the threshold.  Its gradient and
(unprojected) Hessian match central differences of the energy and the
gradient; point-triangle pairs are untouched."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2510_10256_gb300 import scenes as S

L, H, XI, DH = 1.0, 0.32, 0.3, 0.05


def _cross(theta, h=H, shift=0.0):
    c, s = math.cos(theta), math.sin(theta)
    x = np.array([[-L / 2, L / 2, -L / 2 * c + shift, L / 2 * c + shift],
                  [0.0, 0.0, -L / 2 * s, L / 2 * s],
                  [0.0, 0.0, h, h]])
    return S.Scene("rod", x.copy(), x.copy(), np.zeros_like(x), XI, DH, rod_ptr=np.array([0, 2, 4], np.int32))


def _energies(sc):
    a = O.contact_pass(sc, ccd=False)
    b = O.contact_pass(sc, ccd=False, mollifier=True)
    assert a.active.sum() == 1 and b.active.sum() == 1
    return a.energy, b.energy


@pytest.mark.parametrize("theta", [1e-3, 0.01, 0.02, 0.03, 0.05, 0.2, 1.0])
def test_energy_ratio_closed_form(theta):
    e, em = _energies(_cross(theta))
    s = math.sin(theta) ** 2 / 1e-3
    m = (2.0 - s) * s if s < 1.0 else 1.0
    assert em == pytest.approx(m * e, rel=1e-9)


def test_parallel_edges_have_no_mollified_energy():
    sc = _cross(0.0, shift=0.2)
    e, em = _energies(sc)
    assert e > 0.0 and em == 0.0
    r = O.contact_pass(sc, ccd=False, mollifier=True)
    assert np.all(r.grad == 0.0)


def test_continuous_at_the_threshold():
    th = math.asin(math.sqrt(1e-3))
    below = _energies(_cross(th * (1 - 1e-7)))[1]
    above = _energies(_cross(th * (1 + 1e-7)))[1]
    assert below == pytest.approx(above, rel=1e-5)


def test_gradient_and_hessian_by_finite_differences():
    sc = _cross(0.02, shift=0.05)
    x0 = sc.x.copy()
    rng = np.random.default_rng(2)
    r = O.contact_pass(sc, ccd=False, mollifier=True, project=False)
    Hd = O.bsr_dense(r, sc.n)
    h = 1e-7
    for _ in range(4):
        v = rng.normal(size=x0.shape)
        ep = O.contact_pass(sc, ccd=False, mollifier=True, x=x0 + h * v).energy
        em = O.contact_pass(sc, ccd=False, mollifier=True, x=x0 - h * v).energy
        fd = (ep - em) / (2 * h)
        an = float(np.sum(r.grad * v))
        assert abs(fd - an) <= 1e-6 * float(np.sum(np.abs(r.grad) * np.abs(v))) + 1e-12, (fd, an)
        gp = O.contact_pass(sc, ccd=False, mollifier=True, project=False, x=x0 + h * v).grad
        gm = O.contact_pass(sc, ccd=False, mollifier=True, project=False, x=x0 - h * v).grad
        # bsr_dense is vertex-major (index 3 v + c); gradients are (3, n)
        fdg = ((gp - gm) / (2 * h)).T.reshape(-1)
        vv = v.T.reshape(-1)
        Hv = Hd @ vv
        scale = np.abs(Hd) @ np.abs(vv)
        assert np.all(np.abs(fdg - Hv) <= 1e-5 * scale + 1e-9), np.max(np.abs(fdg - Hv) / (scale + 1e-300))


def test_point_triangle_pairs_untouched_and_projected_psd():
    sc = S.tiny_shell(3)
    a = O.contact_pass(sc, ccd=False)
    b = O.contact_pass(sc, ccd=False, mollifier=True)
    keys = a.C[a.active]
    t, _, _ = O.key_parts(keys)
    pt = t == O.PT
    assert pt.any()
    assert np.array_equal(a.pair_energy[pt], b.pair_energy[pt])
    thr = O.mollifier_thresholds(sc, O.topology(sc), keys)
    assert np.all(thr[pt] == 0.0) and np.all(thr[~pt] > 0.0)
    # every pair's mollified energy is at most the plain one (0 <= m <= 1)
    assert np.all(b.pair_energy <= a.pair_energy * (1 + 1e-12) + 1e-300)
    Hd = O.bsr_dense(b, sc.n)
    assert np.linalg.eigvalsh(0.5 * (Hd + Hd.T)).min() >= -1e-9 * np.abs(Hd).max()
