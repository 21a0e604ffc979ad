"""Lagged friction on the GPU (friction_lag / friction_eval / friction_spmv)
against the oracle (oracle/friction.py): the lagged pair set bit-exact; each
pair's normal force, closest-point weights and normal; the energy, gradient
and per-pair tangent Hessians at a displaced state with pairs on both sides
of eps; the matrix-free Hessian product; and a Newton run in which friction
holds back a tangential push."""
import numpy as np
import pytest

import oracle as O
import oracle.friction as Fr
from paper_2510_10256_gb300 import scenes as S

pytestmark = pytest.mark.gpu

MU, EPS = 0.4, 2e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_10256_gb300 import contact
    contact.build()
    contact.lib()


def _scene(name):
    return {"tiny_shell": lambda: S.tiny_shell(3),
            "pleated": lambda: S.pleated_sheet(nx=24),
            "woven": lambda: S.woven_patch(n_warp=2, n_weft=2, nseg=48),
            "rods": lambda: S.tiny_rods(2)}[name]()


def _gpu(sc, x1, v):
    import torch
    from paper_2510_10256_gb300.contact import ContactScene
    dev = torch.device("cuda:0")
    cs = ContactScene.from_scene(sc)
    x0 = torch.from_numpy(np.ascontiguousarray(sc.x)).to(dev)
    energy = torch.zeros(1, dtype=torch.float64, device=dev)
    grad = torch.zeros(3, sc.n, dtype=torch.float64, device=dev)
    cs.contact_build(x0)
    cs.contact_filter()
    cs.barrier_eval(x0, energy, grad)
    cs.friction_lag(x0, MU, EPS)
    xt = torch.from_numpy(np.ascontiguousarray(x1)).to(dev)
    e = torch.zeros(1, dtype=torch.float64, device=dev)
    g = torch.zeros(3, sc.n, dtype=torch.float64, device=dev)
    cs.friction_eval(xt, x0, e, g)
    e_only = torch.zeros(1, dtype=torch.float64, device=dev)
    cs.friction_eval(xt, x0, e_only)
    y = torch.zeros(3, sc.n, dtype=torch.float64, device=dev)
    cs.friction_spmv(torch.from_numpy(np.ascontiguousarray(v)).to(dev), y)
    torch.cuda.synchronize()
    out = cs.friction()
    assert cs.sync_status() == 0
    cs.close()
    out.update(energy=float(e.item()), energy_only=float(e_only.item()), grad=g.cpu().numpy(), y=y.cpu().numpy())
    return out


def _pack(H):
    return np.stack([H[:, 0, 0], H[:, 0, 1], H[:, 0, 2], H[:, 1, 1], H[:, 1, 2], H[:, 2, 2]], 1)


@pytest.mark.parametrize("name", ["tiny_shell", "pleated", "woven", "rods"])
def test_friction_matches_oracle(name):
    sc = _scene(name)
    res = O.contact_pass(sc, ccd=False)
    L = Fr.lag(sc, res, sc.x, MU, EPS)
    assert L.keys.size > 10
    rng = np.random.default_rng(17)
    x1 = sc.x + rng.normal(0.0, EPS, size=sc.x.shape)
    v = rng.normal(size=sc.x.shape)
    ev = Fr.evaluate(L, x1, sc.x)
    assert np.any(ev.y < EPS) and np.any(ev.y > EPS)
    g = _gpu(sc, x1, v)
    o = np.argsort(g["keys"])
    assert np.array_equal(g["keys"][o], L.keys), "lagged pair sets differ"
    lam, beta, nrm, hw = g["lam"][o], g["beta"][o], g["nrm"][o], g["hw"][o]
    lmax = float(L.lam.max())
    assert np.all(np.abs(lam - L.lam) <= 1e-9 * np.maximum(np.abs(L.lam), 1e-4 * lmax)), \
        np.max(np.abs(lam - L.lam) / np.maximum(np.abs(L.lam), 1e-4 * lmax))
    assert np.max(np.abs(beta - L.beta)) <= 1e-9
    assert np.max(np.abs(nrm - L.nrm)) <= 1e-9
    assert abs(g["energy"] - ev.energy) <= 1e-9 * ev.energy
    assert abs(g["energy_only"] - g["energy"]) <= 1e-12 * ev.energy
    gmax = float(np.abs(ev.grad).max())
    assert np.all(np.abs(g["grad"] - ev.grad) <= 1e-9 * ev.grad_abs + 1e-15 * gmax), \
        np.max(np.abs(g["grad"] - ev.grad) / (ev.grad_abs + 1e-300))
    hp = _pack(ev.Hw)
    hsc = np.abs(hp).max(axis=1, keepdims=True)
    assert np.all(np.abs(hw - hp) <= 1e-9 * hsc + 1e-300), np.max(np.abs(hw - hp) / (hsc + 1e-300))
    yo = Fr.hessian_matvec(L, ev.Hw, v)
    La = Fr.FrictionLag(L.keys, L.st, L.lam, np.abs(L.beta), L.nrm, L.mu, L.eps)
    ysc = Fr.hessian_matvec(La, np.abs(ev.Hw), np.abs(v))
    assert np.all(np.abs(g["y"] - yo) <= 1e-9 * ysc + 1e-300), np.max(np.abs(g["y"] - yo) / (ysc + 1e-300))


def test_friction_call_order_errors():
    import torch
    from paper_2510_10256_gb300.contact import ContactError, ContactScene
    sc = S.tiny_shell(1)
    dev = torch.device("cuda:0")
    cs = ContactScene.from_scene(sc)
    x0 = torch.from_numpy(np.ascontiguousarray(sc.x)).to(dev)
    e = torch.zeros(1, dtype=torch.float64, device=dev)
    y = torch.zeros_like(x0)
    with pytest.raises(ContactError):
        cs.friction_eval(x0, x0, e)          # before friction_lag
    cs.contact_build(x0)
    cs.contact_filter()
    cs.barrier_eval(x0, e, torch.zeros_like(x0))
    with pytest.raises(ContactError):
        cs.friction_lag(x0, MU, 0.0)          # eps must be > 0
    cs.friction_lag(x0, MU, EPS)
    cs.friction_eval(x0, x0, e)               # energy only: no Hessian kept
    with pytest.raises(ContactError):
        cs.friction_spmv(x0, y)
    cs.friction_eval(x0, x0, e, torch.zeros_like(x0))
    cs.friction_spmv(x0, y)
    torch.cuda.synchronize()
    cs.close()


def test_newton_with_friction_holds_back_a_tangential_push():
    """Two stacked layers pressed together, then the top one pushed
    sideways: with friction it slides less than without, and both solves
    stay penetration-free and converge."""
    import torch
    from paper_2510_10256_gb300.contact import ContactScene
    from paper_2510_10256_gb300.newton import minimize
    sc = S.tiny_shell(1)
    dev = torch.device("cuda:0")
    top = np.arange(sc.n) >= sc.n // 2
    target = sc.x.copy()
    target[2, top] -= 1.5 * sc.thickness
    cs = ContactScene.from_scene(sc)
    x0 = torch.from_numpy(np.ascontiguousarray(sc.x)).to(dev)
    xp, _ = minimize(cs, x0, torch.from_numpy(target).to(dev), 0.05, tol=1e-6, max_iters=40)
    shift = np.zeros_like(target)
    shift[0, top] = 0.1
    xt = xp + torch.from_numpy(shift).to(dev)
    slides = {}
    for mu in (0.0, 0.8):
        x, hist = minimize(cs, xp, xt, 0.05, tol=1e-6, max_iters=40,
                           friction=(mu, 1e-3) if mu > 0 else None)
        assert hist[-1].grad_norm < 0.05 * hist[0].grad_norm, [it.grad_norm for it in hist]
        assert cs.sync_status() == 0
        d = (x - xp).cpu().numpy()
        slides[mu] = float(d[0, top].mean())
        xf = x.cpu().numpy()
        o = O.contact_pass(sc, x=xf, p=np.zeros_like(xf), ccd=False)
        assert np.isfinite(o.energy) and not o.penetration
    print(slides)
    assert slides[0.0] > 0.05
    assert slides[0.8] < 0.9 * slides[0.0], slides
    cs.close()
