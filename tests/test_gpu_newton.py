"""The BSR product and the contact-only Newton driver on the GPU.

cb_bsr_spmv against the assembled matrix read back on the host; the driver
pushes one shell layer into another (and crossing yarns together) through
the target term and must keep every iterate penetration-free (the CCD bound
and the energy-only line search), decrease Phi monotonically, and end where
the GPU's gradient equals the oracle's."""
import numpy as np
import pytest

import oracle as O
from paper_2510_10256_gb300 import scenes as S
from tests.parity import compare, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_10256_gb300 import contact
    contact.build()
    contact.lib()


@pytest.mark.parametrize("shift", [0.0, 7.5])
def test_bsr_spmv_matches_assembled_matrix(shift):
    import torch
    from paper_2510_10256_gb300.contact import ContactScene
    sc = S.pleated_sheet(nx=24)
    cs = ContactScene.from_scene(sc)
    dev = torch.device("cuda:0")
    x = torch.from_numpy(np.ascontiguousarray(sc.x)).to(dev)
    e = torch.zeros(1, dtype=torch.float64, device=dev)
    g = torch.zeros(3, sc.n, dtype=torch.float64, device=dev)
    cs.contact_build(x)
    cs.contact_filter()
    cs.barrier_eval(x, e, g)
    rp, col, val = cs.bsr()
    assert col.size > 0
    rng = np.random.default_rng(7)
    v = rng.normal(size=(3, sc.n))
    # host product: rows of 3x3 blocks on the [n][3] interleaving of v
    vi = v.T.copy()
    yi = shift * vi
    for r in range(sc.n):
        for k in range(rp[r], rp[r + 1]):
            yi[r] += val[k].reshape(3, 3) @ vi[col[k]]
    vd = torch.from_numpy(v).to(dev)
    yd = torch.empty_like(vd)
    cs.bsr_spmv(vd, yd, shift)
    y = yd.cpu().numpy().T
    scale = np.abs(yi).max()
    assert np.abs(y - yi).max() <= 1e-12 * scale
    cs.close()


def _push_case(kind):
    if kind == "shell":
        sc = S.tiny_shell(1)
        target = sc.x.copy()
        top = np.arange(sc.n) >= sc.n // 2
        target[2, top] -= 1.5 * sc.thickness
        return sc, target, 0.05
    sc = S.woven_patch(n_warp=2, n_weft=2, nseg=48)
    target = sc.x.copy()
    target[2] *= 0.0  # flatten the weave: crossing yarns pushed into each other
    return sc, target, 0.05


@pytest.mark.parametrize("kind", ["shell", "rod"])
def test_newton_driver_stays_penetration_free(kind):
    import torch
    from paper_2510_10256_gb300.contact import ContactScene
    from paper_2510_10256_gb300.newton import minimize
    sc, target, h = _push_case(kind)
    cs = ContactScene.from_scene(sc)
    dev = torch.device("cuda:0")
    x0 = torch.from_numpy(np.ascontiguousarray(sc.x)).to(dev)
    xt = torch.from_numpy(np.ascontiguousarray(target)).to(dev)
    x, hist = minimize(cs, x0, xt, h, tol=1e-6, max_iters=40)
    print(kind, [(round(it.phi, 6), round(it.grad_norm, 6), round(it.alpha_max, 4), it.cg_iters) for it in hist])
    assert len(hist) >= 3
    phis = [it.phi for it in hist]
    assert all(np.isfinite(phis))
    assert all(b <= a * (1 + 1e-12) + 1e-12 for a, b in zip(phis, phis[1:])), phis
    assert all(0.0 < it.alpha <= it.alpha_max <= 1.0 for it in hist if it.alpha > 0)
    assert max(it.active for it in hist) > 0, "the push should reach contact"
    # barrier Newton from a deep push: the first steps are CCD-limited, then
    # full steps; a 20x smaller gradient within 40 iterations
    assert hist[-1].grad_norm < 0.05 * hist[0].grad_norm, [it.grad_norm for it in hist]
    assert cs.sync_status() == 0
    xf = x.cpu().numpy()
    # the end point against the oracle: no penetration, same pass results
    o = O.contact_pass(sc, x=xf, p=np.zeros_like(xf))
    assert np.isfinite(o.energy) and not o.penetration
    compare(sc, run_gpu(sc, x=xf, p=np.zeros_like(xf)), o)
    cs.close()
