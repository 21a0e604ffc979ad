"""barrier_energy, the line-search call: the energy of barrier_eval (Eq. 2-4)
without its gradient and Hessian kernels.

It must give the energy of the full pass at the pass positions (summation
order aside), the oracle's energy at a trial point along the CCD direction
(after contact_build / contact_filter there), +inf on penetration, and fewer
kernel launches than barrier_eval."""
import numpy as np
import pytest

import oracle as O
from paper_2510_10256_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_10256_gb300 import contact
    contact.build()
    contact.lib()


def _scenes():
    return [S.tiny_shell(1), S.tiny_shell(4, nx=6, thickness=0.3, dhat=0.07), S.pleated_sheet(nx=24),
            S.woven_patch(n_warp=2, n_weft=2, nseg=48), S.tiny_rods(2)]


def _tensors(sc, x=None):
    import torch
    dev = torch.device("cuda:0")
    xx = torch.from_numpy(np.ascontiguousarray(sc.x if x is None else x)).to(dev)
    pp = torch.from_numpy(np.ascontiguousarray(sc.p)).to(dev)
    return xx, pp, torch.zeros(1, dtype=torch.float64, device=dev)


@pytest.mark.parametrize("k", range(5))
def test_energy_only_equals_full_pass(k):
    import torch
    from paper_2510_10256_gb300 import contact
    from paper_2510_10256_gb300.contact import ContactScene
    sc = _scenes()[k]
    cs = ContactScene.from_scene(sc)
    x, p, e_full = _tensors(sc)
    grad = torch.zeros(3, sc.n, dtype=torch.float64, device=x.device)
    cs.contact_build(x)
    cs.contact_filter()
    n0 = contact.kernel_launches()
    cs.barrier_eval(x, e_full, grad)
    n_full = contact.kernel_launches() - n0
    e_only = torch.full((1,), -1.0, dtype=torch.float64, device=x.device)
    n0 = contact.kernel_launches()
    cs.barrier_energy(x, e_only)
    n_only = contact.kernel_launches() - n0
    torch.cuda.synchronize()
    a, b = float(e_only.item()), float(e_full.item())
    assert b > 0.0, "scene should have active pairs"
    assert abs(a - b) <= 1e-12 * abs(b), (a, b)
    assert n_only < n_full, (n_only, n_full)
    orc = O.contact_pass(sc, ccd=False)
    assert abs(a - orc.energy) <= 1e-9 * abs(orc.energy), (a, orc.energy)
    cs.close()


@pytest.mark.parametrize("k", range(5))
def test_energy_at_trial_point_matches_oracle(k):
    """x' = x + t alpha p with t in {0.5, 1}: rebuild and refilter at x', then
    the energy-only pass against the oracle's pass at x'."""
    import torch
    from paper_2510_10256_gb300.contact import ContactScene
    sc = _scenes()[k]
    cs = ContactScene.from_scene(sc)
    x, p, alpha = _tensors(sc)
    cs.contact_build(x)
    cs.contact_filter()
    cs.ccd_step(x, p, alpha)
    torch.cuda.synchronize()
    a = float(alpha.item())
    assert 0.0 < a <= 1.0
    for t in (0.5, 1.0):
        xt = sc.x + t * a * sc.p
        xd, _, e = _tensors(sc, xt)
        cs.contact_build(xd)
        cs.contact_filter()
        cs.barrier_energy(xd, e)
        torch.cuda.synchronize()
        orc = O.contact_pass(sc, x=xt, ccd=False)
        g = float(e.item())
        assert np.isfinite(orc.energy) and np.isfinite(g), (t, g, orc.energy)
        assert abs(g - orc.energy) <= 1e-9 * max(abs(orc.energy), 1e-300), (t, g, orc.energy)
    cs.close()


def test_energy_only_reports_penetration():
    import torch
    from paper_2510_10256_gb300.contact import ContactScene
    sc = S.woven_patch(n_warp=2, n_weft=2, nseg=48)
    cs = ContactScene.from_scene(sc, core_temp=False)
    x, _, e = _tensors(sc)
    cs.contact_build(x)
    cs.contact_filter()
    cs.barrier_energy(x, e)
    torch.cuda.synchronize()
    assert not np.isfinite(float(e.item()))
    assert cs.sync_status() == 4
    cs.close()
