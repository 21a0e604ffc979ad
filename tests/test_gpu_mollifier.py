"""IPC's edge-edge mollifier on the GPU (CB_EE_MOLLIFIER) against the oracle
(contact_pass(mollifier=True)): two crossing edges below, at and above the
threshold and parallel ones, a pleated sheet (its stacked layers hold many
near-parallel edge pairs of every distance type), a bundle of nearly
parallel rods, and the energy-only pass against the full pass."""
import math

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


def _cross(theta, shift=0.0):
    c, s = math.cos(theta), math.sin(theta)
    x = np.array([[-0.5, 0.5, -0.5 * c + shift, 0.5 * c + shift], [0.0, 0.0, -0.5 * s, 0.5 * s],
                  [0.0, 0.0, 0.32, 0.32]])
    return S.Scene("rod", x.copy(), x.copy(), np.zeros_like(x), 0.3, 0.05, rod_ptr=np.array([0, 2, 4], np.int32))


@pytest.mark.parametrize("theta,shift", [(0.01, 0.05), (0.02, 0.3), (0.03, 0.0), (0.2, 0.0), (0.0, 0.2)])
def test_crossing_edges_match_oracle(theta, shift):
    sc = _cross(theta, shift)
    o = O.contact_pass(sc, mollifier=True)
    rep = compare(sc, run_gpu(sc, mollifier=True), o)
    assert rep["active"] == 1


def _bundle(n_rods=6, nseg=8, seed=4):
    """Nearly parallel rods 0.31 apart (thickness 0.3): tilts of a few
    hundredths of a radian put many edge pairs below the threshold."""
    rng = np.random.default_rng(seed)
    pts, rp = [], [0]
    for r in range(n_rods):
        th = rng.uniform(0.0, 0.04)
        for k in range(nseg + 1):
            u = -0.5 + k / nseg
            pts.append((u * math.cos(th), u * math.sin(th) + rng.normal(0.0, 1e-3), 0.31 * r))
        rp.append(len(pts))
    x = np.array(pts).T.copy()
    p = rng.normal(0.0, 0.02, size=x.shape)
    return S.Scene("rod", x.copy(), x.copy(), p, 0.3, 0.05, rod_ptr=np.array(rp, np.int32))


@pytest.mark.parametrize("name", ["pleated", "bundle"])
def test_scenes_match_oracle(name):
    sc = S.pleated_sheet(nx=24) if name == "pleated" else _bundle()
    o = O.contact_pass(sc, mollifier=True)
    plain = O.contact_pass(sc)
    assert o.energy < plain.energy  # some edge-edge pairs are below their threshold
    compare(sc, run_gpu(sc, mollifier=True), o)


def test_energy_only_pass_matches_full_pass():
    import torch
    from paper_2510_10256_gb300.contact import ContactScene
    sc = S.pleated_sheet(nx=24)
    dev = torch.device("cuda:0")
    cs = ContactScene.from_scene(sc, mollifier=True)
    x = torch.from_numpy(np.ascontiguousarray(sc.x)).to(dev)
    e_full = torch.zeros(1, dtype=torch.float64, device=dev)
    e_only = torch.zeros(1, dtype=torch.float64, device=dev)
    cs.contact_build(x)
    cs.contact_filter()
    cs.barrier_eval(x, e_full, torch.zeros_like(x))
    cs.barrier_energy(x, e_only)
    torch.cuda.synchronize()
    a, b = float(e_full.item()), float(e_only.item())
    assert abs(a - b) <= 1e-12 * abs(a)
    assert abs(a - O.contact_pass(sc, ccd=False, mollifier=True).energy) <= 1e-9 * abs(a)
    cs.close()
