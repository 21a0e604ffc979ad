"""Per-component dbar_min (CB_DBAR_PER_COMPONENT) on the GPU against the
oracle: two yarns of different segment lengths and a two-layer shell with
different edge lengths per layer, at rest and compressed (where the coarse
component's filtered pairs switch on at its own width), single scenes and a
batch."""
import numpy as np
import pytest

import oracle as O
from paper_2510_10256_gb300 import scenes as S
from tests.parity import compare, run_gpu
from tests.test_oracle_kaldor import two_yarns

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_10256_gb300 import contact
    contact.build()
    contact.lib()


def two_layers(nx1=9, L1=0.3, nx2=6, L2=0.55, gap=3.0, thickness=0.6, dhat=0.05):
    """Two flat grids (separate components), 3 mm apart, of edge lengths L1, L2."""
    r1, t1 = S.grid_mesh(nx1, nx1, L1)
    r2, t2 = S.grid_mesh(nx2, nx2, L2)
    r2 = r2.copy()
    r2[2] += gap
    rest = np.concatenate([r1, r2], axis=1)
    tris = np.concatenate([t1, t2 + r1.shape[1]], axis=1).astype(np.int32)
    return S.Scene("shell", rest.copy(), rest.copy(), np.zeros_like(rest), thickness, dhat, tris=tris)


def _compressed(sc, first_of_second, f=0.8):
    x = sc.x.copy()
    c = x[:2, first_of_second:].mean(axis=1, keepdims=True)
    x[:2, first_of_second:] = c + f * (x[:2, first_of_second:] - c)
    return x


@pytest.mark.parametrize("kind", ["rod", "shell"])
def test_per_component_matches_oracle(kind):
    sc = two_yarns() if kind == "rod" else two_layers()
    split = 31 if kind == "rod" else 81
    for x in (sc.x, _compressed(sc, split, 0.85 if kind == "rod" else 0.8)):
        p = np.zeros_like(x)
        p[2, split:] = -0.05
        o = O.contact_pass(sc, x=x, p=p, per_component=True)
        g = run_gpu(sc, x=x, p=p, per_component=True)
        compare(sc, g, o)
    og = O.contact_pass(sc, x=x, p=p)
    assert o.energy > og.energy  # the coarse component's own, wider width


def test_per_component_batch_equals_single_scenes():
    import torch
    from paper_2510_10256_gb300.contact import ContactBatch, ContactScene
    dev = torch.device("cuda:0")
    scs = [two_yarns(), two_yarns(L1=0.05, L2=0.08, n1=20, n2=16)]
    xs = [_compressed(scs[0], 31, 0.85), _compressed(scs[1], 21, 0.9)]
    singles = []
    for sc, x in zip(scs, xs):
        g = run_gpu(sc, x=x, per_component=True)
        singles.append(g["energy"])
    members = [ContactScene.from_scene(sc, per_component=True) for sc in scs]
    b = ContactBatch(members)
    xb = torch.from_numpy(np.ascontiguousarray(np.concatenate(xs, axis=1))).to(dev)
    pb = torch.zeros_like(xb)
    e = torch.zeros(2, dtype=torch.float64, device=dev)
    gr = torch.zeros_like(xb)
    a = torch.zeros(2, dtype=torch.float64, device=dev)
    b.run_pass(xb, pb, e, gr, a)
    torch.cuda.synchronize()
    for k in range(2):
        assert abs(float(e[k].item()) - singles[k]) <= 1e-9 * max(abs(singles[k]), 1e-300)
    b.close()
    for m in members:
        m.close()
