"""Kaldor culling (CB_FILTER_KALDOR) on the GPU against the oracle: the same
candidate, culled and CCD sets, barrier, gradient, Hessian and step bound;
and the negative control of Invariant 3 on the hairpin (culling leaves the
step unbounded, the filter does not)."""
import numpy as np
import pytest

import oracle as O
from paper_2510_10256_gb300 import scenes as S
from tests.parity import compare, run_gpu
from tests.test_oracle_kaldor import hairpin

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_10256_gb300 import contact
    contact.build()
    contact.lib()


@pytest.mark.parametrize("case", ["woven", "rods", "hairpin", "straight"])
@pytest.mark.parametrize("radius", [5, 11])
def test_kaldor_matches_oracle(case, radius):
    sc = {"woven": lambda: S.woven_patch(n_warp=2, n_weft=2, nseg=48),
          "rods": lambda: S.tiny_rods(3),
          "hairpin": lambda: hairpin(push=0.35),
          "straight": lambda: S.straight_rod(n_seg=30, seg=0.1, thickness=0.25, dhat=0.05)}[case]()
    g = run_gpu(sc, mode="kaldor", cull_radius=radius)
    o = O.contact_pass(sc, mode="kaldor", cull_radius=radius)
    compare(sc, g, o, mode="off")
    culled_o = o.ccd_keys[o.ccd_klass == O.KLASS_X]
    culled_g = g["ccd"]["keys"][(g["ccd"]["klass"] & 0x7F) == O.KLASS_X]
    assert np.array_equal(np.sort(culled_g), np.sort(culled_o))
    if case in ("hairpin", "straight"):
        assert culled_o.size > 0


def test_kaldor_negative_control_on_gpu():
    sc = hairpin(push=0.35)
    kal = run_gpu(sc, mode="kaldor", cull_radius=11)
    fil = run_gpu(sc)
    assert kal["alpha"] == 1.0 and fil["alpha"] < 0.9


def test_kaldor_rejects_shells_and_zero_radius():
    from paper_2510_10256_gb300.contact import ContactError, ContactScene
    sh = S.tiny_shell(1)
    with pytest.raises(ContactError):
        ContactScene.from_scene(sh, mode="kaldor", cull_radius=5)
    rod = S.tiny_rods(1)
    with pytest.raises(ContactError):
        ContactScene.from_scene(rod, mode="kaldor", cull_radius=0)
