"""Per-stencil activation on the GPU (CB_PER_STENCIL, the extension Sec. 3.3
leaves for later) against the oracle's contact_pass(per_stencil=True): a
filtered candidate stays a candidate only if its FP64 boxes, inflated by
half its own width, overlap.  Candidate, filtered and active sets bit-exact,
numerics within the parity tolerance; dropping those pairs changes no value
of the pass (they are farther apart than their width)."""
import numpy as np
import pytest

import oracle as O
from paper_2510_10256_gb300 import scenes as S
from tests.parity import compare, run_gpu, run_gpu_batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_10256_gb300 import contact
    contact.build()
    contact.lib()


CASES = [lambda: S.pleated_sheet(nx=48), lambda: S.woven_patch(n_warp=3, n_weft=3, nseg=64),
         lambda: S.tiny_shell(4, nx=6), lambda: S.graded_disk(target_tris=6000, L0=0.5),
         lambda: S.ring_chain(n_rings=12, m=48)]


@pytest.mark.parametrize("make", CASES)
@pytest.mark.parametrize("per_component", [False, True])
def test_per_stencil_matches_the_oracle(make, per_component):
    sc = make()
    g = run_gpu(sc, per_stencil=True, per_component=per_component)
    o = O.contact_pass(sc, per_stencil=True, per_component=per_component)
    rep = compare(sc, g, o)
    full = O.contact_pass(sc, per_component=per_component, ccd=False)
    dropped = full.C.size - o.C.size
    assert g["stats"]["n_stencil_dropped"] == dropped and dropped > 0
    assert rep["C"] == g["stats"]["n_candidates"]
    # the same barrier as the full activation: energy, active set, gradient
    assert np.array_equal(o.active_keys, full.active_keys)
    assert abs(g["energy"] - full.energy) <= 1e-9 * max(abs(full.energy), 1e-300)


def test_per_stencil_batch_equals_its_members():
    scenes = [S.pleated_sheet(nx=24), S.tiny_shell(5, nx=6), S.graded_disk(target_tris=3000, L0=0.5)]
    res = run_gpu_batch(scenes, per_stencil=True)
    for sc, g in zip(scenes, res):
        compare(sc, g, O.contact_pass(sc, per_stencil=True))
