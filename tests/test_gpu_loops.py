"""Closed yarn loops on the GPU against the oracle: a chain of interlocked
rings (the backward arc-length window across each loop's seam, CCD classes),
Kaldor culling whose gaps wrap, loops inside a batch (the windows offset per
member), and the argument check for a loop of two vertices."""
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


@pytest.mark.parametrize("m,n_rings", [(48, 3), (37, 4)])
def test_ring_chain_matches_oracle(m, n_rings):
    sc = S.ring_chain(m=m, n_rings=n_rings)
    o = O.contact_pass(sc)
    rep = compare(sc, run_gpu(sc), o)
    assert rep["F"] > 0 and rep["active"] > 0


def test_polygon_loop_filter_matches_oracle():
    sc = S.polygon_loop(40, thickness=0.45)
    rng = np.random.default_rng(3)
    sc.x = sc.x + rng.normal(0.0, 0.002, size=sc.x.shape)
    sc.p = rng.normal(0.0, 0.05, size=sc.x.shape)
    compare(sc, run_gpu(sc), O.contact_pass(sc))


def test_kaldor_on_loops_matches_oracle():
    sc = S.ring_chain()
    compare(sc, run_gpu(sc, mode="kaldor", cull_radius=3), O.contact_pass(sc, mode="kaldor", cull_radius=3))


def test_loops_in_a_batch_match_each_oracle():
    scenes = [S.ring_chain(m=40), S.tiny_rods(2), S.ring_chain(seed=5, m=44, n_rings=2)]
    outs = run_gpu_batch(scenes)
    for sc, g in zip(scenes, outs):
        compare(sc, g, O.contact_pass(sc))


def test_two_vertex_loop_is_rejected():
    from paper_2510_10256_gb300.contact import ContactError, ContactScene
    x = np.array([[0.0, 1.0], [0.0, 0.0], [0.0, 0.0]])
    with pytest.raises(ContactError):
        ContactScene("rod", x, 0.1, 0.01, rod_ptr=np.array([0, 2], np.int32), rod_closed=[1])
