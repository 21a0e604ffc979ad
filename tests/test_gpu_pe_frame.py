"""Point-edge pairs are projected in their own frame unless that frame is
ill-conditioned (the point nearly on the edge's line: |w| |u| > 64 |u x w|),
in which case they take the generic 6x6 path.  A rod endpoint hovering at
height h above the middle of a 1 mm edge gives |w| / d = 0.5 / h: h = 0.05
takes the frame path, h = 0.005 the generic one; both against the oracle."""
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


def _hover(h, seed=0):
    a = np.array([[0.0, 1.0, 2.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    b = np.array([[0.5, 0.5, 0.5], [0.0, 1.0, 2.0], [h, 1.0 + h, 2.0 + h]])
    pos = np.concatenate([a, b], axis=1)
    rng = np.random.default_rng(seed)
    p = rng.normal(0.0, 0.002, pos.shape)
    return S.Scene("rod", pos.copy(), pos.copy(), p, 0.2, 0.05, rod_ptr=np.array([0, 3, 6], np.int32),
                   name=f"hover_{h}")


@pytest.mark.parametrize("h", [0.05, 0.005, 0.02, 0.0075])
def test_point_edge_frame_and_fallback_match_oracle(h):
    sc = _hover(h)
    o = O.contact_pass(sc)
    rep = compare(sc, run_gpu(sc), o)
    assert rep["active"] >= 1
    # the hovering endpoint against the first edge is a point-edge pair
    assert np.isin(o.dtype[o.active], [4, 5, 6, 7]).any()
