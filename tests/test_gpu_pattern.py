"""Shells cut from a flat pattern (cb_scene_desc.rest_uv) on the GPU against
the oracle: two coaxial rolled sheets whose reference distances are taken
in the pattern."""
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


def test_rolled_sheets_match_oracle():
    sc = S.rolled_sheet()
    rep = compare(sc, run_gpu(sc), O.contact_pass(sc))
    assert rep["F"] > 0 and rep["active"] > 0
    g = run_gpu(sc)
    assert abs(g["stats"]["dbar_min"] - 0.25 / 2 ** 0.5) <= 1e-15
