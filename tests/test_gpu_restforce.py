"""Rest forces (Fig. 3) on the GPU: exactly zero with the barrier filter at
every resolution and thickness of a small sweep, positive and growing under
refinement without it, and equal to the oracle's."""
import numpy as np
import pytest

import oracle as O
from paper_2510_10256_gb300 import restforce as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_10256_gb300 import contact
    contact.build()
    contact.lib()


def test_rest_force_sweep():
    rows = R.sweep(rod_segments=(20, 40, 80), rod_thickness=(0.13, 0.23), shell_nx=(9, 17, 33),
                   shell_thickness=(0.55, 1.05))
    for r in rows:
        if r["mode"] == "double":
            assert r["energy"] == 0.0 and r["force_max"] == 0.0 and r["active"] == 0, r
            assert r["filtered"] > 0, r
        else:
            assert r["energy"] > 0.0 and r["force_norm"] > 0.0, r
    # refinement at fixed thickness: more neighbours within reach, larger unfiltered force
    for kind, key, ths in (("rod", "segments", (0.13, 0.23)), ("shell", "nx", (0.55, 1.05))):
        for th in ths:
            f = [r["force_norm"] for r in rows if r["kind"] == kind and r["thickness"] == th and r["mode"] == "off"]
            assert all(b > a for a, b in zip(f, f[1:])), (kind, th, f)


@pytest.mark.parametrize("kind", ["rod", "shell"])
def test_rest_force_matches_oracle(kind):
    sc = R.rod_at_rest(40) if kind == "rod" else R.shell_at_rest(17)
    for mode in ("double", "off"):
        g = R.rest_force(sc, mode, keep_grad=True)
        o = O.contact_pass(sc, mode=mode, ccd=False)
        assert abs(g["energy"] - o.energy) <= 1e-9 * max(abs(o.energy), 1e-300), (mode, g["energy"], o.energy)
        # the rest force element by element, within the parity tolerance of each entry
        err = np.abs(g["grad"] - o.grad)
        assert np.all(err <= 1e-9 * o.grad_abs + 1e-30), (mode, float((err / (o.grad_abs + 1e-300)).max()))
        if mode == "double":
            assert np.all(g["grad"] == 0.0) and np.all(o.grad == 0.0)
        else:
            assert np.count_nonzero(o.grad) > 0
