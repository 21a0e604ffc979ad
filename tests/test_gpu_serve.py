"""Served stream on the GPU: requests that overlap on the device (batched with
whatever else is resident) give the same per-step results as the same
request alone -- the step bound exactly (it decides the trajectory), the
energy within the parity tolerance (atomic summation order)."""
import numpy as np
import pytest

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


def test_served_results_equal_alone():
    from paper_2510_10256_gb300.serve import DeviceEngine, Server, poisson_requests, run_alone
    pool = [S.tiny_shell(1), S.tiny_shell(2, nx=6, thickness=0.3, dhat=0.07), S.pleated_sheet(nx=20),
            S.tiny_rods(1), S.woven_patch(n_warp=2, n_weft=2, nseg=48), S.tiny_rods(4)]
    reqs = poisson_requests(pool, 10, rate=400.0, steps=4, seed=11)
    eng = DeviceEngine()
    eng.calibrate([pool[0], pool[3]])
    rep = Server(eng, hbm_budget=150 << 30, max_slots=6, keep_results=True).run(reqs)
    assert rep["steps"] == 40 and not rep["rejected"]
    assert rep["max_resident"] > 1 and rep["iterations"] < rep["steps"], "requests never overlapped"
    for r in reqs:
        mix = rep["results"][r.rid]
        alone = run_alone(eng, r)
        assert len(mix) == len(alone) == r.steps
        for k, (a, b) in enumerate(zip(mix, alone)):
            assert a.alpha == b.alpha, (r.rid, k, a.alpha, b.alpha)
            assert np.isfinite(a.energy) and np.isfinite(b.energy)
            assert abs(a.energy - b.energy) <= 1e-9 * max(abs(b.energy), 1e-300), (r.rid, k, a.energy, b.energy)
    eng.close()


@pytest.mark.slow
def test_serve_pool_scenes_match_oracle():
    """The served stream's scenes at full size (every rod, and the shells up
    to 80k triangles; the two largest shells would take the brute-force
    oracle minutes each) against the oracle.  Served results equal these
    single-scene results (test above), so this pins the served stream too."""
    from tests.parity import compare, run_gpu
    import oracle as O
    pool = S.serve_pool()
    picked = [sc for sc in pool if sc.kind == "rod" or sc.tris.shape[1] <= 80_000]
    assert sum(sc.kind == "shell" for sc in picked) >= 5
    for sc in picked:
        compare(sc, run_gpu(sc), O.contact_pass(sc))
