"""GPU (through the C ABI) vs the FP64 oracle, element by element."""
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


def _pair(sc, mode="double", **kw):
    g = run_gpu(sc, mode=mode, **kw)
    lit = kw.get("paper_literal", False)
    o = O.contact_pass(sc, mode=mode, core_temp=kw.get("core_temp", True), paper_literal=lit)
    return compare(sc, g, o, mode=mode, paper_literal=lit), g, o


@pytest.mark.parametrize("seed", range(6))
def test_tiny_shells(seed):
    rep, _, _ = _pair(S.tiny_shell(seed))
    assert rep["active"] > 0


@pytest.mark.parametrize("seed", range(6))
def test_tiny_rods(seed):
    rep, _, _ = _pair(S.tiny_rods(seed))
    assert rep["C"] > 0


@pytest.mark.parametrize("mode", ["double", "single", "off"])
def test_modes_shell(mode):
    _pair(S.tiny_shell(3, nx=6), mode=mode)


@pytest.mark.parametrize("mode", ["double", "single", "off"])
def test_modes_rod(mode):
    _pair(S.woven_patch(n_warp=2, n_weft=2, nseg=48), mode=mode)


@pytest.mark.parametrize("make", [lambda: S.woven_patch(n_warp=2, n_weft=2, nseg=48),
                                  lambda: S.tiny_rods(2), lambda: S.tiny_shell(3, nx=6),
                                  lambda: S.pleated_sheet(nx=24)])
@pytest.mark.parametrize("mode", ["double", "single"])
def test_paper_literal_mapping(make, mode):
    """CB_THICK_PAPER_LITERAL (activation = thickness, offset = thickness -
    dhat; Sec. 3.1 / 3.3, Eq. 1 / 4) against the oracle's paper_literal pass:
    a smaller activation changes the candidate, filtered, class-C and active
    sets, the offsets of the barrier and of the CCD step."""
    sc = make()
    rep, g, o = _pair(sc, mode=mode, paper_literal=True)
    st = g["stats"]
    assert st["offset"] == sc.thickness - sc.dhat and st["activation"] == sc.thickness
    assert rep["C"] > 0 and rep["active"] > 0 and rep["bsr_compared"] > 0
    # the default mapping really is different on this scene
    assert not np.array_equal(O.contact_pass(sc, mode=mode, ccd=False).C, o.C)


def test_no_core_temp_reports_penetration():
    sc = S.woven_patch(n_warp=2, n_weft=2, nseg=48)
    g = run_gpu(sc, core_temp=False)
    assert g["status"] == 4 and not np.isfinite(g["energy"])


def test_woven_patch_full():
    """The 16-yarn woven patch (4,112 vertices) in full."""
    rep, g, o = _pair(S.woven_patch())
    assert rep["core"] > 0 and rep["F"] > 0


def test_pleated_sheet_reduced():
    """48 x 48 pleated sheet: several hash tiles, all three classes active."""
    rep, g, o = _pair(S.pleated_sheet(nx=48))
    assert rep["F"] > 0 and rep["active"] > 1000


def test_graded_disk_reduced():
    _pair(S.graded_disk(target_tris=6000, L0=0.5))


def test_flat_rest_no_rest_forces():
    sc = S.flat_grid(nx=20)
    g = run_gpu(sc)
    assert g["energy"] == 0.0 and g["A"]["keys"].size == 0
    g2 = run_gpu(sc, mode="off")
    assert g2["energy"] > 0.0


def test_empty_and_degenerate_inputs():
    import torch
    from paper_2510_10256_gb300.contact import ContactScene, ContactError
    # single triangle: no non-incident pairs at all
    sc = S.Scene("shell", np.array([[0, 1, 0], [0, 0, 1], [0, 0, 0.]]), np.array([[0, 1, 0], [0, 0, 1], [0, 0, 0.]]),
                 np.zeros((3, 3)), 0.1, 0.01, tris=np.array([[0], [1], [2]], np.int32))
    g = run_gpu(sc)
    assert g["C"].size == 0 and g["energy"] == 0.0 and g["alpha"] == 1.0
    # far-apart rods: nothing within reach
    sc = S.tiny_rods(1)
    sc.x = sc.x.copy()
    sc.x[2, : sc.rod_ptr[1]] += 100.0
    g = run_gpu(sc)
    o = O.contact_pass(sc)
    compare(sc, g, o)
    # coincident rest vertices of a stencil -> degenerate
    rest = np.array([[0, 1, 1, 2.0], [0, 0, 0, 0.0], [0, 0, 0, 0.0]])
    with pytest.raises(ContactError):
        ContactScene("rod", rest, 0.5, 0.1, rod_ptr=np.array([0, 4], np.int32))
    # bad topology
    with pytest.raises(ContactError):
        ContactScene("shell", np.zeros((3, 3)), 0.1, 0.01, tris=np.array([[0], [1], [5]], np.int32))


@pytest.mark.parametrize("shift", [(1000.0, -500.0, 300.0), (-3.0e4, 2.0e4, 1.0e4)])
def test_far_from_origin(shift):
    """Coordinates far from the origin stress the FP32 screens (their rounding
    grows with |x|); decisions must still match the FP64 oracle."""
    sc = S.pleated_sheet(nx=24)
    off = np.array(shift)[:, None]
    sc.rest = sc.rest + off
    sc.x = sc.x + off
    _pair(sc)
    sc2 = S.woven_patch(n_warp=2, n_weft=2, nseg=40)
    sc2.rest = sc2.rest + off
    sc2.x = sc2.x + off
    _pair(sc2)


@pytest.mark.slow
def test_pleated_sheet_full_size():
    """The bench workload itself (256 x 256 grid, 130,050 triangles) against the
    full brute-force oracle: every candidate, class, active pair, distance,
    gradient entry, BSR block and the step bound."""
    rep, g, o = _pair(S.pleated_sheet())
    print("pleated 256x256", rep)
    assert rep["C"] > 10_000_000 and rep["active"] > 500_000
    # the BSR was compared, all but the blocks of tie-band pairs
    assert rep["bsr_compared"] > 1_000_000 and rep["bsr_blocks_skipped"] <= 1e-4 * rep["nnzb"], rep


@pytest.mark.slow
def test_graded_disk_full_size():
    """Graded twisted disk (~200k triangles, 0.1-4 mm edges) against the full
    oracle."""
    rep, g, o = _pair(S.graded_disk())
    print("graded disk", rep)
    assert rep["F"] > 0
    assert rep["bsr_compared"] > 0 and rep["bsr_blocks_skipped"] <= 1e-4 * rep["nnzb"], rep


@pytest.mark.parametrize("factor,block", [(0.5, 128), (2.0, 64), (32.0, 128)])
def test_tuning_knobs_change_nothing(factor, block):
    """The broad-phase knobs the autotuner sets change speed only: every set
    and value still matches the oracle.  At 32x the mean primitive extent a
    cell holds most of the sheet, so entries' partner ranges run to
    thousands of tests laid end to end across many warps."""
    import torch
    from paper_2510_10256_gb300.contact import ContactScene
    sc = S.pleated_sheet(nx=32)
    o = O.contact_pass(sc)
    dev = torch.device("cuda:0")
    cs = ContactScene.from_scene(sc)
    for ph in (0, 1):
        cs.set_tuning(ph, factor, block)
        assert cs.tuning(ph) == (factor, block)
    x = torch.from_numpy(sc.x).to(dev)
    p = torch.from_numpy(sc.p).to(dev)
    energy = torch.zeros(1, dtype=torch.float64, device=dev)
    grad = torch.zeros(3, sc.n, dtype=torch.float64, device=dev)
    alpha = torch.zeros(1, dtype=torch.float64, device=dev)
    cs.run_pass(x, p, energy, grad, alpha)
    torch.cuda.synchronize()
    g = dict(C=cs.pairs("candidate"), F=cs.pairs("filtered"), CC=cs.pairs("core"), A=cs.active(), ccd=cs.ccd(),
             bsr=cs.bsr(), energy=float(energy.item()), grad=grad.cpu().numpy(), alpha=float(alpha.item()),
             stats=cs.stats(), status=cs.sync_status(), frest=cs.pairs("rest_filtered"))
    cs.close()
    compare(sc, g, o)
    assert g["stats"]["n_pair_overflow"] == 0  # shells never re-test


def test_dense_rod_bundle_overflows_the_pair_stage():
    """200 short parallel rods 0.005 mm apart (thickness 0.1): every edge has
    over a hundred candidate partners, so entries find more pairs than the
    32 the rod broad phase stages and its fill pass re-tests them."""
    n_rods, nseg, seg = 200, 3, 0.05
    pts, rp = [], [0]
    for r in range(n_rods):
        for k in range(nseg + 1):
            pts.append((k * seg, 0.005 * r, 0.0))
        rp.append(len(pts))
    x = np.array(pts, np.float64).T.copy()
    rng = np.random.default_rng(5)
    p = rng.normal(0.0, 0.002, size=x.shape)
    sc = S.Scene("rod", x.copy(), x.copy(), p, 0.1, 0.01, rod_ptr=np.array(rp, np.int32), name="bundle")
    g = run_gpu(sc)
    o = O.contact_pass(sc)
    rep = compare(sc, g, o)
    per_edge = 2.0 * rep["C"] / (n_rods * nseg)
    assert per_edge > 100, per_edge
    assert g["stats"]["n_pair_overflow"] > 0
