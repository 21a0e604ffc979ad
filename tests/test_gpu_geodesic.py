"""Geodesic reference distances (CB_DBAR_GEODESIC) on the GPU against the
oracle: the rest-filtered set and every pair's dbar on doubly curved sheets
(a dome and a saddle), on a polyhedral cone with a saddle apex whose
shortest paths bend at the apex, and on a sheet rolled onto a cylinder; then
the whole contact pass on the curved sheets.

Tolerances: the key sets are equal; dbar agrees to 1e-12 relative (both
sides unfold the same faces in FP64 but round in different orders, and a
strip crosses at most a few dozen faces)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2510_10256_gb300 import scenes as S
from tests.parity import compare, run_gpu
from tests.test_oracle_geodesic import SADDLE, _cone, _cylinder, _shell

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_10256_gb300 import contact
    contact.build()
    contact.lib()


def _gpu_rest_filter(sc):
    from paper_2510_10256_gb300.contact import ContactScene
    cs = ContactScene.from_scene(sc)
    try:
        keys, dbar = cs.rest_filter()
        dmin = cs.stats()["dbar_min"]
    finally:
        cs.close()
    return keys, dbar, dmin


def _check_rest_filter(sc, min_pairs):
    a = sc.thickness + sc.dhat
    Fo, do = O.rest_filter(sc, O.topology(sc), a)
    Fg, dg, dmin = _gpu_rest_filter(sc)
    assert Fo.size >= min_pairs
    assert np.array_equal(Fg, Fo), (Fg.size, Fo.size)
    rel = np.abs(dg - do) / do
    assert rel.max() <= 1e-12, rel.max()
    assert abs(dmin - do.min()) <= 1e-12 * do.min()
    return Fo, do


@pytest.mark.parametrize("shape", ["dome", "saddle"])
def test_curved_sheet_rest_filter(shape):
    sc = S.curved_sheet(shape=shape)
    F, d = _check_rest_filter(sc, 50_000)
    # the geodesic distances are no shorter than the 3D ones, some strictly longer
    sc.rest_geodesic = False
    Fe, de = O.rest_filter(sc, O.topology(sc), sc.thickness + sc.dhat)
    pos = np.searchsorted(Fe, F)
    assert np.all(Fe[pos] == F) and np.all(d >= de[pos] * (1 - 1e-14)) and np.any(d > de[pos] * (1 + 1e-9))


def test_saddle_apex_paths_bend_at_the_apex():
    rest, tris, alpha, idx = _cone(16, 5, SADDLE)
    # an activation off the sums of integer slant radii: a path through the
    # apex of length exactly a would fall on either side of it by rounding
    sc = _shell(rest, tris, a=5.7)
    F, d = _check_rest_filter(sc, 1000)
    topo = O.topology(sc)
    eid = {(int(a), int(b)): k for k, (a, b) in enumerate(zip(*topo.edges))}
    A, B = eid[(idx(2, 0), idx(2, 1))], eid[(idx(3, 8), idx(3, 9))]
    key = (O.EE << 62) | (min(A, B) << 31) | max(A, B)
    exact = 2 * math.cos(alpha[0] / 2) + 3 * math.cos(alpha[8] / 2)
    k = np.searchsorted(F, np.uint64(key))
    assert F[k] == key and abs(d[k] - exact) <= 1e-13 * exact


def test_rolled_sheet_geodesic_is_its_pattern():
    cyl, pattern, tris, chord = _cylinder(24, 12, 1.5, 0.25, 0.25)
    sc = _shell(cyl, tris, a=0.45)
    F, d = _check_rest_filter(sc, 10_000)
    tw = _shell(pattern, tris, a=0.45, geodesic=False)
    Fp, dp = O.rest_filter(tw, O.topology(tw), 0.45)
    assert np.array_equal(F, Fp) and np.max(np.abs(d - dp) / dp) <= 1e-13


@pytest.mark.parametrize("shape", ["dome", "saddle"])
def test_curved_sheet_pass_matches_oracle(shape):
    sc = S.curved_sheet(shape=shape)
    rep = compare(sc, run_gpu(sc), O.contact_pass(sc))
    assert rep["F"] > 0 and rep["active"] > 0


def test_geodesic_scenes_in_a_batch():
    """Geodesic scenes keep their rest filters when batched with a plain
    shell: each member's pass matches its own oracle."""
    from tests.parity import run_gpu_batch
    scenes = [S.curved_sheet(shape="dome", nx=16), S.curved_sheet(shape="saddle", nx=20, seed=S.BASE_SEED + 10),
              S.tiny_shell(S.BASE_SEED + 11)]
    for sc, g in zip(scenes, run_gpu_batch(scenes)):
        rep = compare(sc, g, O.contact_pass(sc))
        assert rep["C"] > 0


def test_geodesic_with_per_component_widths():
    """CB_DBAR_PER_COMPONENT on geodesic reference distances: each nested
    sheet's filtered pairs take their own component's smallest dbar."""
    sc = S.curved_sheet(shape="saddle", nx=24)
    rep = compare(sc, run_gpu(sc, per_component=True), O.contact_pass(sc, per_component=True))
    assert rep["F"] > 0


def test_l_shaped_sheet_paths_bend_at_the_corner():
    """A flat L-shaped sheet: pairs on either side of the reflex corner are
    as far apart as the path around the corner, on the GPU as in the
    oracle (an activation off the sums of grid distances)."""
    from tests.test_oracle_geodesic import _l_sheet
    rest, tris, _ = _l_sheet(8, 0.1)
    sc = _shell(rest, tris, a=0.3517)
    F, d = _check_rest_filter(sc, 2000)
    sc.rest_geodesic = False
    Fe, de = O.rest_filter(sc, O.topology(sc), 0.3517)
    assert F.size < Fe.size   # pairs across the corner are farther apart on the sheet than in space
