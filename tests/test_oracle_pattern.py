"""Pins of the oracle's reference distances for shells cut from a flat
pattern (scene.rest_uv): the same sheets rolled onto cylinders at rest
filter exactly as the flat pattern does (the distances are taken in the
pattern, Sec. 3.2's 2D rest domain), with dbar_min = L / sqrt(2), the
closest non-incident stencil of a regular grid (a vertex and the opposite
diagonal); taken on the 3D rest shape instead, chords undercut the rolled
surface and dbar_min shrinks."""
import math

import numpy as np

import oracle as O
from paper_2510_10256_gb300 import scenes as S


def _flat_twin(sc):
    uv = np.asarray(sc.rest_uv, np.float64)
    flat = np.vstack([uv, np.zeros((1, uv.shape[1]))])
    return S.Scene("shell", flat.copy(), flat.copy(), np.zeros_like(flat), sc.thickness, sc.dhat, tris=sc.tris)


def test_rolled_sheet_filters_as_its_pattern():
    sc = S.rolled_sheet()
    a = sc.thickness + sc.dhat
    t = O.topology(sc)
    F, dbar = O.rest_filter(sc, t, a)
    tw = _flat_twin(sc)
    F2, dbar2 = O.rest_filter(tw, O.topology(tw), a)
    assert np.array_equal(F, F2) and np.array_equal(dbar, dbar2)
    assert abs(dbar.min() - 0.25 / math.sqrt(2.0)) <= 1e-15


def test_3d_rest_shape_undercuts_the_pattern():
    sc = S.rolled_sheet()
    a = sc.thickness + sc.dhat
    _, dbar_uv = O.rest_filter(sc, O.topology(sc), a)
    sc.rest_uv = None
    _, dbar_3d = O.rest_filter(sc, O.topology(sc), a)
    assert dbar_3d.min() < dbar_uv.min() * (1 - 1e-4)
