"""Pins for the oracle's paper-literal thickness mapping (activation a = h,
offset eta = h - dhat; Sec. 3.1 places the activation at the thickness h,
Sec. 3.3 splits it as eta + dhat, Eq. 1 / Eq. 4).

Each pin is fixed by the paper's formulas or by closed forms, not by the
oracle itself: the straight-rod filtered set at activation h, the Eq. 2 barrier
of a skew perpendicular edge pair at its known distance with the offset
h - dhat, class C (Sec. 3.4) at the shifted offset, the CCD offset of an
unfiltered pair, and the flat rest shell's zero energy.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2510_10256_gb300 import scenes as S


def _b(y, dh):
    """Eq. 2: b(y, dhat) = -(y - dhat)^2 ln(y / dhat) for 0 < y < dhat."""
    return -(y - dh) ** 2 * math.log(y / dh) if 0.0 < y < dh else 0.0


def test_offsets_mapping():
    sc = S.straight_rod(thickness=0.27, dhat=0.05)
    assert O.offsets(sc) == (0.27, 0.05)
    xi, dh = O.offsets(sc, paper_literal=True)
    assert xi == 0.27 - 0.05 and dh == 0.05
    with pytest.raises(ValueError):
        O.offsets(S.straight_rod(thickness=0.01, dhat=0.05), paper_literal=True)


def test_straight_rod_filter_at_activation_h():
    """Straight rod of segment L = 0.1: edges k < l are filtered iff
    l - k >= 2 and (l - k - 1) L < a.  With h = 0.27, dhat = 0.05 the
    paper-literal activation 0.27 keeps index gaps 2 and 3; the default
    activation 0.32 also keeps gap 4."""
    n = 20
    for literal, max_gap in ((True, 3), (False, 4)):
        sc = S.straight_rod(n_seg=n, seg=0.1, thickness=0.27, dhat=0.05)
        r = O.contact_pass(sc, paper_literal=literal)
        _, k, l = O.key_parts(r.F_rest)
        expect = {(a, b) for a in range(n) for b in range(a + 2, n) if b - a <= max_gap}
        assert set(zip(k.tolist(), l.tolist())) == expect
        assert r.dbar_min == pytest.approx(0.1, rel=1e-12)
        # the straight rod at rest: filtered pairs sit at or beyond their width
        assert r.energy == 0.0


def _crossing(D, h, dhat):
    """Two perpendicular rods, each of 2 segments, crossing at height D: the
    middle segments' edge-edge distance is D (interior type)."""
    x = np.array([[-0.05, 0.0, 0.05, 0.0, 0.0, 0.0],
                  [0.0, 0.0, 0.0, -0.05, 0.0, 0.05],
                  [0.0, 0.0, 0.0, D, D, D]])
    rp = np.array([0, 3, 6], np.int32)
    return S.Scene("rod", x.copy(), x.copy(), np.zeros_like(x), h, dhat, rod_ptr=rp, name="crossing")


@pytest.mark.parametrize("D", [0.195, 0.1995, 0.205])
def test_crossing_barrier_closed_form(D):
    """Eq. 2 at the closed-form distance D of two crossing rods (4 edge pairs
    all at distance D: the two edges of each rod meet at the crossing).

    Paper-literal: eta = h - dhat = 0.19, dhat = 0.01, so an unfiltered pair
    at D = 0.195 has y = 0.005 and energy b(0.005, 0.01) per pair; the default
    mapping puts it inside the offset 0.2, so class C (Sec. 3.4: eta
    temporarily 0) with width a = 0.21 and energy b(D, 0.21).  At D = 0.205
    the literal activation 0.2 leaves no candidate, the default one gives
    b(0.005, 0.01)."""
    h, dhat = 0.2, 0.01
    sc = _crossing(D, h, dhat)
    for literal in (True, False):
        xi = h - dhat if literal else h
        a = xi + dhat
        if D - xi <= 0.0:
            per_pair, klass = _b(D, a), O.KLASS_C
        else:
            per_pair, klass = _b(D - xi, dhat), O.KLASS_U
        r = O.contact_pass(sc, paper_literal=literal, ccd=False)
        if D > a:
            # the boxes, inflated by a/2 each, are D - a apart along z: no candidate
            assert r.C.size == 0 and r.energy == 0.0
            continue
        assert r.C.size == 4
        assert np.all(r.klass == klass)
        assert np.allclose(r.d, D, rtol=1e-14)
        assert r.energy == pytest.approx(4 * per_pair, rel=1e-12, abs=1e-300)
        assert (r.energy > 0.0) == (per_pair > 0.0)


def test_ccd_offset_is_the_literal_offset():
    """Head-on approach of the crossing rods (speed 1 along -z from D = 0.3):
    an unfiltered pair keeps the offset eta, so the additive-CCD bound is
    below (D - eta) / 1 and within the factor (1 - s) of it after the first
    step.  Paper-literal eta = 0.19, default eta = 0.2."""
    h, dhat, D = 0.2, 0.01, 0.3
    sc = _crossing(D, h, dhat)
    p = np.zeros_like(sc.x)
    p[2, 3:] = -1.0
    for literal in (True, False):
        eta = h - dhat if literal else h
        r = O.contact_pass(sc, paper_literal=literal, p=p)
        toi = D - eta
        assert r.alpha < toi
        assert r.alpha >= (1.0 - O.ACCD_S) * toi * (1.0 - 1e-12)
        xe = sc.x + r.alpha * p
        # no unfiltered pair ends inside the offset
        d = [O.distance(True, np.concatenate([xe[:, a], xe[:, a + 1], xe[:, b], xe[:, b + 1]]))[0]
             for a in (0, 1) for b in (3, 4)]
        assert min(d) > eta


def test_flat_grid_rest_energy_zero_literal():
    """Invariant 2 under the literal mapping: at the flat rest every stencil
    neighbour closer than the activation (now h) is filtered with width
    dbar_min = L / sqrt 2 and sits at or beyond it; with the filter off the
    rest energy is positive (contact locking, Fig. 2)."""
    sc = S.flat_grid(nx=7, L=0.5, thickness=1.0, dhat=0.05)
    r = O.contact_pass(sc, paper_literal=True, ccd=False)
    assert r.energy == 0.0 and r.dbar_min == pytest.approx(0.5 / math.sqrt(2.0), rel=1e-14)
    off = O.contact_pass(sc, paper_literal=True, mode="off", ccd=False)
    assert off.energy > 0.0
    # the literal activation is smaller, so it filters fewer stencil pairs
    dflt = O.contact_pass(sc, ccd=False)
    assert set(r.F_rest.tolist()) < set(dflt.F_rest.tolist())
