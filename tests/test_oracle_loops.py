"""Pins of the oracle on closed yarn loops (rods whose last vertex joins the
first): the closing edge, the reference distance the shorter way round the
loop, and Kaldor gaps that wrap.  On a regular m-gon of edge length l every
count and distance has a closed form: two edges whose index gap the short
way round is g (2 <= g <= m/2) are (g - 1) l apart along the loop, and
there are m such pairs for g < m/2 (m/2 for g = m/2)."""
import math

import numpy as np

import oracle as O
from paper_2510_10256_gb300 import scenes as S


def _edge_len(m, R=1.0):
    return 2.0 * R * math.sin(math.pi / m)


def test_closing_edge_and_loop_sizes():
    sc = S.polygon_loop(12)
    t = O.topology(sc)
    assert t.edges.shape[1] == 12
    assert tuple(t.edges[:, -1]) == (11, 0)
    assert np.all(t.loop_ne == 12)
    o = S.polygon_loop(12, closed=False)
    to = O.topology(o)
    assert to.edges.shape[1] == 11 and np.all(to.loop_ne == 0)


def _expected_counts(m, l, a):
    total = 0
    for g in range(2, m // 2 + 1):
        if (g - 1) * l < a:
            total += m // 2 if (m % 2 == 0 and g == m // 2) else m
    return total


def test_regular_polygon_filter_closed_form():
    for m, thick in ((24, 0.3), (25, 0.6), (40, 0.45)):
        sc = S.polygon_loop(m, thickness=thick)
        a = sc.thickness + sc.dhat
        l = _edge_len(m)
        # keep every (g - 1) l away from the threshold, so rounding cannot decide
        assert min(abs((g - 1) * l - a) for g in range(2, m // 2 + 1)) > 1e-9
        t = O.topology(sc)
        F, dbar = O.rest_filter(sc, t, a)
        assert F.size == _expected_counts(m, l, a)
        i = ((F >> np.uint64(31)) & np.uint64(0x7FFFFFFF)).astype(np.int64)
        j = (F & np.uint64(0x7FFFFFFF)).astype(np.int64)
        g = np.minimum(j - i, m - (j - i))
        assert np.allclose(dbar, (g - 1) * l, rtol=1e-12, atol=1e-14)
        assert abs(dbar.min() - l) < 1e-12
        # rotational symmetry: every edge has the same number of filtered partners
        deg = np.bincount(np.concatenate([i, j]), minlength=m)
        assert np.all(deg == deg[0])
        # pairs across the seam (index gap the long way > m/2) are filtered the short way round
        assert np.any(j - i > m // 2)


def test_open_polyline_has_no_seam_pairs():
    m = 24
    sc = S.polygon_loop(m, closed=False)
    a = sc.thickness + sc.dhat
    F, dbar = O.rest_filter(sc, O.topology(sc), a)
    i = ((F >> np.uint64(31)) & np.uint64(0x7FFFFFFF)).astype(np.int64)
    j = (F & np.uint64(0x7FFFFFFF)).astype(np.int64)
    l = _edge_len(m)
    assert np.allclose(dbar, (j - i - 1) * l, rtol=1e-12, atol=1e-14)
    assert np.all((j - i - 1) * l < a)
    closed = S.polygon_loop(m)
    Fc, _ = O.rest_filter(closed, O.topology(closed), a)
    assert set(F.tolist()) < set(Fc.tolist())


def test_kaldor_gap_wraps_on_loops():
    m, R = 30, 4
    sc = S.polygon_loop(m)
    t = O.topology(sc)
    k, l = np.triu_indices(m, 1)
    inc = (np.abs(l - k) == 1) | ((k == 0) & (l == m - 1))
    keys = (k[~inc].astype(np.uint64) << np.uint64(31)) | l[~inc].astype(np.uint64)
    culled = O.kaldor_culled(t, keys, R)
    # short-way gaps 2..R, m pairs each
    assert culled.sum() == m * (R - 1)
    g = np.minimum(l[~inc] - k[~inc], m - (l[~inc] - k[~inc]))
    assert np.array_equal(culled, g <= R)


def test_ring_chain_pass_is_consistent():
    """The chain's pass: the filtered set is exactly the rest filter's within
    the candidates, no penetration, and contacts between linked rings."""
    sc = S.ring_chain()
    r = O.contact_pass(sc)
    assert not r.penetration
    t = O.topology(sc)
    act = r.C[r.active]
    st = O.stencils(t, act)
    cross = t.comp[st[:, 0]] != t.comp[st[:, 2]]
    assert cross.sum() > 0
    assert np.array_equal(r.keys_of(O.KLASS_F), np.intersect1d(r.C, r.F_rest))
    assert abs(r.dbar_min - _edge_len(48)) < 1e-12
    assert r.alpha < 1.0
