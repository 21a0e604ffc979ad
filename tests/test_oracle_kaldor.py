"""Kaldor culling (mode "kaldor"), the comparison the paper runs against its
filter: rod edge pairs of one polyline at most R edges apart are removed from
contact.  Pinned by the closed-form culled set on a straight rod, and used
as the negative control of Invariant 3: on a hairpin whose upper leg is
pushed through the lower one, culling leaves the step unbounded and the
legs end inside each other's thickness, while the filtered model stops the
step with every unfiltered pair outside its offset and no pair intersecting."""
import numpy as np
import pytest

import oracle as O
from paper_2510_10256_gb300 import scenes as S


def hairpin(L=0.1, legs=4, h=0.25, thickness=0.2, dhat=0.01, push=None):
    """Lower leg along +x (legs edges), a vertical turn of height h (2 edges),
    upper leg back along -x at z = h; the push moves the upper leg's
    vertices by -push in z."""
    pts = [(k * L, 0.0, 0.0) for k in range(legs + 1)]
    pts += [(legs * L, 0.0, 0.5 * h), (legs * L, 0.0, h)]
    pts += [((legs - k) * L, 0.0, h) for k in range(1, legs + 1)]
    x = np.array(pts, np.float64).T.copy()
    p = np.zeros_like(x)
    if push is not None:
        p[2, legs + 3:] = -push
    return S.Scene("rod", x.copy(), x.copy(), p, thickness, dhat,
                   rod_ptr=np.array([0, x.shape[1]], np.int32), name="hairpin")


def test_culled_set_closed_form_straight_rod():
    """Straight rod of n segments, every pair overlapping the broad phase
    culled iff its edge gap is at most R (non-incident pairs: gap >= 2)."""
    sc = S.straight_rod(n_seg=30, seg=0.1, thickness=0.25, dhat=0.05)
    for R in (5, 11):
        r = O.contact_pass(sc, mode="kaldor", cull_radius=R, ccd=False)
        i = ((r.C >> np.uint64(31)) & np.uint64(0x7FFFFFFF)).astype(np.int64)
        j = (r.C & np.uint64(0x7FFFFFFF)).astype(np.int64)
        assert np.all(j - i >= 2)
        assert np.array_equal(r.klass == O.KLASS_X, j - i <= R)
        assert not r.active[r.klass == O.KLASS_X].any()
        # the rest of the straight rod locks as in the unfiltered control
        off = O.contact_pass(sc, mode="off", ccd=False)
        assert r.energy < off.energy


def _min_distance(sc, x, cls_model="double"):
    """Per class of the filtered model at x: the smallest distance over the
    candidates (the broad phase at the full activation is a superset of all
    pairs within reach)."""
    r = O.contact_pass(sc, mode=cls_model, x=x, ccd=False)
    out = {}
    for k in (O.KLASS_U, O.KLASS_F, O.KLASS_C):
        m = r.klass == k
        out[k] = float(r.d[m].min()) if m.any() else np.inf
    return out


def test_kaldor_is_the_negative_control_of_invariant_3():
    sc = hairpin(push=0.25 + 0.1)  # through the lower leg, ending 0.1 below it
    xi = sc.thickness
    kal = O.contact_pass(sc, mode="kaldor", cull_radius=11)
    fil = O.contact_pass(sc, mode="double")
    assert (kal.ccd_klass == O.KLASS_X).any()
    assert kal.alpha == 1.0                      # nothing constrains the step
    assert fil.alpha < 0.9                       # the filtered model stops it
    xk = sc.x + kal.alpha * sc.p
    xf = sc.x + fil.alpha * sc.p
    dk = _min_distance(sc, xk)
    df = _min_distance(sc, xf)
    # filtered model: Invariant 3 holds
    assert df[O.KLASS_U] > xi and df[O.KLASS_F] > 0 and df[O.KLASS_C] > 0
    # culled model: pairs the filtered model keeps unfiltered end inside the thickness
    assert dk[O.KLASS_U] <= xi or dk[O.KLASS_C] <= xi, dk


def two_yarns(L1=0.04, L2=0.1, n1=30, n2=12, thickness=0.25, dhat=0.01):
    """Two straight yarns 2 mm apart, of segment lengths L1 and L2."""
    a_pts = np.stack([L1 * np.arange(n1 + 1), np.zeros(n1 + 1), np.zeros(n1 + 1)])
    b_pts = np.stack([L2 * np.arange(n2 + 1), np.full(n2 + 1, 2.0), np.zeros(n2 + 1)])
    x = np.concatenate([a_pts, b_pts], axis=1)
    rp = np.array([0, n1 + 1, n1 + n2 + 2], np.int32)
    return S.Scene("rod", x.copy(), x.copy(), np.zeros_like(x), thickness, dhat, rod_ptr=rp)


def test_per_component_dbar_min():
    """Two yarns of different segment lengths: with one scene-wide dbar_min
    the coarse yarn's filtered pairs get the fine yarn's (smaller) width; per
    component each keeps its own, the smallest reference distance of its own
    filtered pairs -- the closed form of a straight rod, its segment length."""
    L1, L2, n1, n2 = 0.04, 0.1, 30, 12
    sc = two_yarns(L1, L2, n1, n2)
    x = sc.x
    glob = O.contact_pass(sc, ccd=False)
    comp = O.contact_pass(sc, ccd=False, per_component=True)
    assert np.isclose(glob.dbar_min, L1)
    topo = O.topology(sc)
    st = O.stencils(topo, comp.C)
    Fm = comp.klass == O.KLASS_F
    lab = topo.comp[st[:, 0]]
    assert np.allclose(comp.fwidth[Fm & (lab == 0)], L1) and np.allclose(comp.fwidth[Fm & (lab == 1)], L2)
    # same classes; at rest both models are inactive (every filtered pair sits at
    # or beyond its own width)
    assert np.array_equal(glob.klass, comp.klass)
    assert glob.energy == 0.0 and comp.energy == 0.0
    # the coarse yarn compressed to 0.85 of its segment length: its filtered
    # gap-2 pairs (now 0.85 L2 apart) switch on at its own width L2, not at L1
    xc = x.copy()
    xc[0, n1 + 1:] = 0.85 * L2 * np.arange(n2 + 1)
    g2 = O.contact_pass(sc, x=xc, ccd=False)
    c2 = O.contact_pass(sc, x=xc, ccd=False, per_component=True)
    act_g, act_c = set(g2.active_keys.tolist()), set(c2.active_keys.tolist())
    extra = np.array(sorted(act_c - act_g), np.uint64)
    assert act_g < act_c and extra.size == n2 - 2  # the gap-2 pairs of the n2 edges
    assert np.all(c2.klass[np.searchsorted(c2.C, extra)] == O.KLASS_F)
    assert c2.energy > g2.energy
