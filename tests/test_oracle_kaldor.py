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
