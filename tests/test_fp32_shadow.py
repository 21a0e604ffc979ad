"""FP32 vs FP64 on the barrier argument y = d - xi (test only: nothing in the
library computes distances in FP32 without an FP64 decision behind it).

On the woven rod patch the crossing pairs of different yarns sit at
d ~ thickness, so y is a small difference of O(1) numbers.  The same
edge-edge distance evaluated in FP32 (a plain clamped segment-segment
closest-point routine) errs in y by a sizeable fraction of y itself and of
dhat near activation, far above the 1e-12 distance tolerance the FP64 path
meets; the barrier's log(y / dhat) and 1/y terms amplify that further.
"""
import numpy as np

import oracle as O
from paper_2510_10256_gb300 import scenes as S


def _seg_dist(p0, p1, q0, q1, dt):
    p0, p1, q0, q1 = (np.asarray(v, dt) for v in (p0, p1, q0, q1))
    d1, d2, r = p1 - p0, q1 - q0, p0 - q0
    a, e, f = (d1 * d1).sum(-1), (d2 * d2).sum(-1), (d2 * r).sum(-1)
    c, b = (d1 * r).sum(-1), (d1 * d2).sum(-1)
    den = a * e - b * b
    s = np.where(den > 0, np.clip((b * f - c * e) / np.where(den > 0, den, 1), 0, 1), 0).astype(dt)
    t = (b * s + f) / e
    s = np.where(t < 0, np.clip(-c / a, 0, 1), np.where(t > 1, np.clip((b - c) / a, 0, 1), s)).astype(dt)
    t = np.clip(t, 0, 1).astype(dt)
    diff = (p0 + s[:, None] * d1) - (q0 + t[:, None] * d2)
    return np.sqrt((diff * diff).sum(-1))


def test_fp32_shadow_error_of_y_on_crossings():
    sc = S.woven_patch()
    r = O.contact_pass(sc, ccd=False)
    topo = O.topology(sc)
    st = O.stencils(topo, r.C)
    x = sc.x.T
    xi, dhat = sc.thickness, sc.dhat
    # crossing pairs: different yarns (components), within the activation
    comp = topo.comp
    cross = (comp[st[:, 0]] != comp[st[:, 2]]) & (r.d < xi + dhat)
    assert cross.sum() > 100
    P = st[cross]
    d64 = r.d[cross]
    d32 = _seg_dist(x[P[:, 0]], x[P[:, 1]], x[P[:, 2]], x[P[:, 3]], np.float32).astype(np.float64)
    dref = _seg_dist(x[P[:, 0]], x[P[:, 1]], x[P[:, 2]], x[P[:, 3]], np.float64)
    # the FP64 routine here agrees with the oracle's distances to rounding
    assert np.max(np.abs(dref - d64) / d64) < 1e-12
    y64 = d64 - xi
    err = np.abs(d32 - d64)
    near = np.abs(y64) < dhat
    rel_dhat = err.max() / dhat
    rel_y = np.max(err[near] / np.maximum(np.abs(y64[near]), 1e-300))
    print(f"FP32 shadow error on {cross.sum()} crossing pairs: max |dy| = {err.max():.3e} mm "
          f"= {rel_dhat:.2e} dhat; max |dy|/|y| over pairs within dhat of the offset = {rel_y:.2e}")
    # far outside the 1e-12 relative distance tolerance of the FP64 path
    assert rel_y > 1e-6 and err.max() / xi > 1e-9
