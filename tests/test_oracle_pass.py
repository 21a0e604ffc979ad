"""Pins for the oracle's whole-pass pieces: rest filter (Sec. 3.2), broad phase
at full activation (Sec. 3.3), class C (Sec. 3.4), assembly, and the additive
CCD step bound with its non-intersection invariant."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2510_10256_gb300 import scenes as S

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))


# ---------------------------------------------------------------- filter ----

def test_straight_rod_filter_closed_form():
    g = GOLD["straight_rod_filter"]
    sc = S.straight_rod(n_seg=g["n_seg"], seg=g["L"], thickness=g["thickness"], dhat=g["dhat"])
    topo = O.topology(sc)
    F, dbar = O.rest_filter(sc, topo, sc.activation)
    _, k, l = O.key_parts(F)
    expect = {(a, b) for a in range(g["n_seg"]) for b in range(a + 2, g["n_seg"])
              if b - a <= g["max_gap"]}
    assert set(zip(k.tolist(), l.tolist())) == expect
    assert dbar.min() == pytest.approx(g["dbar_min"], rel=1e-12)
    # every filtered pair is at rest distance (l-k-1) L
    assert np.allclose(dbar, (l - k - 1) * g["L"], rtol=1e-12)


def test_grid_dbar_min_closed_form():
    g = GOLD["grid_dbar_min"]
    sc = S.flat_grid(nx=7, L=g["L"])
    topo = O.topology(sc)
    F, dbar = O.rest_filter(sc, topo, sc.activation)
    assert dbar.min() == pytest.approx(g["dbar_min"], rel=1e-14)


@pytest.mark.parametrize("seed", range(3))
def test_filter_is_exactly_the_locking_pairs(seed):
    """Invariant 1: every same-component stencil pair of K with dbar < a is
    filtered, and nothing else is (checked by enumerating K with the pinned
    distance routine, no boxes)."""
    sc = S.tiny_shell(seed, nx=4, layers=2)
    topo = O.topology(sc)
    a = sc.activation
    F, dbar = O.rest_filter(sc, topo, a)
    expect = set()
    n, T, E = sc.n, topo.tris.shape[1], topo.edges.shape[1]
    X = sc.rest
    for v in range(n):
        for t in range(T):
            tv = topo.tris[:, t]
            if v in tv or topo.comp[v] != topo.comp[tv[0]]:
                continue
            d, _ = O.distance(False, np.concatenate([X[:, v], X[:, tv[0]], X[:, tv[1]], X[:, tv[2]]]))
            if d < a:
                expect.add(int(O.PT) << 62 | v << 31 | t)
    for e in range(E):
        for f in range(e + 1, E):
            ve, vf = topo.edges[:, e], topo.edges[:, f]
            if set(ve) & set(vf) or topo.comp[ve[0]] != topo.comp[vf[0]]:
                continue
            d, _ = O.distance(True, np.concatenate([X[:, ve[0]], X[:, ve[1]], X[:, vf[0]], X[:, vf[1]]]))
            if d < a:
                expect.add(int(O.EE) << 62 | e << 31 | f)
    assert set(F.tolist()) == expect


@pytest.mark.parametrize("mode", ["double", "single"])
def test_flat_rest_has_zero_energy_when_filtered(mode):
    """Invariant 2: at the flat rest of a fine grid the filtered barrier is
    inactive everywhere (no rest forces); unfiltered it locks (E > 0), the
    contact-locking of Fig. 2 / Fig. 3."""
    sc = S.flat_grid(nx=9, L=0.5, thickness=1.0, dhat=0.05)
    r = O.contact_pass(sc, mode=mode, ccd=False)
    assert r.energy == 0.0
    assert not r.active.any()
    assert (r.klass == O.KLASS_F).sum() > 0
    off = O.contact_pass(sc, mode="off", ccd=False)
    assert off.energy > 0.0
    assert np.abs(off.grad).max() > 0.0


def test_rod_rest_forces_vanish_when_filtered():
    """A single polyline with turning angles < 90 degrees has no rest forces
    with the filter, and locks without it (Fig. 3 left)."""
    rng = np.random.default_rng(3)
    n = 40
    ang = np.cumsum(rng.uniform(-0.6, 0.6, n - 1))
    seg = 0.05
    pts = np.zeros((3, n))
    pts[0, 1:] = np.cumsum(seg * np.cos(ang))
    pts[1, 1:] = np.cumsum(seg * np.sin(ang))
    sc = S.Scene("rod", pts.copy(), pts.copy(), np.zeros_like(pts), 0.2, 0.01,
                 rod_ptr=np.array([0, n], np.int32))
    r = O.contact_pass(sc, ccd=False)
    assert r.energy == 0.0 or r.energy < 1e-30
    off = O.contact_pass(sc, mode="off", ccd=False)
    assert off.energy > 0.0


def test_no_filtering_when_dbar_min_above_activation():
    """dbar_min >= a: F is empty and the filtered pass equals the plain one."""
    sc = S.tiny_rods(2, seg=0.4, thickness=0.2, dhat=0.05)
    r = O.contact_pass(sc)
    assert r.F_rest.size == 0 and (r.klass == O.KLASS_F).sum() == 0
    off = O.contact_pass(sc, mode="off")
    assert r.energy == off.energy
    assert np.array_equal(r.grad, off.grad)
    assert r.alpha == off.alpha


def test_pattern_pairs_are_never_filtered():
    """Pairs from different components (pattern-induced closeness, Sec. 3.4)
    are never filtered however close they are."""
    sc = S.tiny_shell(9, nx=4, layers=2, noise=0.0)
    r = O.contact_pass(sc, ccd=False)
    st = O.stencils(O.topology(sc), r.C)
    comp = O.topology(sc).comp
    cross = comp[st[:, 0]] != comp[st[:, 2]]
    assert cross.any()
    assert (r.klass[cross] != O.KLASS_F).all()


# ----------------------------------------------------------- broad phase ----

@pytest.mark.parametrize("maker,seed", [(S.tiny_shell, s) for s in range(4)] +
                         [(S.tiny_rods, s) for s in range(4)])
def test_broad_phase_superset_and_bounds(maker, seed):
    """Every non-incident pair closer than the activation is a candidate; no
    candidate is farther apart than its boxes allow; no candidate is incident."""
    sc = maker(seed)
    topo = O.topology(sc)
    a = sc.activation
    Cset = set(O.broad_phase(topo, sc.x, 0.5 * a).tolist())
    X = sc.x
    T, E = topo.tris.shape[1], topo.edges.shape[1]

    def bbox(vs):
        P = X[:, vs]
        return P.min(1), P.max(1)

    def box_gap(v1, v2):
        l1, h1 = bbox(v1)
        l2, h2 = bbox(v2)
        return np.maximum(0, np.maximum(l1 - h2, l2 - h1))

    pairs = []
    if topo.kind == 1:
        for v in range(sc.n):
            for t in range(T):
                if v not in topo.tris[:, t]:
                    pairs.append((int(O.PT) << 62 | v << 31 | t, False, [v], list(topo.tris[:, t])))
    ety = O.EE if topo.kind == 1 else O.ROD_EE
    for e in range(E):
        for f in range(e + 1, E):
            if not set(topo.edges[:, e]) & set(topo.edges[:, f]):
                pairs.append((int(ety) << 62 | e << 31 | f, True, list(topo.edges[:, e]), list(topo.edges[:, f])))
    n_close = 0
    for key, is_ee, v1, v2 in pairs:
        gap = box_gap(v1, v2)
        x12 = np.concatenate([X[:, v] for v in v1 + v2])
        d, _ = O.distance(is_ee, x12)
        if d < a:
            n_close += 1
            assert key in Cset
        if key in Cset:
            assert gap.max() <= a * (1 + 1e-12)
        else:
            assert gap.max() >= a * (1 - 1e-12)
    assert n_close > 0
    all_keys = {k for k, *_ in pairs}
    assert Cset <= all_keys


# --------------------------------------------------------------- classes ----

def test_class_c_marks_core_intersections():
    """Sec. 3.4: unfiltered pairs already within the offset get a temporary
    zero offset (class C) and stay finite; without it they are penetrations."""
    sc = S.woven_patch(n_warp=2, n_weft=2, nseg=40)
    r = O.contact_pass(sc, ccd=False)
    cc = r.klass == O.KLASS_C
    assert cc.any()
    assert (r.d[cc] <= sc.thickness).all()
    assert ((r.d[r.klass == O.KLASS_U] > sc.thickness)).all()
    assert np.isfinite(r.energy) and not r.penetration
    r2 = O.contact_pass(sc, ccd=False, core_temp=False)
    assert r2.penetration and not np.isfinite(r2.energy)


# -------------------------------------------------------------- assembly ----

def _fd_setup(seed):
    sc = S.tiny_shell(seed, nx=4, layers=2)
    topo = O.topology(sc)
    filt = O.rest_filter(sc, topo, sc.activation)
    return sc, topo, filt


@pytest.mark.parametrize("seed", range(3))
def test_gradient_is_energy_derivative(seed):
    """Assembled gradient equals the central difference of the total energy
    (catches stencil index, sign and scatter mistakes)."""
    sc, topo, filt = _fd_setup(seed)
    r = O.contact_pass(sc, ccd=False, topo=topo, filt=filt)
    assert r.active.sum() > 0
    rng = np.random.default_rng(seed)
    verts = np.unique(O.stencils(topo, r.active_keys))
    h = 1e-7
    checked = 0
    for v in rng.choice(verts, size=min(8, verts.size), replace=False):
        for k in range(3):
            xp, xm = sc.x.copy(), sc.x.copy()
            xp[k, v] += h
            xm[k, v] -= h
            rp = O.contact_pass(sc, ccd=False, x=xp, topo=topo, filt=filt)
            rm = O.contact_pass(sc, ccd=False, x=xm, topo=topo, filt=filt)
            if not (np.array_equal(rp.klass, r.klass) and np.array_equal(rm.klass, r.klass)):
                continue
            fd = (rp.energy - rm.energy) / (2 * h)
            assert r.grad[k, v] == pytest.approx(fd, rel=1e-5, abs=1e-6 * (1 + abs(fd)))
            checked += 1
    assert checked >= 6


@pytest.mark.parametrize("seed", range(2))
def test_unprojected_hessian_is_gradient_derivative(seed):
    sc, topo, filt = _fd_setup(seed)
    r = O.contact_pass(sc, ccd=False, topo=topo, filt=filt, project=False)
    A = O.bsr_dense(r, sc.n)
    rng = np.random.default_rng(seed)
    verts = np.unique(O.stencils(topo, r.active_keys))
    h = 1e-7
    checked = 0
    for v in rng.choice(verts, size=min(5, verts.size), replace=False):
        for k in range(3):
            xp, xm = sc.x.copy(), sc.x.copy()
            xp[k, v] += h
            xm[k, v] -= h
            rp = O.contact_pass(sc, ccd=False, x=xp, topo=topo, filt=filt)
            rm = O.contact_pass(sc, ccd=False, x=xm, topo=topo, filt=filt)
            if not (np.array_equal(rp.active, r.active) and np.array_equal(rm.active, r.active)
                    and np.array_equal(rp.klass, r.klass) and np.array_equal(rm.klass, r.klass)):
                continue
            fd = ((rp.grad - rm.grad) / (2 * h)).reshape(-1)     # d grad / d x[k, v]
            col = A[:, 3 * v + k]
            # dense layout is vertex-major (3 v + k); grad is (3, n) axis-major
            fdv = fd.reshape(3, sc.n).T.reshape(-1)
            scale = np.abs(col).max() + 1e-12
            assert np.abs(col - fdv).max() <= 1e-4 * scale
            checked += 1
    assert checked >= 3


@pytest.mark.parametrize("seed", range(3))
def test_projected_bsr_symmetric_psd_and_pattern(seed):
    sc, topo, filt = _fd_setup(seed)
    r = O.contact_pass(sc, ccd=False, topo=topo, filt=filt)
    A = O.bsr_dense(r, sc.n)
    assert np.abs(A - A.T).max() <= 1e-12 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() >= -1e-10 * np.abs(A).max()
    st = O.stencils(topo, r.active_keys)
    want = {(int(i), int(j)) for s in st for i in s for j in s}
    got = set()
    for row in range(sc.n):
        for q in range(r.bsr_row_ptr[row], r.bsr_row_ptr[row + 1]):
            got.add((row, int(r.bsr_col[q])))
    assert got == want
    assert np.all(np.diff(r.bsr_col[r.bsr_row_ptr[0]:r.bsr_row_ptr[1]]) > 0)


# ------------------------------------------------------------------- CCD ----

def test_accd_head_on_closed_form():
    """Point moving straight at a static triangle face: the additive CCD
    returns (1 - s) of the time of impact with the offset."""
    tri = [np.array([0.0, 0, 0]), np.array([1.0, 0, 0]), np.array([0.0, 1.0, 0])]
    p0 = np.array([0.25, 0.25, 0.8])
    xi = 0.1
    v = 1.4
    x12 = np.concatenate([p0] + tri)
    p12 = np.concatenate([np.array([0, 0, -v])] + [np.zeros(3)] * 3)
    t, st, it = O.accd(False, x12, p12, xi)
    t_star = (0.8 - xi) / v
    assert st == 0
    assert t == pytest.approx((1 - O.ACCD_S) * t_star, rel=1e-12)
    # moving away: no impact within [0, 1]
    t2, _, _ = O.accd(False, x12, -p12, xi)
    assert t2 == 1.0


def _true_toi(is_ee, x12, p12, off, n=20000):
    ts = np.linspace(0, 1, n + 1)
    prev = 0.0
    for t in ts:
        d, _ = O.distance(is_ee, x12 + t * p12)
        if d - off <= 0:
            lo, hi = prev, t
            for _ in range(60):
                mid = 0.5 * (lo + hi)
                dm, _ = O.distance(is_ee, x12 + mid * p12)
                if dm - off <= 0:
                    hi = mid
                else:
                    lo = mid
            return hi
        prev = t
    return 2.0


@pytest.mark.parametrize("seed", range(30))
def test_accd_never_overshoots_sampled_toi(seed):
    rng = np.random.default_rng(1000 + seed)
    is_ee = bool(seed % 2)
    x12 = rng.normal(size=12)
    p12 = rng.normal(size=12) * 1.5
    d0, _ = O.distance(is_ee, x12)
    off = 0.3 * d0
    t, st, _ = O.accd(is_ee, x12, p12, off)
    assert st == 0
    tt = _true_toi(is_ee, x12, p12, off, n=4000)
    assert t <= tt
    d1, _ = O.distance(is_ee, x12 + t * p12)
    assert d1 - off > 0


@pytest.mark.parametrize("maker,seed", [(S.tiny_shell, 21), (S.tiny_shell, 22), (S.tiny_rods, 23),
                                        (S.tiny_rods, 24)])
def test_step_bound_keeps_every_pair_outside_its_offset(maker, seed):
    """Invariant 3: after x + alpha p no pair of the whole mesh (brute force, not
    only the CCD candidates) has crossed its offset: unfiltered pairs that were
    outside the thickness stay outside it, filtered / class-C pairs stay apart."""
    sc = maker(seed)
    topo = O.topology(sc)
    r = O.contact_pass(sc, topo=topo)
    assert 0 < r.alpha <= 1
    x1 = sc.x + r.alpha * sc.p
    allp = O.broad_phase(topo, sc.x, 1e9)            # every non-incident pair
    r0 = O.contact_pass(sc, topo=topo, ccd=False, x=sc.x)
    Fset = set(r.F_rest.tolist())
    st = O.stencils(topo, allp)
    for key, s in zip(allp.tolist(), st):
        is_ee = (key >> 62) != O.PT
        d0, _ = O.distance(is_ee, np.concatenate([sc.x[:, v] for v in s]))
        d1, _ = O.distance(is_ee, np.concatenate([x1[:, v] for v in s]))
        if key in Fset or d0 <= sc.thickness:
            assert d1 > 0
        else:
            assert d1 > sc.thickness
    # and the full step usually is not safe on these scenes
    assert r.alpha < 1


def test_ccd_candidates_cover_swept_contacts():
    """Every pair whose distance along the linear path x + t p (t in [0,1],
    sampled) drops below the offset of a U pair is a CCD candidate."""
    sc = S.tiny_shell(31)
    topo = O.topology(sc)
    keys = set(O.broad_phase(topo, sc.x, 0.5 * sc.thickness, p=sc.p).tolist())
    allp = O.broad_phase(topo, sc.x, 1e9)
    st = O.stencils(topo, allp)
    hits = 0
    for key, s in zip(allp.tolist(), st):
        is_ee = (key >> 62) != O.PT
        for t in np.linspace(0, 1, 11):
            xt = sc.x + t * sc.p
            d, _ = O.distance(is_ee, np.concatenate([xt[:, v] for v in s]))
            if d < sc.thickness:
                hits += 1
                assert key in keys
                break
    assert hits > 0
