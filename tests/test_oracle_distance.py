"""Pins for the oracle's point-triangle and edge-edge distances and types:
closed forms on hand-built configurations, and brute-force closest-point search
(dense sampling + refinement, written independently of the oracle)."""
import numpy as np
import pytest

import oracle as O
from tests._geom import closest_ee_search, closest_pt_search, random_rotation

pytestmark = pytest.mark.filterwarnings("ignore")


def _place(rng, pts):
    """Random rigid motion of a set of points (catches axis/sign slips)."""
    R = random_rotation(rng)
    t = rng.uniform(-50, 50, 3)
    return [R @ p + t for p in pts]


@pytest.mark.parametrize("seed", range(5))
def test_pt_face_height(seed):
    rng = np.random.default_rng(seed)
    z = 0.37
    t0, t1, t2 = np.array([0.0, 0, 0]), np.array([1.0, 0, 0]), np.array([0.0, 1.0, 0])
    p = np.array([0.2, 0.3, z])
    pts = _place(rng, [p, t0, t1, t2])
    d, ty = O.distance(False, np.concatenate(pts))
    assert ty == 6
    assert abs(d - z) <= 1e-12 * 50


@pytest.mark.parametrize("seed", range(5))
def test_pt_vertex_region(seed):
    rng = np.random.default_rng(seed)
    t0, t1, t2 = np.array([0.0, 0, 0]), np.array([1.0, 0, 0]), np.array([0.0, 1.0, 0])
    p = np.array([1.5, -0.4, 0.3])           # beyond t1
    pts = _place(rng, [p, t0, t1, t2])
    d, ty = O.distance(False, np.concatenate(pts))
    assert ty == 1
    assert abs(d - np.linalg.norm(p - t1)) <= 1e-12 * 50


@pytest.mark.parametrize("seed", range(5))
def test_pt_edge_region(seed):
    rng = np.random.default_rng(seed)
    t0, t1, t2 = np.array([0.0, 0, 0]), np.array([1.0, 0, 0]), np.array([0.0, 1.0, 0])
    p = np.array([0.4, -0.3, 0.2])           # beside edge t0 t1
    pts = _place(rng, [p, t0, t1, t2])
    d, ty = O.distance(False, np.concatenate(pts))
    assert ty == 3
    assert abs(d - np.hypot(0.3, 0.2)) <= 1e-12 * 50
    # beside the hypotenuse t1 t2
    p = np.array([0.8, 0.8, -0.1])
    pts = _place(rng, [p, t0, t1, t2])
    d, ty = O.distance(False, np.concatenate(pts))
    assert ty == 4
    h = (0.8 + 0.8 - 1.0) / np.sqrt(2.0)
    assert abs(d - np.hypot(h, 0.1)) <= 1e-12 * 50


@pytest.mark.parametrize("seed", range(5))
def test_ee_skew_perpendicular(seed):
    rng = np.random.default_rng(seed)
    sep = 0.123
    a0, a1 = np.array([-1.0, 0, 0]), np.array([1.0, 0, 0])
    b0, b1 = np.array([0.0, -1.0, sep]), np.array([0.0, 1.0, sep])
    pts = _place(rng, [a0, a1, b0, b1])
    d, ty = O.distance(True, np.concatenate(pts))
    assert ty == 8
    assert abs(d - sep) <= 1e-12 * 50


@pytest.mark.parametrize("seed", range(5))
def test_ee_parallel_and_collinear(seed):
    rng = np.random.default_rng(seed)
    # parallel, overlapping in projection: distance is the offset
    a0, a1 = np.array([0.0, 0, 0]), np.array([1.0, 0, 0])
    b0, b1 = np.array([0.5, 0.2, 0]), np.array([1.5, 0.2, 0])
    pts = _place(rng, [a0, a1, b0, b1])
    d, ty = O.distance(True, np.concatenate(pts))
    assert ty in (5, 6)                       # PE(a1, b) or PE(b0, a): both exact
    assert abs(d - 0.2) <= 1e-12 * 50
    # collinear with a gap: endpoint distance
    b0, b1 = np.array([1.3, 0.0, 0]), np.array([2.0, 0.0, 0])
    pts = _place(rng, [a0, a1, b0, b1])
    d, ty = O.distance(True, np.concatenate(pts))
    assert ty == 2                            # PP(a1, b0)
    assert abs(d - 0.3) <= 1e-12 * 50


def _check_pt_type(ty, u, v, tol=1e-6):
    """Type must agree with where the refined closest point lies."""
    w0 = 1.0 - u - v
    at_vertex = [w0 > 1 - tol, u > 1 - tol, v > 1 - tol]
    on_edge = [v < tol, w0 < tol, u < tol]    # t0t1, t1t2, t2t0
    if ty <= 2:
        return at_vertex[ty]
    if ty <= 5:
        return on_edge[ty - 3]
    return not any(on_edge)


@pytest.mark.parametrize("seed", range(40))
def test_pt_bruteforce(seed):
    rng = np.random.default_rng(100 + seed)
    t = rng.normal(size=(3, 3))
    p = rng.normal(size=3) * 1.5
    d, ty = O.distance(False, np.concatenate([p, t[0], t[1], t[2]]))
    ds, u, v = closest_pt_search(p, t[0], t[1], t[2], n=600)
    L = np.abs(t).max()
    assert ds >= d - 1e-12 * L            # sampling never beats the distance
    assert ds <= d + 1e-9 * L             # and the refined search reaches it
    assert _check_pt_type(ty, u, v)


def _check_ee_type(ty, s, t, tol=1e-6):
    ends = {0: (0, 0), 1: (0, 1), 2: (1, 0), 3: (1, 1)}
    if ty in ends:
        es, et = ends[ty]
        return abs(s - es) < tol and abs(t - et) < tol
    if ty == 4:
        return s < tol
    if ty == 5:
        return s > 1 - tol
    if ty == 6:
        return t < tol
    if ty == 7:
        return t > 1 - tol
    return tol < s < 1 - tol and tol < t < 1 - tol


@pytest.mark.parametrize("seed", range(40))
def test_ee_bruteforce(seed):
    rng = np.random.default_rng(300 + seed)
    x = rng.normal(size=(4, 3))
    d, ty = O.distance(True, x.reshape(-1))
    ds, s, t = closest_ee_search(x[0], x[1], x[2], x[3], n=600)
    L = np.abs(x).max()
    assert ds >= d - 1e-12 * L
    assert ds <= d + 1e-9 * L
    assert _check_ee_type(ty, s, t)


def test_all_types_reached():
    """Random stencils reach every point-triangle and edge-edge type."""
    rng = np.random.default_rng(7)
    seen_pt, seen_ee = set(), set()
    for _ in range(4000):
        x = rng.normal(size=12)
        seen_pt.add(O.distance(False, x)[1])
        seen_ee.add(O.distance(True, x)[1])
    assert seen_pt == set(range(7))
    assert seen_ee == set(range(9))
