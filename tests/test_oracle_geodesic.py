"""Pins of the oracle's geodesic reference distances (scene.rest_geodesic,
oracle/geodesic.c): shells whose rest shape is not cut from a flat pattern
take dbar as the shortest-path distance on the rest mesh between the two
primitives (Sec. 3.2's 2D rest-domain distance; the paper leaves non-flat
rest shapes to future work).

What fixes the values independently of the oracle's method:
  * a flat sheet (convex, rigidly rotated into 3D) and a sheet rolled onto a
    cylinder (isometric to its chord pattern) filter exactly as the pattern
    does: same keys, dbar equal to rounding;
  * polyhedral cones, flat except at the apex: the distance between two
    points is the law of cosines in the unrolled cone when their unrolled
    angular separation is below pi, and the sum of their slant radii (a path
    through the apex) otherwise -- a convex apex (angle sum < 2 pi) and a
    saddle apex (angle sum > 2 pi);
  * on the saddle cone, the edge-edge and point-triangle distances across the
    apex are the sums of the closed-form distances to the apex;
  * a flat L-shaped sheet: a path whose straight segment would leave the
    sheet bends at the reflex corner, |p - c| + |c - q|;
  * a Steiner-point graph (points on every edge, straight segments within
    each face) gives paths on the surface: its distances bound the geodesic
    from above and close in on it as the points get denser -- vertex to
    vertex, vertex to edge, and primitive to primitive for the filtered
    pairs' dbar;
  * symmetry, the triangle inequality, and geodesic >= 3D distance;
  * a spherical cap: distances approach the great-circle arcs at second
    order in the edge length.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2510_10256_gb300 import scenes as S


def _shell(rest, tris, a=1.0, geodesic=True):
    rest = np.ascontiguousarray(rest, np.float64)
    return S.Scene("shell", rest.copy(), rest.copy(), np.zeros_like(rest), 0.9 * a, 0.1 * a,
                   tris=np.ascontiguousarray(tris, np.int32), rest_geodesic=geodesic)


def _cone(m, rings, beta, dr=1.0):
    """Apex (vertex 0) and `rings` rings of m vertices on the generators
    g_i = (sin b_i cos phi_i, sin b_i sin phi_i, cos b_i), phi_i = 2 pi i / m,
    ring k at slant radius k dr.  Each sector between two generators is
    planar (both pass through the apex), so the surface is flat except at the
    apex.  Returns rest, tris, sector angles (angle between g_i and g_i+1),
    and the vertex id function idx(k, i)."""
    phi = 2.0 * np.pi * np.arange(m) / m
    b = np.array([beta(i) for i in range(m)])
    g = np.stack([np.sin(b) * np.cos(phi), np.sin(b) * np.sin(phi), np.cos(b)])
    rest = np.concatenate([np.zeros((3, 1))] + [k * dr * g for k in range(1, rings + 1)], axis=1)

    def idx(k, i):
        return 0 if k == 0 else 1 + (k - 1) * m + (i % m)
    tris = []
    for i in range(m):
        tris.append((0, idx(1, i), idx(1, i + 1)))
        for k in range(1, rings):
            tris.append((idx(k, i), idx(k + 1, i), idx(k + 1, i + 1)))
            tris.append((idx(k, i), idx(k + 1, i + 1), idx(k, i + 1)))
    alpha = np.array([math.acos(max(-1.0, min(1.0, float(g[:, i] @ g[:, (i + 1) % m])))) for i in range(m)])
    return rest, np.array(tris, np.int32).T, alpha, idx


CONVEX = lambda i: math.radians(60.0)                                  # noqa: E731
SADDLE = lambda i: math.radians(90.0 + (30.0 if i % 2 else -30.0))     # noqa: E731


@pytest.mark.parametrize("beta", [CONVEX, SADDLE], ids=["convex_apex", "saddle_apex"])
def test_cone_vertex_distances_closed_form(beta):
    m, R = 16, 6
    rest, tris, alpha, idx = _cone(m, R, beta)
    theta = alpha.sum()
    assert (theta < 2 * math.pi) == (beta is CONVEX)
    cum = np.concatenate([[0.0], np.cumsum(alpha)])
    sc = _shell(rest, tris)
    for src_k, src_i in [(6, 0), (3, 5), (1, 2)]:
        dv, _ = O.geodesic_from(sc, idx(src_k, src_i), 100.0)
        assert abs(dv[0] - src_k) <= 1e-14 * src_k
        for k in range(1, R + 1):
            for i in range(m):
                d = abs(cum[i] - cum[src_i])
                D = min(d, theta - d)
                if D < math.pi:
                    exact = math.sqrt(src_k * src_k + k * k - 2.0 * src_k * k * math.cos(D))
                else:
                    exact = src_k + k
                got = dv[idx(k, i)]
                assert abs(got - exact) <= 1e-13 * max(exact, 1.0), (k, i, got, exact)


def _pt_seg_2d(p, a, b):
    """Distance from point p to segment ab in the plane (textbook projection)."""
    ab, ap = b - a, p - a
    t = min(1.0, max(0.0, float(ap @ ab) / float(ab @ ab)))
    return float(np.linalg.norm(ap - t * ab))


def test_saddle_apex_edge_edge_and_point_triangle():
    m, R = 16, 5
    rest, tris, alpha, idx = _cone(m, R, SADDLE)
    sc = _shell(rest, tris, a=20.0)
    topo = O.topology(sc)
    F, dbar = O.rest_filter(sc, topo, 20.0)
    got = dict(zip(F.tolist(), dbar.tolist()))
    eid = {(int(a), int(b)): k for k, (a, b) in enumerate(zip(*topo.edges))}

    def edge(u, v):
        return eid[(min(u, v), max(u, v))]

    def polar(r, ang):
        return np.array([r * math.cos(ang), r * math.sin(ang)])
    # ring edges in sectors 0 and 8: seven sectors apart either way round (> pi)
    assert 7 * alpha[0] > math.pi
    for kA, kB in [(2, 3), (4, 1), (5, 5)]:
        A, B = edge(idx(kA, 0), idx(kA, 1)), edge(idx(kB, 8), idx(kB, 9))
        key = (O.EE << 62) | (min(A, B) << 31) | max(A, B)
        exact = kA * math.cos(alpha[0] / 2) + kB * math.cos(alpha[8] / 2)
        assert abs(got[key] - exact) <= 1e-13 * exact, (got[key], exact)
        # the same pair's distance through its end points alone is longer
        ends = []
        for v, other in [(idx(kA, 0), B), (idx(kA, 1), B), (idx(kB, 8), A), (idx(kB, 9), A)]:
            ends.append(O.geodesic_from(sc, v, 20.0, topo)[1][other])
        assert min(ends) > exact + 0.1
    # vertex on generator 0, triangle (k, 8), (k+1, 8), (k+1, 9) in sector 8
    tv = {tuple(sorted(t)): j for j, t in enumerate(tris.T.tolist())}
    for kp, kt in [(3, 2), (1, 4)]:
        p = idx(kp, 0)
        j = tv[tuple(sorted((idx(kt, 8), idx(kt + 1, 8), idx(kt + 1, 9))))]
        key = (O.PT << 62) | (p << 31) | j
        T = [polar(kt, 0.0), polar(kt + 1, 0.0), polar(kt + 1, alpha[8])]   # sector 8 unrolled
        o = np.zeros(2)
        exact = kp + min(_pt_seg_2d(o, T[q], T[(q + 1) % 3]) for q in range(3))
        assert abs(got[key] - exact) <= 1e-13 * exact, (got[key], exact)


def _flat_noisy(nx, L, seed):
    rng = np.random.default_rng(seed)
    rest, tris = S.grid_mesh(nx, nx, L)
    half = 0.5 * (nx - 1) * L - 1e-9
    inner = (np.abs(rest[0]) < half) & (np.abs(rest[1]) < half)   # the boundary stays straight: convex
    rest[:2, inner] += rng.uniform(-0.3 * L, 0.3 * L, (2, int(inner.sum())))
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    return (q * np.sign(np.diag(r))) @ rest, tris


@pytest.mark.parametrize("a", [0.25, 0.35])
def test_flat_sheet_matches_euclidean(a):
    rest, tris = _flat_noisy(20, 0.1, 3)
    sc = _shell(rest, tris, a=a)
    topo = O.topology(sc)
    Fg, dg = O.rest_filter(sc, topo, a)
    sc.rest_geodesic = False
    Fe, de = O.rest_filter(sc, topo, a)
    assert Fg.size > 1000 and np.array_equal(Fg, Fe)
    assert np.max(np.abs(dg - de) / de) <= 1e-13


def _cylinder(nx, ny, R, arc, dz):
    rest, tris = S.grid_mesh(nx, ny, 1.0)
    i = np.round(rest[0] + 0.5 * (nx - 1)).astype(int)
    j = np.round(rest[1] + 0.5 * (ny - 1)).astype(int)
    th = i * (arc / R)
    cyl = np.stack([R * np.sin(th), j * dz, R - R * np.cos(th)])
    chord = 2.0 * R * math.sin(0.5 * arc / R)
    pattern = np.stack([i * chord, j * dz, np.zeros(i.size)])
    return cyl, pattern, tris, chord


@pytest.mark.parametrize("a", [0.45, 0.7])
def test_rolled_sheet_matches_its_chord_pattern(a):
    cyl, pattern, tris, chord = _cylinder(24, 12, 1.5, 0.25, 0.25)
    sc = _shell(cyl, tris, a=a)
    topo = O.topology(sc)
    Fg, dg = O.rest_filter(sc, topo, a)
    tw = _shell(pattern, tris, a=a, geodesic=False)
    Fp, dp = O.rest_filter(tw, topo, a)
    assert np.array_equal(Fg, Fp)
    assert np.max(np.abs(dg - dp) / dp) <= 1e-13
    # closest stencil: a vertex and the opposite diagonal of its cell (the cell's altitude)
    assert abs(dg.min() - chord * 0.25 / math.hypot(chord, 0.25)) <= 1e-13
    sc.rest_geodesic = False
    _, d3 = O.rest_filter(sc, topo, a)
    assert d3.min() < dg.min() * (1.0 - 1e-4)                        # chords through the cylinder undercut it


def _bumpy(nx, L, seed, amp=0.25):
    rng = np.random.default_rng(seed)
    rest, tris = S.grid_mesh(nx, nx, L)
    W = nx * L
    rest[2] = amp * W * np.sin(2.1 * np.pi * rest[0] / W) * np.cos(1.7 * np.pi * rest[1] / W) \
        + rng.normal(0.0, 0.05 * L, rest.shape[1])
    return _shell(rest, tris)


def _steiner_graph(sc, k):
    """Vertices plus k evenly spaced points inside every edge; within each
    face, every two of its boundary points joined by their 3D distance."""
    from scipy.sparse import coo_matrix
    topo = O.topology(sc)
    n = sc.n
    e0, e1 = topo.edges
    s = np.arange(1, k + 1) / (k + 1)
    P = sc.rest[:, e0][:, :, None] * (1 - s) + sc.rest[:, e1][:, :, None] * s
    pos = np.concatenate([sc.rest.T, P.transpose(1, 2, 0).reshape(-1, 3)])
    eid = {(int(a), int(b)): i for i, (a, b) in enumerate(zip(e0, e1))}
    rows, cols = [], []
    for f in range(sc.tris.shape[1]):
        vs = sc.tris[:, f].tolist()
        nodes = list(vs)
        for q in range(3):
            u, v = vs[q], vs[(q + 1) % 3]
            e = eid[(min(u, v), max(u, v))]
            nodes += [n + e * k + j for j in range(k)]
        I, J = np.meshgrid(nodes, nodes)
        msk = I < J
        rows.append(I[msk])
        cols.append(J[msk])
    key = np.unique(np.concatenate(rows).astype(np.int64) * len(pos) + np.concatenate(cols))
    r, c = key // len(pos), key % len(pos)
    w = np.linalg.norm(pos[r] - pos[c], axis=1)
    return coo_matrix((w, (r, c)), shape=(len(pos), len(pos))).tocsr(), topo


def test_steiner_graph_bounds_from_above():
    pytest.importorskip("scipy")
    from scipy.sparse.csgraph import dijkstra
    sc = _bumpy(7, 0.1, 1)
    gaps = {}
    for k in (8, 16):
        G, topo = _steiner_graph(sc, k)
        worst = 0.0
        for src in (0, 10, 24):
            dv, de = O.geodesic_from(sc, src, 10.0, topo)
            gd = dijkstra(G, directed=False, indices=src)
            gap = gd[:sc.n] - dv
            assert gap.min() >= -1e-13                           # never shorter than a surface path
            worst = max(worst, float(np.max(gap[dv > 0] / dv[dv > 0])))
            # edges: the nearest graph node on an edge bounds g(src, e) from above
            on_edge = np.minimum(gd[topo.edges[0]], gd[topo.edges[1]])
            inner = gd[sc.n:].reshape(-1, k).min(axis=1)
            ub = np.minimum(on_edge, inner)
            assert np.all(de <= ub + 1e-13)
            assert np.max(ub - de) <= 0.01
        gaps[k] = worst
    assert gaps[16] <= 0.006 and gaps[16] < gaps[8]


def test_symmetry_triangle_inequality_and_chord_bound():
    sc = _bumpy(7, 0.1, 1)
    topo = O.topology(sc)
    D = np.array([O.geodesic_from(sc, s, 10.0, topo)[0] for s in range(sc.n)])
    assert np.max(np.abs(D - D.T) / np.maximum(D, 1e-300)) <= 1e-13
    for a in range(sc.n):
        assert np.all(D[a][:, None] <= D[a][None, :] + D + 1e-13)
    chord = np.linalg.norm(sc.rest[:, :, None] - sc.rest[:, None, :], axis=0)
    assert np.all(D >= chord * (1 - 1e-14))


def test_rest_filter_bounds_on_a_doubly_curved_sheet():
    sc = _bumpy(24, 0.1, 5, amp=0.15)
    a = 0.3
    topo = O.topology(sc)
    Fg, dg = O.rest_filter(sc, topo, a)
    sc.rest_geodesic = False
    Fe, de = O.rest_filter(sc, topo, a)
    assert Fg.size > 1000
    pos = np.searchsorted(Fe, Fg)
    assert np.all(Fe[pos] == Fg)                     # the geodesic set is a subset of the 3D one
    assert np.all(dg >= de[pos] * (1 - 1e-14))       # and its distances are no shorter
    assert np.any(dg > de[pos] * (1 + 1e-6))         # curved: some are strictly longer


def _cap(nx, W, R):
    rest, tris = S.grid_mesh(nx, nx, W / (nx - 1))
    v = np.stack([rest[0], rest[1], np.full(rest.shape[1], R)])
    return _shell(R * v / np.linalg.norm(v, axis=0), tris)


def test_spherical_cap_second_order():
    R = 1.0
    errs, hs = [], []
    for nx in (9, 17):
        sc = _cap(nx, 1.0, R)
        topo = O.topology(sc)
        src = (nx // 2) * nx + nx // 2
        dv, _ = O.geodesic_from(sc, src, 10.0, topo)
        p = sc.rest
        arc = R * np.arccos(np.clip((p.T @ p[:, src]) / R ** 2, -1.0, 1.0))
        m = arc > 0
        rel = np.abs(dv[m] - arc[m]) / arc[m]
        h = float(np.max(np.linalg.norm(p[:, topo.edges[0]] - p[:, topo.edges[1]], axis=0)))
        assert rel.max() <= h * h / (4.0 * R * R)
        errs.append(rel.max())
        hs.append(h)
    order = math.log(errs[0] / errs[1]) / math.log(hs[0] / hs[1])
    assert 1.7 <= order <= 2.3


def _l_sheet(n, L):
    """An L-shaped flat sheet: the (2n+1) x (2n+1) vertex grid of spacing L
    without its upper-right quadrant's open interior, so (0, 0) is a reflex
    corner of the boundary (inner angle 3 pi / 2)."""
    idx, pts = {}, []
    for j in range(-n, n + 1):
        for i in range(-n, n + 1):
            if i > 0 and j > 0:
                continue
            idx[(i, j)] = len(pts)
            pts.append((i * L, j * L, 0.0))
    tris = []
    for j in range(-n, n):
        for i in range(-n, n):
            q = [(i, j), (i + 1, j), (i + 1, j + 1), (i, j + 1)]
            if not all(c in idx for c in q):
                continue
            tris.append((idx[q[0]], idx[q[1]], idx[q[2]]))
            tris.append((idx[q[0]], idx[q[2]], idx[q[3]]))
    return np.array(pts).T, np.array(tris, np.int32).T, idx


def test_paths_bend_at_a_reflex_boundary_corner():
    """On a flat L-shaped sheet the shortest path between two vertices is
    the straight segment when it stays in the sheet, else the two segments
    through the reflex corner (0, 0): |p - c| + |c - q|."""
    n, L = 4, 0.25
    rest, tris, idx = _l_sheet(n, L)
    sc = _shell(rest, tris)
    topo = O.topology(sc)
    src = (4, -1)   # below the corner, right of it
    dv, _ = O.geodesic_from(sc, idx[src], 100.0, topo)
    p = np.array(src, float) * L
    bent = 0
    for (i, j), v in idx.items():
        q = np.array((i, j), float) * L
        # the segment p -> q leaves the sheet iff it passes through the open
        # quadrant x > 0, y > 0: for p right of the y axis and below the x
        # axis, iff q is above the x axis and the corner lies strictly left
        # of the directed segment p -> q
        straight = float(np.linalg.norm(q - p))
        crosses = q[1] > 0 and (q[0] - p[0]) * (0 - p[1]) - (q[1] - p[1]) * (0 - p[0]) > 0
        exact = float(np.linalg.norm(p)) + float(np.linalg.norm(q)) if crosses else straight
        bent += crosses
        assert abs(dv[v] - exact) <= 1e-13 * max(exact, 1.0), ((i, j), dv[v], exact)
    assert bent >= 8


def test_pair_distances_within_the_steiner_bound():
    """dbar of every filtered pair of a bumpy sheet (both curvature signs)
    lies between the 3D distance of its primitives and the Steiner graph's
    shortest path between their points (a multi-source search from the
    first primitive's points), which it approaches from below."""
    pytest.importorskip("scipy")
    from scipy.sparse.csgraph import dijkstra
    sc = _bumpy(7, 0.1, 1)
    a = 0.3
    topo = O.topology(sc)
    F, dbar = O.rest_filter(sc, topo, a)
    k = 8
    G, _ = _steiner_graph(sc, k)
    n, E, T = sc.n, topo.edges.shape[1], sc.tris.shape[1]
    eid = {(int(u), int(v)): i for i, (u, v) in enumerate(zip(*topo.edges))}

    def edge_nodes(e):
        return [int(topo.edges[0, e]), int(topo.edges[1, e])] + [n + e * k + j for j in range(k)]

    def tri_edges(t):
        vs = sc.tris[:, t].tolist()
        return [eid[(min(vs[q], vs[(q + 1) % 3]), max(vs[q], vs[(q + 1) % 3]))] for q in range(3)]
    sel = np.random.default_rng(2).choice(F.size, size=min(300, F.size), replace=False)
    worst = 0.0
    for c in sel:
        key = int(F[c])
        ty, i, j = key >> 62, (key >> 31) & 0x7FFFFFFF, key & 0x7FFFFFFF
        if ty == O.PT:
            src = [i]
            dst = sorted({v for e in tri_edges(j) for v in edge_nodes(e)})
        else:
            src, dst = edge_nodes(i), edge_nodes(j)
        dist = dijkstra(G, directed=False, indices=src, min_only=True)
        ub = float(np.min(dist[dst]))
        assert dbar[c] <= ub + 1e-13, (key, dbar[c], ub)
        worst = max(worst, ub - dbar[c])
    assert worst <= 0.01
