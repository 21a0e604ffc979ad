"""Independent geometric helpers for the pins: closest points by dense sampling
plus pattern-search refinement (no formula shared with the oracle)."""
import numpy as np


def random_rotation(rng):
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def tri_points(t0, t1, t2, u, v):
    """Points of the triangle for barycentric (1-u-v, u, v), u,v >= 0, u+v <= 1."""
    return t0[None, :] + u[:, None] * (t1 - t0)[None, :] + v[:, None] * (t2 - t0)[None, :]


def closest_pt_search(p, t0, t1, t2, n=1000):
    """min over the triangle of |p - q| by a grid then a shrinking pattern search."""
    g = np.linspace(0.0, 1.0, n)
    U, V = np.meshgrid(g, g, indexing="ij")
    m = (U + V) <= 1.0
    u, v = U[m], V[m]
    d = np.linalg.norm(tri_points(t0, t1, t2, u, v) - p[None, :], axis=1)
    k = int(np.argmin(d))
    bu, bv, bd = u[k], v[k], d[k]
    h = 1.0 / n
    while h > 1e-13:
        improved = False
        for du, dv in ((h, 0), (-h, 0), (0, h), (0, -h), (h, -h), (-h, h)):
            nu, nv = bu + du, bv + dv
            if nu < 0 or nv < 0 or nu + nv > 1:
                nu, nv = max(nu, 0.0), max(nv, 0.0)
                s = nu + nv
                if s > 1:
                    nu, nv = nu / s, nv / s
            dd = np.linalg.norm(tri_points(t0, t1, t2, np.array([nu]), np.array([nv]))[0] - p)
            if dd < bd:
                bu, bv, bd, improved = nu, nv, dd, True
        if not improved:
            h *= 0.5
    return bd, bu, bv


def closest_ee_search(a0, a1, b0, b1, n=1000):
    g = np.linspace(0.0, 1.0, n)
    S, T = np.meshgrid(g, g, indexing="ij")
    s, t = S.ravel(), T.ravel()
    P = a0[None, :] + s[:, None] * (a1 - a0)[None, :]
    Q = b0[None, :] + t[:, None] * (b1 - b0)[None, :]
    d = np.linalg.norm(P - Q, axis=1)
    k = int(np.argmin(d))
    bs, bt, bd = s[k], t[k], d[k]
    h = 1.0 / n
    while h > 1e-13:
        improved = False
        for ds, dt in ((h, 0), (-h, 0), (0, h), (0, -h), (h, h), (-h, -h), (h, -h), (-h, h)):
            ns, nt = min(max(bs + ds, 0.0), 1.0), min(max(bt + dt, 0.0), 1.0)
            dd = np.linalg.norm(a0 + ns * (a1 - a0) - b0 - nt * (b1 - b0))
            if dd < bd:
                bs, bt, bd, improved = ns, nt, dd, True
        if not improved:
            h *= 0.5
    return bd, bs, bt
