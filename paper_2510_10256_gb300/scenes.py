"""Seeded synthetic scenes shaped like the paper's yarn and cloth workloads.

This module only *places* geometry: polylines, triangle grids, disks and random
displacements.  It holds none of the contact method's arithmetic (no distances,
no filter, no barrier), so both the CPU oracle and the CUDA path can take their
inputs from here without sharing any of the method.

Units are millimetres.  Positions are SoA float64 arrays of shape (3, n).

Workload shapes (paper Table 1 cloth, Table 2 yarn):
  * woven_patch   -- 8 warp + 8 weft open polylines, over/under weave (yarn, Table 2
                     thickness range 0.18-0.5 mm; here r = 0.1, thickness 2r).
  * pleated_sheet -- 256x256 regular triangle grid folded into tight pleats
                     (cloth, Table 1 sizes 10k-100k triangles).
  * graded_disk   -- graded Delaunay disk, 0.1 mm edges at the centre, 4 mm at the
                     rim, twisted about a diameter (cloth, the graded drape of Sec. 4).
  * rod_batch     -- 64 weave/knit rod scenes of log-uniform size.
  * tiny scenes   -- small random meshes for property tests.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

BASE_SEED = 20251010


@dataclass
class Scene:
    kind: str                      # "rod" or "shell"
    rest: np.ndarray               # (3, n) float64 reference (undeformed) positions
    x: np.ndarray                  # (3, n) float64 current positions
    p: np.ndarray                  # (3, n) float64 search direction for the CCD bound
    thickness: float               # xi: thickness offset (rods: 2r)
    dhat: float                    # barrier width; activation a = thickness + dhat
    rod_ptr: np.ndarray | None = None   # int32 (n_rods+1,) for rods
    tris: np.ndarray | None = None      # int32 (3, T) for shells
    kappa: float = 1.0
    name: str = ""
    seed: int = 0
    meta: dict = field(default_factory=dict)
    rod_closed: np.ndarray | None = None  # uint8 (n_rods,) for rods: 1 = closed loop (last vertex joins the first)
    rest_uv: np.ndarray | None = None     # (2, n) for shells: the flat pattern the rest shape is made from
    rest_geodesic: bool = False           # shells: reference distances are geodesic distances on the rest mesh

    @property
    def n(self) -> int:
        return int(self.rest.shape[1])

    @property
    def activation(self) -> float:
        return self.thickness + self.dhat


def _soa(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(3, -1))


# ---------------------------------------------------------------------------
# Rods
# ---------------------------------------------------------------------------

def woven_patch(seed: int = BASE_SEED + 1, n_warp: int = 8, n_weft: int = 8,
                nseg: int = 256, seg: float = 0.05, r: float = 0.1,
                spacing: float = 0.5, jitter_frac: float = 0.01,
                dhat: float = 0.01, sigma: float = 0.02) -> Scene:
    """Plain-weave patch of open polylines.

    Warp yarn j runs along x at y = spacing*j with height r*cos(pi*x/spacing + pi*j);
    weft yarn i runs along y at x = spacing*i with height -r*cos(pi*y/spacing + pi*i).
    At every crossing the two centrelines are exactly 2r apart before jitter.
    Every coordinate gets seeded uniform jitter of +-jitter_frac*r.  The jittered
    polylines are both the reference and the current configuration.
    """
    rng = np.random.default_rng(seed)
    length = nseg * seg
    centre = 0.5 * spacing * (max(n_warp, n_weft) - 1)
    s0 = centre - 0.5 * length
    # snap the start to the segment lattice so that vertices land on the crossings
    # (the spacing is a whole number of segments)
    s0 = seg * round(s0 / seg)
    k = np.arange(nseg + 1, dtype=np.float64)
    coords = []
    for j in range(n_warp):
        xs = s0 + seg * k
        ys = np.full_like(xs, spacing * j)
        zs = r * np.cos(np.pi * xs / spacing + np.pi * j)
        coords.append(np.stack([xs, ys, zs]))
    for i in range(n_weft):
        ys = s0 + seg * k
        xs = np.full_like(ys, spacing * i)
        zs = -r * np.cos(np.pi * ys / spacing + np.pi * i)
        coords.append(np.stack([xs, ys, zs]))
    pos = np.concatenate(coords, axis=1)
    pos = pos + rng.uniform(-jitter_frac * r, jitter_frac * r, size=pos.shape)
    n_rods = n_warp + n_weft
    rod_ptr = (np.arange(n_rods + 1) * (nseg + 1)).astype(np.int32)
    p = rng.normal(0.0, sigma, size=pos.shape)
    pos = _soa(pos)
    return Scene("rod", pos.copy(), pos.copy(), _soa(p), 2.0 * r, dhat, rod_ptr=rod_ptr,
                 name="woven_patch", seed=seed,
                 meta=dict(n_warp=n_warp, n_weft=n_weft, nseg=nseg, seg=seg, r=r,
                           spacing=spacing, sigma=sigma))


def _helix_row(x0: float, y0: float, n_vert: int, seg: float, radius: float,
               pitch: float) -> np.ndarray:
    """Helix along +x: (x0 + pitch*t/2pi, y0 + R cos t, R sin t), sampled at equal
    parameter steps chosen so that the chord is close to `seg`."""
    per_turn_len = math.hypot(2 * math.pi * radius, pitch)
    dt = 2 * math.pi * seg / per_turn_len
    t = dt * np.arange(n_vert)
    return np.stack([x0 + pitch * t / (2 * math.pi),
                     y0 + radius * np.cos(t), radius * np.sin(t)])


def _min_helix_gap(radius: float, pitch: float, dy: float) -> float:
    """Closest approach of two parallel helices, the second shifted by dy across
    and half a pitch along the axis: a coarse parameter grid, then three local
    zooms around the best cell (each 10x finer)."""
    def pts(t, shift, y0):
        return (shift + pitch * t / (2 * math.pi), y0 + radius * np.cos(t), radius * np.sin(t))

    def grid_min(t, s):
        ax, ay, az = pts(t, 0.0, 0.0)
        bx, by, bz = pts(s, 0.5 * pitch, dy)
        d2 = (ax[:, None] - bx[None, :]) ** 2 + (ay[:, None] - by[None, :]) ** 2 + \
            (az[:, None] - bz[None, :]) ** 2
        i, j = np.unravel_index(int(np.argmin(d2)), d2.shape)
        return float(d2[i, j]), float(t[i]), float(s[j])

    ht, hs = 2 * math.pi / 180, 6 * math.pi / 540
    best, t0, s0 = grid_min(np.linspace(0.0, 2 * math.pi, 181), np.linspace(-2 * math.pi, 4 * math.pi, 541))
    for _ in range(3):
        best, t0, s0 = grid_min(np.linspace(t0 - ht, t0 + ht, 21), np.linspace(s0 - hs, s0 + hs, 21))
        ht, hs = ht / 10, hs / 10
    return math.sqrt(best)


def knit_rows(seed: int, n_target: int, r: float, seg: float, dhat: float,
              sigma: float) -> Scene:
    """Interlocking-loop knit: rows of helices (radius 2r, pitch 4r) along x, each
    row half a pitch ahead of the previous one, rows spaced so that neighbouring
    loops pass at a seeded gap in [0.97, 1.03] x thickness."""
    rng = np.random.default_rng(seed)
    radius, pitch, thick = 2.0 * r, 4.0 * r, 2.0 * r
    target = thick * rng.uniform(0.97, 1.03)
    lo, hi = 0.0, 4.0 * radius + thick
    for _ in range(50):
        mid = 0.5 * (lo + hi)
        if _min_helix_gap(radius, pitch, mid) < target:
            lo = mid
        else:
            hi = mid
    dy = hi
    n_rows = max(2, int(round(math.sqrt(n_target / 60.0))))
    per_row = max(8, n_target // n_rows)
    rows = []
    for k in range(n_rows):
        rows.append(_helix_row(0.5 * pitch * (k % 2), dy * k, per_row, seg, radius, pitch))
    pos = np.concatenate(rows, axis=1)
    rod_ptr = (np.arange(n_rows + 1) * per_row).astype(np.int32)
    p = rng.normal(0.0, sigma, size=pos.shape)
    pos = _soa(pos)
    return Scene("rod", pos.copy(), pos.copy(), _soa(p), thick, dhat, rod_ptr=rod_ptr,
                 name="knit_rows", seed=seed,
                 meta=dict(r=r, seg=seg, rows=n_rows, per_row=per_row, dy=dy))


def weave_sized(seed: int, n_target: int, r: float, seg: float, dhat: float,
                sigma: float) -> Scene:
    """Plain weave with about n_target vertices: square patch, yarn spacing 5r."""
    spacing = 5.0 * r
    n_y = max(2, int(round(math.sqrt(n_target * seg / (2 * spacing)))))
    nseg = max(8, int(round(n_target / (2 * n_y))) - 1)
    # keep crossings on vertices: spacing must be a multiple of seg
    seg = spacing / max(1, round(spacing / seg))
    sc = woven_patch(seed=seed, n_warp=n_y, n_weft=n_y, nseg=nseg, seg=seg, r=r,
                     spacing=spacing, dhat=dhat, sigma=sigma)
    sc.name = "weave_sized"
    return sc


def rod_batch(seed: int = BASE_SEED + 4, n_scenes: int = 64, n_lo: float = 1e3,
              n_hi: float = 6.4e4) -> list[Scene]:
    """Batch of rod scenes: sizes log-uniform in [n_lo, n_hi] vertices, yarn radius
    U[0.05, 0.3], segment U[0.2r, 1.0r], dhat = 0.1r; even index weave, odd knit."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_scenes):
        n_t = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        r = float(rng.uniform(0.05, 0.3))
        seg = float(rng.uniform(0.2 * r, 1.0 * r))
        if i % 2 == 0:
            sc = weave_sized(seed + 1000 + i, n_t, r, seg, 0.1 * r, sigma=0.2 * r)
        else:
            sc = knit_rows(seed + 1000 + i, n_t, r, seg, 0.1 * r, sigma=0.2 * r)
        out.append(sc)
    return out


def serve_pool(seed: int = BASE_SEED + 5, n_rod: int = 8, n_shell: int = 8, rod_lo: float = 5e3,
               rod_hi: float = 2e5, tri_lo: float = 1e4, tri_hi: float = 5e5) -> list[Scene]:
    """Scenes a served request stream draws from: rods with vertex counts and
    shells with triangle counts log-uniform in the given ranges, seeded.  Rods
    take the woven-patch parameters (r 0.1, segment 0.05, dhat 0.01, sigma
    0.02), alternately plain weave and helix-loop knit; shells alternate the
    pleated sheet (L 0.5, thickness 1, dhat 0.05, sigma 0.1) and the graded
    twisted disk (0.1-4 mm edges, same thickness and dhat)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_rod):
        n_t = int(round(math.exp(rng.uniform(math.log(rod_lo), math.log(rod_hi)))))
        if i % 2 == 0:
            sc = weave_sized(seed + 100 + i, n_t, 0.1, 0.05, 0.01, 0.02)
        else:
            sc = knit_rows(seed + 100 + i, n_t, 0.1, 0.05, 0.01, 0.02)
        sc.meta = dict(sc.meta or {}, sigma=0.02)
        out.append(sc)
    for i in range(n_shell):
        T = int(round(math.exp(rng.uniform(math.log(tri_lo), math.log(tri_hi)))))
        if i % 2 == 0:
            nx = max(8, int(round(1 + math.sqrt(T / 2.0))))
            sc = pleated_sheet(seed=seed + 200 + i, nx=nx)
        else:
            sc = graded_disk(seed=seed + 200 + i, target_tris=T)
        sc.meta = dict(sc.meta or {}, sigma=0.1)
        out.append(sc)
    return out


def straight_rod(n_seg: int = 20, seg: float = 0.1, thickness: float = 0.25,
                 dhat: float = 0.05) -> Scene:
    """One straight uniform polyline along x (no jitter)."""
    xs = seg * np.arange(n_seg + 1, dtype=np.float64)
    pos = np.stack([xs, np.zeros_like(xs), np.zeros_like(xs)])
    return Scene("rod", pos.copy(), pos.copy(), np.zeros_like(pos), thickness, dhat,
                 rod_ptr=np.array([0, n_seg + 1], np.int32), name="straight_rod")


# ---------------------------------------------------------------------------
# Shells
# ---------------------------------------------------------------------------

def grid_mesh(nx: int, ny: int, L: float) -> tuple[np.ndarray, np.ndarray]:
    """Regular nx x ny vertex grid, centred at the origin, consistent diagonal.
    Vertex (i, j) has index j*nx + i; each quad is split along (i,j)-(i+1,j+1)."""
    i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    X = (i.astype(np.float64) - 0.5 * (nx - 1)) * L
    Y = (j.astype(np.float64) - 0.5 * (ny - 1)) * L
    pos = np.stack([X.ravel(), Y.ravel(), np.zeros(nx * ny)])
    qi, qj = np.meshgrid(np.arange(nx - 1), np.arange(ny - 1), indexing="xy")
    v00 = (qj * nx + qi).ravel()
    v10 = v00 + 1
    v01 = v00 + nx
    v11 = v01 + 1
    t1 = np.stack([v00, v10, v11])
    t2 = np.stack([v00, v11, v01])
    tris = np.empty((3, 2 * v00.size), np.int64)
    tris[:, 0::2] = t1
    tris[:, 1::2] = t2
    return pos, tris.astype(np.int32)


def _fold_profile(s_lo: float, s_hi: float, amps, lams, phis, c: float, ds: float):
    """Planar curve parametrised by arc length whose tangent angle is
    theta(s) = c * sum_k (2 pi A_k / lam_k) sin(2 pi s / lam_k + phi_k)."""
    s = np.arange(s_lo, s_hi + ds, ds)
    th = np.zeros_like(s)
    for A, lam, ph in zip(amps, lams, phis):
        th += (2 * math.pi * A / lam) * np.sin(2 * math.pi * s / lam + ph)
    th *= c
    cx, cz = np.cos(th), np.sin(th)
    px = np.concatenate([[0.0], np.cumsum(0.5 * (cx[1:] + cx[:-1]) * ds)])
    pz = np.concatenate([[0.0], np.cumsum(0.5 * (cz[1:] + cz[:-1]) * ds)])
    return s, px, pz


def _profile_min_gap(s, px, pz, sep: float, step: int) -> float:
    """Smallest chord between curve samples at least `sep` apart in arc length."""
    ss, xx, zz = s[::step], px[::step], pz[::step]
    best = np.inf
    m = ss.size
    for a in range(0, m, 512):
        b = min(m, a + 512)
        dx = xx[a:b, None] - xx[None, :]
        dz = zz[a:b, None] - zz[None, :]
        d = np.hypot(dx, dz)
        far = np.abs(ss[a:b, None] - ss[None, :]) >= sep
        if far.any():
            best = min(best, float(d[far].min()))
    return best


def pleated_sheet(seed: int = BASE_SEED + 2, nx: int = 256, L: float = 0.5,
                  thickness: float = 1.0, dhat: float = 0.05, sigma: float = 0.1,
                  gap_lo: float = 0.9, gap_hi: float = 1.0) -> Scene:
    """Flat nx x nx grid (rest) folded into three superposed sinusoidal pleats.

    The fold keeps arc length along a seeded in-plane direction u (a developable
    bend): the cross-section is the curve whose tangent angle is a sum of three
    sines (amplitudes A_k in U[2,5] mm, wavelengths lam_k in U[3,8] mm, seeded
    phases), extruded along the perpendicular direction.  A single scale c on the
    angle is chosen by bisection so that the closest approach between curve points
    at least one activation distance apart in arc length equals a seeded target in
    [gap_lo, gap_hi] x thickness: folded layers come within thickness, nothing
    intersects.  (A pure height field could never do this: projection onto the rest
    plane shortens distances, so 3D distances would never drop below rest ones.)
    """
    rng = np.random.default_rng(seed)
    rest, tris = grid_mesh(nx, nx, L)
    amps = rng.uniform(2.0, 5.0, 3)
    lams = rng.uniform(3.0, 8.0, 3)
    phis = rng.uniform(0.0, 2 * math.pi, 3)
    ang = rng.uniform(0.0, math.pi)
    target = thickness * rng.uniform(gap_lo, gap_hi)
    u = np.array([math.cos(ang), math.sin(ang)])
    v = np.array([-math.sin(ang), math.cos(ang)])
    s_v = u[0] * rest[0] + u[1] * rest[1]
    t_v = v[0] * rest[0] + v[1] * rest[1]
    s_lo, s_hi = float(s_v.min()) - 1.0, float(s_v.max()) + 1.0
    act = thickness + dhat
    ds = 0.01
    step = 10

    def gap(c):
        s, px, pz = _fold_profile(s_lo, s_hi, amps, lams, phis, c, ds)
        return _profile_min_gap(s, px, pz, act, step)

    lo, hi = 0.0, 1.0
    if gap(hi) >= target:
        c = hi
    else:
        for _ in range(40):
            mid = 0.5 * (lo + hi)
            if gap(mid) > target:
                lo = mid
            else:
                hi = mid
        c = lo
    s, px, pz = _fold_profile(s_lo, s_hi, amps, lams, phis, c, ds)
    fx = np.interp(s_v, s, px)
    fz = np.interp(s_v, s, pz)
    fx -= 0.5 * (fx.max() + fx.min())
    x = np.stack([fx * u[0] + t_v * v[0], fx * u[1] + t_v * v[1], fz])
    p = rng.normal(0.0, sigma, size=x.shape)
    return Scene("shell", _soa(rest), _soa(x), _soa(p), thickness, dhat, tris=tris,
                 name="pleated_sheet", seed=seed,
                 meta=dict(nx=nx, L=L, amps=amps.tolist(), lams=lams.tolist(),
                           phis=phis.tolist(), angle=ang, scale=c, target_gap=target,
                           min_gap=gap(c), sigma=sigma))


def graded_points(R: float, L0: float, L1: float, rng: np.random.Generator,
                  jitter: float = 0.15) -> np.ndarray:
    """Graded point set on a disk of radius R: rings whose spacing and in-ring
    spacing follow L(rho) = L0 + (L1 - L0) rho / R, with seeded jitter of
    `jitter` x L in radius and angle (a cheap stand-in for graded Poisson-disk
    sampling with the same local spacing)."""
    pts = [np.zeros((2, 1))]
    rho = 0.0
    while True:
        Lr = L0 + (L1 - L0) * rho / R
        rho = rho + 0.8660254037844386 * Lr
        if rho > R:
            break
        Lr = L0 + (L1 - L0) * rho / R
        m = max(6, int(round(2 * math.pi * rho / Lr)))
        th = 2 * math.pi * (np.arange(m) + rng.uniform(0, 1)) / m
        rr = np.full(m, rho)
        if rho < R - 0.5 * Lr:
            rr = rr + rng.uniform(-jitter, jitter, m) * Lr
            th = th + rng.uniform(-jitter, jitter, m) * Lr / rho
        pts.append(np.stack([rr * np.cos(th), rr * np.sin(th)]))
    return np.concatenate(pts, axis=1)


def graded_disk(seed: int = BASE_SEED + 3, target_tris: int = 200_000, L0: float = 0.1,
                L1: float = 4.0, thickness: float = 1.0, dhat: float = 0.05,
                sigma: float = 0.1, turns: float = 1.0) -> Scene:
    """Graded Delaunay disk (edge length L0 at the centre, L1 at the rim) twisted
    by turns*360 degrees about the in-plane x axis, angle growing linearly along x."""
    from scipy.spatial import Delaunay
    rng = np.random.default_rng(seed)
    # points ~ 1.294 R^2 for L0=0.1, L1=4 ; triangles ~ 2x points
    coef = 2.0 * 1.294 * (0.1 / L0) ** 0.0
    R = math.sqrt(target_tris / coef)
    pts = graded_points(R, L0, L1, rng)
    tri = Delaunay(pts.T)
    tris = np.ascontiguousarray(tri.simplices.T.astype(np.int32))
    # orient counter-clockwise in the rest plane
    a, b, c = pts[:, tris[0]], pts[:, tris[1]], pts[:, tris[2]]
    cr = (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])
    flip = cr < 0
    tris[1, flip], tris[2, flip] = tris[2, flip].copy(), tris[1, flip].copy()
    rest = np.stack([pts[0], pts[1], np.zeros(pts.shape[1])])
    xmin, xmax = rest[0].min(), rest[0].max()
    th = 2 * math.pi * turns * (rest[0] - xmin) / (xmax - xmin)
    x = np.stack([rest[0], rest[1] * np.cos(th), rest[1] * np.sin(th)])
    p = rng.normal(0.0, sigma, size=x.shape)
    return Scene("shell", _soa(rest), _soa(x), _soa(p), thickness, dhat, tris=tris,
                 name="graded_disk", seed=seed,
                 meta=dict(R=R, L0=L0, L1=L1, turns=turns, sigma=sigma,
                           n_tris=int(tris.shape[1])))


def flat_grid(nx: int = 8, L: float = 0.5, thickness: float = 1.0,
              dhat: float = 0.05) -> Scene:
    """Flat regular grid at rest (current = rest)."""
    rest, tris = grid_mesh(nx, nx, L)
    return Scene("shell", _soa(rest), _soa(rest.copy()), np.zeros_like(rest), thickness,
                 dhat, tris=tris, name="flat_grid")


def rolled_sheet(seed: int = BASE_SEED + 8, nx: int = 24, ny: int = 12, L: float = 0.25, radius: float = 1.5,
                 thickness: float = 0.4, dhat: float = 0.05, sigma: float = 0.05, layers: int = 2) -> Scene:
    """Sheets cut from a flat nx x ny grid pattern (edge L) and rolled at rest
    onto coaxial cylinders (the outer one thickness + 0.6 dhat further out),
    so their rest shape is curved while their pattern is flat: reference
    distances are taken in the pattern (rest_uv).  Current positions: the
    rest shape plus a little noise; p: Gaussian."""
    rng = np.random.default_rng(seed)
    pat, t = grid_mesh(nx, ny, L)
    rest_l, tris_l, uv_l = [], [], []
    for k in range(layers):
        R = radius + k * (thickness + 0.6 * dhat)
        ang = pat[0] / radius   # same angles for every layer: the pattern is rolled, not stretched
        rest_l.append(np.stack([R * np.sin(ang), pat[1], radius - R * np.cos(ang)]))
        tris_l.append(t + k * pat.shape[1])
        uv_l.append(pat[:2])
    rest = np.concatenate(rest_l, axis=1)
    tris = np.concatenate(tris_l, axis=1).astype(np.int32)
    x = rest + rng.normal(0.0, 0.01 * dhat, size=rest.shape)
    p = rng.normal(0.0, sigma, size=rest.shape)
    return Scene("shell", _soa(rest), _soa(x), _soa(p), thickness, dhat, tris=tris, name="rolled_sheet", seed=seed,
                 rest_uv=np.ascontiguousarray(np.concatenate(uv_l, axis=1)))


def curved_sheet(seed: int = BASE_SEED + 9, shape: str = "dome", nx: int = 32, L: float = 0.05,
                 curvature: float = 1.0, thickness: float = 0.06, dhat: float = 0.01, layers: int = 2,
                 sigma: float = 0.02) -> Scene:
    """Doubly curved rest shells with geodesic reference distances
    (rest_geodesic): `layers` nested copies of an nx x nx grid (edge about L)
    laid on a sphere of radius 1 / curvature ("dome", positive Gaussian
    curvature; the grid's distance from its centre kept as arc length) or on
    the saddle z = curvature (x^2 - y^2) / 2 ("saddle", negative), each copy
    offset along the surface normal by thickness +
    0.6 dhat.  The activation thickness + dhat spans about 1.4 edges, so
    stencils of one sheet lie within it at rest.  Current positions: the rest
    shape plus a little noise; p: Gaussian."""
    rng = np.random.default_rng(seed)
    pat, t = grid_mesh(nx, nx, L)
    u, v = pat[0], pat[1]
    rest_l, tris_l = [], []
    for k in range(layers):
        off = k * (thickness + 0.6 * dhat)
        if shape == "dome":
            # azimuthal equidistant: the grid's distance from the centre is the arc length
            R = 1.0 / curvature
            th = np.hypot(u, v) / R
            ph = np.arctan2(v, u)
            nrm = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
            pos = (R + off) * nrm - np.array([[0.0], [0.0], [R]])
        elif shape == "saddle":
            z = 0.5 * curvature * (u * u - v * v)
            g = np.stack([-curvature * u, curvature * v, np.ones(u.size)])
            nrm = g / np.linalg.norm(g, axis=0)
            pos = np.stack([u, v, z]) + off * nrm
        else:
            raise ValueError(shape)
        rest_l.append(pos)
        tris_l.append(t + k * u.size)
    rest = np.concatenate(rest_l, axis=1)
    tris = np.concatenate(tris_l, axis=1).astype(np.int32)
    x = rest + rng.normal(0.0, 0.01 * dhat, size=rest.shape)
    p = rng.normal(0.0, sigma, size=rest.shape)
    return Scene("shell", _soa(rest), _soa(x), _soa(p), thickness, dhat, tris=tris, name=f"{shape}_sheet",
                 seed=seed, rest_geodesic=True)


def tiny_shell(seed: int, nx: int = 5, L: float = 0.3, thickness: float = 0.4,
               dhat: float = 0.1, noise: float = 0.08, layers: int = 2,
               sigma: float = 0.1) -> Scene:
    """Small stacked grids (separate components) with seeded noise: a property-test
    scene where cross-layer pairs, stencil neighbours and near-threshold pairs
    all occur."""
    rng = np.random.default_rng(seed)
    rs, ts, off = [], [], 0
    for k in range(layers):
        r, t = grid_mesh(nx, nx, L)
        r = r.copy()
        r[2] += k * (thickness + 0.5 * dhat)
        r[0] += rng.uniform(-L, L)
        rs.append(r)
        ts.append(t + off)
        off += r.shape[1]
    rest = np.concatenate(rs, axis=1)
    tris = np.concatenate(ts, axis=1).astype(np.int32)
    x = rest + rng.uniform(-noise, noise, size=rest.shape)
    x[2] += rng.uniform(-0.5 * noise, 0.5 * noise, size=x.shape[1])
    p = rng.normal(0.0, sigma, size=x.shape)
    return Scene("shell", _soa(rest), _soa(x), _soa(p), thickness, dhat, tris=tris,
                 name="tiny_shell", seed=seed)


def tiny_rods(seed: int, n_rods: int = 3, nseg: int = 12, seg: float = 0.1,
              thickness: float = 0.2, dhat: float = 0.05, sigma: float = 0.05) -> Scene:
    """A few short wiggly polylines laid across each other."""
    rng = np.random.default_rng(seed)
    polys = []
    for r in range(n_rods):
        ang = rng.uniform(0, math.pi)
        d = np.array([math.cos(ang), math.sin(ang), 0.0])
        start = rng.uniform(-0.3, 0.3, 3) - 0.5 * nseg * seg * d
        start[2] = (r - 0.5 * (n_rods - 1)) * (thickness + 0.3 * dhat)
        steps = np.cumsum(np.vstack([np.zeros(3)] + [seg * d + rng.uniform(-0.3, 0.3, 3) * seg
                                                     for _ in range(nseg)]), axis=0)
        polys.append((start + steps).T)
    pos = np.concatenate(polys, axis=1)
    rod_ptr = (np.arange(n_rods + 1) * (nseg + 1)).astype(np.int32)
    p = rng.normal(0.0, sigma, size=pos.shape)
    pos = _soa(pos)
    return Scene("rod", pos.copy(), pos.copy(), _soa(p), thickness, dhat, rod_ptr=rod_ptr,
                 name="tiny_rods", seed=seed)


def polygon_loop(m: int, R: float = 1.0, closed: bool = True, thickness: float = 0.3,
                 dhat: float = 0.05) -> Scene:
    """One regular m-gon of circumradius R in the xy-plane (a closed yarn
    loop, or the same vertices as an open polyline)."""
    th = 2.0 * math.pi * np.arange(m) / m
    x = np.stack([R * np.cos(th), R * np.sin(th), np.zeros(m)])
    return Scene("rod", x.copy(), x.copy(), np.zeros_like(x), thickness, dhat,
                 rod_ptr=np.array([0, m], np.int32), name=f"polygon{m}{'' if closed else '_open'}",
                 rod_closed=np.array([1 if closed else 0], np.uint8))


def ring_chain(seed: int = BASE_SEED + 7, n_rings: int = 3, m: int = 48, R: float = 1.0,
               thickness: float = 0.3, dhat: float = 0.05, sigma: float = 0.15) -> Scene:
    """Interlocked closed rings (a chain: ring i in the xy-plane for even i,
    the xz-plane for odd i, centres along x).  Rest: centres 1.6 R apart.
    Current positions: the rings pulled apart (each translated along x)
    until neighbouring rings' vertices come within thickness + 0.6 dhat,
    plus a little noise; p: Gaussian."""
    rng = np.random.default_rng(seed)

    def ring(i, spacing):
        th = 2.0 * math.pi * np.arange(m) / m + 0.37 * i
        c, s_ = R * np.cos(th), R * np.sin(th)
        z = np.zeros(m)
        pts = np.stack([c, s_, z]) if i % 2 == 0 else np.stack([c, z, s_])
        pts[0] += i * spacing
        return pts

    def min_gap(spacing):
        a, b = ring(0, spacing), ring(1, spacing)
        d = a[:, :, None] - b[:, None, :]
        return float(np.sqrt((d * d).sum(0)).min())

    target = thickness + 0.6 * dhat
    lo, hi = 1.6 * R, 2.0 * R   # linked rings: the gap shrinks as they are pulled apart
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if min_gap(mid) > target:
            lo = mid
        else:
            hi = mid
    rest = np.concatenate([ring(i, 1.6 * R) for i in range(n_rings)], axis=1)
    x = np.concatenate([ring(i, lo) for i in range(n_rings)], axis=1)
    x = x + rng.normal(0.0, 0.01 * dhat, size=x.shape)
    p = rng.normal(0.0, sigma, size=x.shape)
    rp = np.arange(0, (n_rings + 1) * m, m, dtype=np.int32)
    return Scene("rod", rest, x, p, thickness, dhat, rod_ptr=rp, name=f"ring_chain{n_rings}x{m}", seed=seed,
                 rod_closed=np.ones(n_rings, np.uint8))


# ---------------------------------------------------------------------------
# Named configurations
# ---------------------------------------------------------------------------

def config(cid: int, reduced: bool = False) -> Scene | list[Scene]:
    """The five workloads; `reduced` gives a small case with the same recipe."""
    if cid == 1:
        if reduced:
            return woven_patch(n_warp=3, n_weft=3, nseg=64)
        return woven_patch()
    if cid == 2:
        return pleated_sheet(nx=48 if reduced else 256)
    if cid == 3:
        return graded_disk(target_tris=6000 if reduced else 200_000,
                           L0=0.1 if not reduced else 0.5)
    if cid == 4:
        return rod_batch(n_scenes=4 if reduced else 64, n_hi=4e3 if reduced else 6.4e4)
    raise ValueError(cid)
