"""CPU FP64 oracle of the barrier-filtered contact pass -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference leg
may import this package.  The library path never does.  It shares no code with
the CUDA path: the heavy loops live in oracle.c (brute force over all pairs,
hyper-dual derivatives, Jacobi PSD projection, additive CCD), this module only
orders the steps of the method (Sec. 3.2-3.4 of the paper) and assembles results.

Steps of one pass, in the paper's order:
  1. components and the stencil set K (non-incident PT / EE pairs)        Sec. 3.2
  2. reference distances dbar on the rest mesh, filtered set F (dbar < a),
     dbar_min = min over K of dbar                                          Sec. 3.2
  3. broad phase at the full, unmodified activation a (candidate set C)    Sec. 3.3
  4. class per candidate: F if in the filtered set, else U; class C for U
     pairs already within the offset (temporary eta = 0)                    Sec. 3.4
  5. distances; barrier Eq. 4 (Eq. 1 in single mode), gradient, Hessian   Eq. 2-4
     projected to PSD (projected Newton), assembled into g and BSR
  6. CCD candidates (swept boxes), additive CCD with per-class offsets,
     step bound alpha = min(1, min_p t_p)                                   Sec. 3.3

Options of contact_pass beside the paper's pass: mode "single" / "off" /
"kaldor" (Eq. 1, no filter, Kaldor culling), per_component (dbar_min per
component), mollifier (IPC's edge-edge mollifier), per_stencil (filtered
candidates kept at their own width), paper_literal (activation = thickness,
offset = thickness - dhat); rod scenes may mark closed loops
(scene.rod_closed: reference distances the shorter way round); shell
scenes may carry the flat pattern they are cut from (scene.rest_uv:
reference distances taken there) or ask for geodesic reference distances on
the rest mesh (scene.rest_geodesic, geodesic.c).  Lagged
friction on the active pairs: oracle/friction.py.

Pins: tests/test_oracle_*.py.  parity pinned for every function exported here.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SRCS = (_SRC, os.path.join(_HERE, "geodesic.c"))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

ROD_EE, PT, EE = 0, 1, 2
KLASS_U, KLASS_F, KLASS_C, KLASS_X = 0, 1, 2, 3   # X: culled (mode "kaldor")

# additive-CCD constants (C-IPC): minimum-separation fraction s, inner step factor
ACCD_S = 0.1
ACCD_INNER = 0.9
ACCD_MAX_ITER = 10000


def build(force: bool = False) -> str:
    """Compile oracle.c and geodesic.c with the system gcc (OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(map(os.path.getmtime, _SRCS)):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, *_SRCS, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Topo(C.Structure):
    _fields_ = [("kind", C.c_int), ("n", C.c_int), ("n_edges", C.c_int),
                ("edges", C.c_void_p), ("n_tris", C.c_int), ("tris", C.c_void_p),
                ("comp", C.c_void_p)]


class _Params(C.Structure):
    _fields_ = [("xi", C.c_double), ("dhat", C.c_double), ("kappa", C.c_double),
                ("dbar_min", C.c_double), ("single", C.c_int), ("core_temp", C.c_int),
                ("project", C.c_int), ("dbar_comp", C.c_void_p), ("moll_eps", C.c_void_p)]


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        vp, i64, dbl, i32 = C.c_void_p, C.c_int64, C.c_double, C.c_int
        L.orc_broad.restype = i64
        L.orc_broad.argtypes = [C.POINTER(_Topo), vp, vp, dbl, C.POINTER(vp)]
        L.orc_rest_filter.restype = i64
        L.orc_rest_filter.argtypes = [C.POINTER(_Topo), vp, dbl, vp, C.POINTER(vp), C.POINTER(vp)]
        L.orc_arclength.argtypes = [i32, vp, i32, vp, vp]
        L.orc_narrow.restype = i64
        L.orc_narrow.argtypes = [C.POINTER(_Topo), vp, C.POINTER(_Params), i64, vp, vp, vp, vp, vp,
                                 vp, C.POINTER(i32)]
        L.orc_barrier_pairs.argtypes = [C.POINTER(_Topo), vp, C.POINTER(_Params), i64, vp, vp, vp,
                                        vp, vp, vp, vp, vp]
        L.orc_ccd_pairs.argtypes = [C.POINTER(_Topo), vp, vp, i64, vp, vp, dbl, dbl, dbl, dbl, i32,
                                    vp, vp, vp]
        L.orc_free.argtypes = [vp]
        L.orc_distance.restype = i32
        L.orc_distance.argtypes = [i32, vp, C.POINTER(dbl)]
        L.orc_distance_derivs.argtypes = [i32, vp, i32, vp, vp]
        L.orc_barrier.argtypes = [dbl, dbl, C.POINTER(dbl), C.POINTER(dbl), C.POINTER(dbl)]
        L.orc_psd_project.restype = i32
        L.orc_psd_project.argtypes = [i32, vp, vp, vp]
        L.orc_accd.restype = i32
        L.orc_accd.argtypes = [i32, vp, vp, dbl, dbl, dbl, dbl, i32, C.POINTER(dbl), C.POINTER(i32)]
        L.orc_stencil.restype = i32
        L.orc_stencil.argtypes = [C.POINTER(_Topo), C.c_uint64, vp]
        L.orc_geo_source.restype = i32
        L.orc_geo_source.argtypes = [C.POINTER(_Topo), vp, dbl, i32, vp, vp]
        L.orc_geo_rest_filter.restype = i64
        L.orc_geo_rest_filter.argtypes = [C.POINTER(_Topo), vp, dbl, C.POINTER(vp), C.POINTER(vp)]
        L.orc_num_threads.restype = i32
        L.orc_set_num_threads.argtypes = [i32]
        _lib = L
    return _lib


def set_num_threads(n: int) -> int:
    """Threads of the oracle's parallel loops (for timing; results do not
    depend on it); returns the previous count."""
    prev = lib().orc_num_threads()
    lib().orc_set_num_threads(int(n))
    return prev


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


# ---------------------------------------------------------------------------
# Small single-stencil entry points (used by the pins)
# ---------------------------------------------------------------------------

def distance(is_ee: bool, x12) -> tuple[float, int]:
    """Distance and type of one stencil; x12 = 4 points (PT: p,t0,t1,t2;
    EE: a0,a1,b0,b1)."""
    x = np.ascontiguousarray(np.asarray(x12, np.float64).reshape(12))
    d = C.c_double()
    t = lib().orc_distance(int(is_ee), _ptr(x), C.byref(d))
    return d.value, int(t)


def distance_derivs(is_ee: bool, x12, type_: int) -> tuple[np.ndarray, np.ndarray]:
    x = np.ascontiguousarray(np.asarray(x12, np.float64).reshape(12))
    g = np.zeros(12)
    H = np.zeros(144)
    lib().orc_distance_derivs(int(is_ee), _ptr(x), int(type_), _ptr(g), _ptr(H))
    return g, H.reshape(12, 12)


def barrier(y: float, dhat: float) -> tuple[float, float, float]:
    b, b1, b2 = C.c_double(), C.c_double(), C.c_double()
    lib().orc_barrier(float(y), float(dhat), C.byref(b), C.byref(b1), C.byref(b2))
    return b.value, b1.value, b2.value


def psd_project(A) -> tuple[np.ndarray, np.ndarray, int]:
    A = np.ascontiguousarray(np.asarray(A, np.float64))
    n = A.shape[0]
    out = np.zeros_like(A)
    ev = np.zeros(n)
    sweeps = lib().orc_psd_project(n, _ptr(A), _ptr(out), _ptr(ev))
    return out, ev, sweeps


def accd(is_ee: bool, x12, p12, offset: float, s: float = ACCD_S, c_inner: float = ACCD_INNER,
         t_c: float = 1.0, max_iter: int = ACCD_MAX_ITER) -> tuple[float, int, int]:
    x = np.ascontiguousarray(np.asarray(x12, np.float64).reshape(12))
    p = np.ascontiguousarray(np.asarray(p12, np.float64).reshape(12))
    t = C.c_double()
    st = C.c_int()
    it = lib().orc_accd(int(is_ee), _ptr(x), _ptr(p), float(offset), s, c_inner, t_c, max_iter,
                        C.byref(t), C.byref(st))
    return t.value, int(st.value), int(it)


# ---------------------------------------------------------------------------
# Topology
# ---------------------------------------------------------------------------

@dataclass
class Topology:
    kind: int                 # 0 rods, 1 shells
    n: int
    edges: np.ndarray         # int32 (2, E), e0 < e1 for shells; (v, v+1) for rods
    tris: np.ndarray          # int32 (3, T) (empty for rods)
    comp: np.ndarray          # int32 (n,) component label per vertex
    _keep: list = field(default_factory=list)
    loop_ne: np.ndarray | None = None   # rods: per edge, the edge count of its closed loop (0: open polyline)

    def ctype(self) -> _Topo:
        e = np.ascontiguousarray(self.edges, np.int32)
        t = np.ascontiguousarray(self.tris, np.int32)
        c = np.ascontiguousarray(self.comp, np.int32)
        self._keep = [e, t, c]
        return _Topo(self.kind, self.n, e.shape[1], _ptr(e), t.shape[1], _ptr(t), _ptr(c))


def topology(scene) -> Topology:
    """Edges and connected components.  Shell edges: the unique (min, max)
    vertex pairs of the triangles in lexicographic order.  Rod edges: (v, v+1)
    within each polyline, polylines in order.  Components: shared vertices."""
    n = scene.n
    if scene.kind == "rod":
        rp = np.asarray(scene.rod_ptr, np.int64)
        closed = scene.rod_closed if getattr(scene, "rod_closed", None) is not None else np.zeros(rp.size - 1)
        e0, e1, lne = [], [], []
        for r in range(rp.size - 1):
            v = np.arange(rp[r], rp[r + 1] - 1)
            a, b = [v], [v + 1]
            ne = v.size
            if closed[r]:
                # closed loop: the edge from the last vertex back to the first, after the others
                a.append(np.array([rp[r + 1] - 1]))
                b.append(np.array([rp[r]]))
                ne += 1
            e0 += a
            e1 += b
            lne.append(np.full(ne, ne if closed[r] else 0))
        cat = lambda xs: np.concatenate(xs + [np.zeros(0, np.int64)])
        edges = np.stack([cat(e0), cat(e1)]).astype(np.int32)
        comp = np.zeros(n, np.int32)
        for r in range(rp.size - 1):
            comp[rp[r]:rp[r + 1]] = r
        return Topology(0, n, edges, np.zeros((3, 0), np.int32), comp, loop_ne=cat(lne).astype(np.int64))
    tris = np.asarray(scene.tris, np.int64)
    a = np.concatenate([tris[0], tris[1], tris[2]])
    b = np.concatenate([tris[1], tris[2], tris[0]])
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    key = np.unique(lo * n + hi)
    edges = np.stack([key // n, key % n]).astype(np.int32)
    # components by union-find over edges
    parent = np.arange(n)

    def find(i):
        while parent[i] != i:
            parent[i] = parent[parent[i]]
            i = parent[i]
        return i
    for u, v in zip(edges[0].tolist(), edges[1].tolist()):
        ru, rv = find(u), find(v)
        if ru != rv:
            parent[max(ru, rv)] = min(ru, rv)
    comp = np.array([find(i) for i in range(n)], np.int32)
    return Topology(1, n, edges, np.ascontiguousarray(tris.astype(np.int32)), comp)


def key_parts(keys: np.ndarray):
    keys = np.asarray(keys, np.uint64)
    return ((keys >> np.uint64(62)).astype(np.int64),
            ((keys >> np.uint64(31)) & np.uint64(0x7FFFFFFF)).astype(np.int64),
            (keys & np.uint64(0x7FFFFFFF)).astype(np.int64))


def stencils(topo: Topology, keys: np.ndarray) -> np.ndarray:
    """(m, 4) vertex ids of each pair (PT: p,t0,t1,t2; EE: a0,a1,b0,b1)."""
    t, i, j = key_parts(keys)
    out = np.zeros((keys.size, 4), np.int64)
    pt = t == PT
    if pt.any():
        out[pt, 0] = i[pt]
        out[pt, 1:] = topo.tris[:, j[pt]].T
    ee = ~pt
    if ee.any():
        out[ee, 0:2] = topo.edges[:, i[ee]].T
        out[ee, 2:4] = topo.edges[:, j[ee]].T
    return out


# ---------------------------------------------------------------------------
# Pass pieces
# ---------------------------------------------------------------------------

def _take(ptr: C.c_void_p, count: int, dtype) -> np.ndarray:
    if count == 0:
        lib().orc_free(ptr)
        return np.zeros(0, dtype)
    buf = (C.c_char * (count * np.dtype(dtype).itemsize)).from_address(ptr.value)
    arr = np.frombuffer(buf, dtype=dtype).copy()
    lib().orc_free(ptr)
    return arr


def broad_phase(topo: Topology, x: np.ndarray, h: float, p: np.ndarray | None = None) -> np.ndarray:
    """Sorted keys of all non-incident pairs whose boxes [min - h, max + h]
    overlap (static boxes of x, or swept boxes of x and x + p)."""
    tc = topo.ctype()
    x = np.ascontiguousarray(x, np.float64)
    pp = None if p is None else np.ascontiguousarray(p, np.float64)
    out = C.c_void_p()
    m = lib().orc_broad(C.byref(tc), _ptr(x), _ptr(pp), float(h), C.byref(out))
    return _take(out, m, np.uint64)


def arclength(scene) -> np.ndarray:
    rest = np.ascontiguousarray(scene.rest, np.float64)
    rp = np.ascontiguousarray(scene.rod_ptr, np.int32)
    S = np.zeros(scene.n)
    lib().orc_arclength(scene.n, _ptr(rest), rp.size - 1, _ptr(rp), _ptr(S))
    return S


def geodesic_from(scene, src: int, a: float, topo: Topology | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Geodesic distances on a shell's rest mesh from vertex src (geodesic.c):
    to every vertex (n,) and to every edge (E,), below a, +inf elsewhere."""
    topo = topo or topology(scene)
    tc = topo.ctype()
    rest = np.ascontiguousarray(scene.rest, np.float64)
    dv, de = np.zeros(topo.n), np.zeros(topo.edges.shape[1])
    rc = lib().orc_geo_source(C.byref(tc), _ptr(rest), float(a), int(src), _ptr(dv), _ptr(de))
    if rc != 0:
        raise ValueError("geodesic: non-manifold mesh" if rc == -1 else "geodesic: strip too long")
    return dv, de


def _geodesic_rest_filter(scene, topo: Topology, a: float) -> tuple[np.ndarray, np.ndarray]:
    tc = topo.ctype()
    rest = np.ascontiguousarray(scene.rest, np.float64)
    ok, od = C.c_void_p(), C.c_void_p()
    m = lib().orc_geo_rest_filter(C.byref(tc), _ptr(rest), float(a), C.byref(ok), C.byref(od))
    if m < 0:
        raise ValueError("geodesic: non-manifold mesh" if m == -1 else "geodesic: strip too long")
    return _take(ok, m, np.uint64), _take(od, m, np.float64)


def rest_filter(scene, topo: Topology, a: float) -> tuple[np.ndarray, np.ndarray]:
    """Filtered stencil pairs (same component, dbar < a) and their dbar."""
    if topo.kind == 0 and topo.loop_ne is not None and np.any(topo.loop_ne > 0):
        return _rod_rest_filter_loops(scene, topo, a)
    if topo.kind == 1 and getattr(scene, "rest_geodesic", False):
        # a doubly curved rest shell: geodesic distances on the rest mesh
        return _geodesic_rest_filter(scene, topo, a)
    tc = topo.ctype()
    rest = np.ascontiguousarray(scene.rest, np.float64)
    if topo.kind == 1 and getattr(scene, "rest_uv", None) is not None:
        # a shell cut from a flat pattern: the reference distance is taken in
        # the pattern (the geodesic distance of its developable rest shape)
        uv = np.asarray(scene.rest_uv, np.float64)
        rest = np.ascontiguousarray(np.vstack([uv, np.zeros((1, uv.shape[1]))]))
    S = arclength(scene) if topo.kind == 0 else np.zeros(1)
    ok, od = C.c_void_p(), C.c_void_p()
    m = lib().orc_rest_filter(C.byref(tc), _ptr(rest), float(a), _ptr(S), C.byref(ok), C.byref(od))
    return _take(ok, m, np.uint64), _take(od, m, np.float64)


def _rod_rest_filter_loops(scene, topo: Topology, a: float) -> tuple[np.ndarray, np.ndarray]:
    """Rod rest filter for scenes with closed loops, pair by pair within each
    polyline.  An edge runs from arc length s0 to s1 along its polyline (S at
    its vertices; a loop's closing edge ends at the loop length L = S at the
    last vertex plus the closing edge's length).  The reference distance of
    two non-incident edges k < l of one polyline is the arc-length gap
    between them, s0(l) - s1(k); on a closed loop the shorter way round,
    min(s0(l) - s1(k), (L - s1(l)) + s0(k))."""
    S = arclength(scene)
    rest = np.asarray(scene.rest, np.float64)
    e0, e1 = topo.edges[0].astype(np.int64), topo.edges[1].astype(np.int64)
    E = e0.size
    keys, dbs = [], []
    start = 0
    while start < E:
        r = topo.comp[e0[start]]
        stop = start
        while stop < E and topo.comp[e0[stop]] == r:
            stop += 1
        idx = np.arange(start, stop)
        s0 = S[e0[idx]]
        closing = e1[idx] < e0[idx]
        dv = rest[:, e1[idx]] - rest[:, e0[idx]]
        ln = np.sqrt((dv[0] * dv[0] + dv[1] * dv[1]) + dv[2] * dv[2])
        s1 = np.where(closing, s0 + ln, S[np.where(closing, e0[idx], e1[idx])])
        L = s1[closing][0] if closing.any() else None
        k, l = np.triu_indices(idx.size, 1)
        inc = ((e0[idx][k] == e0[idx][l]) | (e0[idx][k] == e1[idx][l]) | (e1[idx][k] == e0[idx][l])
               | (e1[idx][k] == e1[idx][l]))
        g = s0[l] - s1[k]
        if L is not None:
            g = np.minimum(g, (L - s1[l]) + s0[k])
        keep = (~inc) & (g < a)
        keys.append((idx[k][keep].astype(np.uint64) << np.uint64(31)) | idx[l][keep].astype(np.uint64))
        dbs.append(g[keep])
        start = stop
    K = np.concatenate(keys + [np.zeros(0, np.uint64)])
    D = np.concatenate(dbs + [np.zeros(0)])
    o = np.argsort(K)
    return K[o], D[o]


MODES = ("double", "single", "off", "kaldor")


def dbar_min_per_component(topo: Topology, F_rest: np.ndarray, dbar: np.ndarray) -> np.ndarray:
    """Smallest reference distance of the filtered stencil pairs of each
    component, indexed by component label (+inf where none is filtered)."""
    out = np.full(topo.n, np.inf)
    if F_rest.size:
        lab = topo.comp[stencils(topo, F_rest)[:, 0]]
        np.minimum.at(out, lab, dbar)
    return out


def kaldor_culled(topo: Topology, keys: np.ndarray, radius: int) -> np.ndarray:
    """Kaldor et al.'s culling, the comparison the paper runs against its
    filter (the knot test, Fig. 8): rod edge pairs of one polyline at most
    `radius` edges apart are removed from contact.  Edges are numbered
    consecutively along each polyline, so the gap is j - i (on a closed loop
    of m edges, min(j - i, m - (j - i)))."""
    keys = np.asarray(keys, np.uint64)
    i = ((keys >> np.uint64(31)) & np.uint64(0x7FFFFFFF)).astype(np.int64)
    j = (keys & np.uint64(0x7FFFFFFF)).astype(np.int64)
    e0 = topo.edges[0].astype(np.int64)
    same = topo.comp[e0[i]] == topo.comp[e0[j]]
    gap = j - i
    if topo.loop_ne is not None:
        ne = topo.loop_ne[i]
        gap = np.where(ne > 0, np.minimum(gap, ne - gap), gap)   # closed loop: the shorter way round
    return same & (gap <= radius)


@dataclass
class PassResult:
    C: np.ndarray            # candidate keys (sorted)
    klass: np.ndarray        # per candidate: 0 U, 1 F, 2 C
    d: np.ndarray            # per candidate distance at x
    dtype: np.ndarray        # per candidate distance type
    active: np.ndarray       # per candidate bool
    F_rest: np.ndarray       # rest-filtered keys
    dbar: np.ndarray         # their reference distances
    dbar_min: float
    energy: float
    pair_energy: np.ndarray  # per active pair
    grad: np.ndarray         # (3, n)
    grad_abs: np.ndarray     # (3, n) tolerance scale: sum of |contributions| (floored per pair)
    bsr_row_ptr: np.ndarray
    bsr_col: np.ndarray
    bsr_val: np.ndarray      # (nnzb, 3, 3)
    bsr_abs: np.ndarray      # (nnzb, 3, 3) tolerance scale, as grad_abs
    penetration: bool
    ccd_keys: np.ndarray | None = None
    ccd_klass: np.ndarray | None = None
    ccd_t: np.ndarray | None = None
    ccd_iters: np.ndarray | None = None
    ccd_status: np.ndarray | None = None
    alpha: float | None = None
    fwidth: np.ndarray | None = None  # per candidate: the class-F width (per_component passes)
    timings: dict = field(default_factory=dict)

    @property
    def active_keys(self):
        return self.C[self.active]

    def keys_of(self, k: int):
        return self.C[self.klass == k]


def mollifier_thresholds(scene, topo: Topology, keys: np.ndarray) -> np.ndarray:
    """eps_x = 1e-3 |rest e0|^2 |rest e1|^2 of each edge-edge key (0 for
    point-triangle keys): IPC's edge-edge mollifier threshold."""
    keys = np.asarray(keys, np.uint64)
    t, i, j = key_parts(keys)
    out = np.zeros(keys.size)
    ee = t != PT
    if ee.any():
        r = np.asarray(scene.rest, np.float64)
        e = topo.edges.astype(np.int64)
        def len2(k):
            dv = r[:, e[1, k]] - r[:, e[0, k]]
            return (dv * dv).sum(0)
        out[ee] = 1e-3 * len2(i[ee]) * len2(j[ee])
    return np.ascontiguousarray(out)


def _within_own_width(topo: Topology, x, keys, klass, dbar_comp, dbar_min: float) -> np.ndarray:
    """Per candidate: True unless it is filtered and its FP64 boxes, each
    inflated by half its own width, do not overlap (closed intervals)."""
    keep = np.ones(keys.size, bool)
    F = np.flatnonzero(klass == KLASS_F)
    if F.size == 0:
        return keep
    st = stencils(topo, keys[F])
    t, _, _ = key_parts(keys[F])
    pt = t == PT
    fw = dbar_comp[topo.comp[st[:, 0]]] if dbar_comp is not None else np.full(F.size, dbar_min)
    h = 0.5 * fw
    # first primitive: the point (PT) or edge (EE); second: the triangle or edge
    a = np.where(pt[:, None], st[:, [0, 0]], st[:, [0, 1]])
    b = np.where(pt[:, None], st[:, 1:4], st[:, [2, 3, 3]])
    lo1, hi1 = x[:, a].min(axis=2), x[:, a].max(axis=2)
    lo2, hi2 = x[:, b].min(axis=2), x[:, b].max(axis=2)
    ov = np.all((lo1 - h <= hi2 + h) & (lo2 - h <= hi1 + h), axis=0)
    keep[F] = ov
    return keep


def contact_pass(scene, mode: str = "double", core_temp: bool = True, project: bool = True,
                 ccd: bool = True, x: np.ndarray | None = None, p: np.ndarray | None = None,
                 topo: Topology | None = None, filt=None, cull_radius: int = 0,
                 per_component: bool = False, mollifier: bool = False, per_stencil: bool = False,
                 paper_literal: bool = False) -> PassResult:
    """One full pass (stages a-e) at x with CCD direction p.  Mode "kaldor":
    no filter, and rod edge pairs of one polyline at most cull_radius edges
    apart are culled (class X: no barrier, no constraint on the step).
    per_component: a filtered pair's width is the smallest reference distance
    of the filtered pairs of its own component instead of the scene's
    (dbar_min per component).  mollifier: edge-edge pairs take IPC's
    mollifier m(|e0 x e1|^2) with threshold 1e-3 |rest e0|^2 |rest e1|^2
    (the paper's solver uses IPC's contact energy, App. A).  per_stencil:
    each filtered candidate is kept only if its FP64 boxes, inflated by half
    of its own width (dbar_min, or its component's) instead of a / 2,
    overlap -- the per-stencil activation the paper leaves for later
    (Sec. 3.3); a filtered pair outside it is inactive, so only the
    candidate set changes.  paper_literal: the paper's own reading of the
    thickness h (Sec. 3.1 puts the activation at h, Sec. 3.3 splits it as
    eta + dhat): activation a = thickness and offset xi = thickness - dhat,
    instead of xi = thickness, a = thickness + dhat."""
    if mode == "kaldor" and (scene.kind != "rod" or cull_radius < 1):
        raise ValueError("kaldor mode: rods and cull_radius >= 1")
    import time
    tm = {}
    t0 = time.perf_counter()
    topo = topo or topology(scene)
    x = np.ascontiguousarray(scene.x if x is None else x, np.float64)
    p = np.ascontiguousarray(scene.p if p is None else p, np.float64)
    xi, dhat = offsets(scene, paper_literal)
    a = xi + dhat
    # (b) precompute: reference distances on the rest mesh
    if filt is None:
        F_rest, dbar = rest_filter(scene, topo, a)
    else:
        F_rest, dbar = filt
    dbar_min = float(dbar.min()) if dbar.size else math.inf
    tm["filter_precompute"] = time.perf_counter() - t0
    # (a) broad phase at the full activation: boxes inflated by a/2
    t1 = time.perf_counter()
    Cset = broad_phase(topo, x, 0.5 * a)
    tm["broad"] = time.perf_counter() - t1
    # (b) class
    t1 = time.perf_counter()
    if mode in ("off", "kaldor"):
        klass_in = np.zeros(Cset.size, np.uint8)
        if mode == "kaldor":
            klass_in[kaldor_culled(topo, Cset, cull_radius)] = KLASS_X
    else:
        klass_in = np.isin(Cset, F_rest).astype(np.uint8)
    tm["filter"] = time.perf_counter() - t1
    # (c) distances, class C, activity
    t1 = time.perf_counter()
    # per-component dbar_min by component label (the label of a pair's first vertex)
    dbar_comp = dbar_min_per_component(topo, F_rest, dbar) if per_component else None
    if per_stencil and Cset.size:
        keep = _within_own_width(topo, x, Cset, klass_in, dbar_comp,
                                 dbar_min if np.isfinite(dbar_min) else 0.0)
        Cset, klass_in = np.ascontiguousarray(Cset[keep]), np.ascontiguousarray(klass_in[keep])
    P = _Params(xi, dhat, float(scene.kappa), dbar_min if np.isfinite(dbar_min) else 0.0,
                int(mode == "single"), int(core_temp), int(project),
                dbar_comp.ctypes.data if dbar_comp is not None else None)
    tc = topo.ctype()
    m = Cset.size
    d = np.zeros(m)
    dty = np.zeros(m, np.int8)
    kl = np.zeros(m, np.uint8)
    act = np.zeros(m, np.uint8)
    pen = C.c_int(0)
    lib().orc_narrow(C.byref(tc), _ptr(x), C.byref(P), m, _ptr(Cset), _ptr(klass_in), _ptr(d),
                     _ptr(dty), _ptr(kl), _ptr(act), C.byref(pen))
    active = act.astype(bool)
    tm["distance"] = time.perf_counter() - t1
    # (d) barrier, derivatives, PSD projection, assembly
    t1 = time.perf_counter()
    ak = np.ascontiguousarray(Cset[active])
    na = ak.size
    e = np.zeros(na)
    g = np.zeros((na, 12))
    H = np.zeros((na, 144))
    hmax = np.zeros(na)
    akl = np.ascontiguousarray(kl[active])
    ad = np.ascontiguousarray(d[active])
    adt = np.ascontiguousarray(dty[active])
    if mollifier:
        meps = mollifier_thresholds(scene, topo, ak)
        P.moll_eps = meps.ctypes.data
    lib().orc_barrier_pairs(C.byref(tc), _ptr(x), C.byref(P), na, _ptr(ak), _ptr(akl), _ptr(ad),
                            _ptr(adt), _ptr(e), _ptr(g), _ptr(H), _ptr(hmax))
    energy = math.fsum(e.tolist()) if na else 0.0
    n = scene.n
    st = stencils(topo, ak)                                      # (na, 4)
    grad = np.zeros((3, n))
    grad_abs = np.zeros((3, n))
    gi = (np.arange(3)[None, None, :] * n + st[:, :, None]).reshape(-1)
    np.add.at(grad.reshape(-1), gi, g.reshape(-1))
    # tolerance scale: |contribution|, floored at 1e-4 of the pair's largest
    # entry (rounding of a pair's derivatives is relative to its norm)
    # conditioning of b', b'' in the computed distance d near the activation:
    # Eq. 2 is evaluated at y = d - xi_p, so a relative rounding u of d moves y
    # by u d, b'' (~ dhat_p - y) relatively by u kappa and b' (~ (dhat_p -
    # y)^2) by 2 u kappa, kappa = d / (dhat_p - y) (= y / (dhat_p - y) at
    # offset 0).  The floor covers about one ulp of d on either side times the
    # gradient's 2 kappa: 1e-9 f_p >= 2 kappa * 2.2e-16
    ad_xi = np.where(akl == KLASS_U, 0.0 if mode == "single" else xi, 0.0)
    fw = (dbar_comp[topo.comp[st[:, 0]]] if dbar_comp is not None
          else np.full(na, dbar_min if np.isfinite(dbar_min) else 0.0))
    ad_dh = np.where(akl == KLASS_F, fw, np.where((akl == KLASS_C) | (mode == "single"), a, dhat))
    ay = ad - ad_xi
    kappa_p = np.maximum(1.0, ad / np.maximum(ad_dh - ay, 1e-300)) if na else np.zeros(0)
    ffac = np.maximum(1e-4, 5e-7 * kappa_p)
    gfloor = (ffac * np.abs(g).max(axis=1))[:, None] if na else np.zeros((0, 1))
    np.add.at(grad_abs.reshape(-1), gi, np.maximum(np.abs(g), gfloor).reshape(-1))
    rows = np.repeat(st, 4, axis=1).reshape(-1)                  # r of (i, j)
    cols = np.tile(st, (1, 4)).reshape(-1)                       # c of (i, j)
    blk = H.reshape(na, 4, 3, 4, 3).transpose(0, 1, 3, 2, 4).reshape(-1, 3, 3)
    # floor: 1e-4 of the pair's largest Hessian entry BEFORE projection -- the
    # projection is 1-Lipschitz, so rounding in forming H carries into H+ at
    # the scale of H, however much of H the projection removes
    hfloor = ffac * np.maximum(hmax, np.abs(H).max(axis=1)) if na else np.zeros(0)
    blk_scale = np.maximum(np.abs(blk), np.repeat(hfloor, 16)[:, None, None])
    bkey = rows * n + cols
    ukeys, inv = np.unique(bkey, return_inverse=True)
    nnzb = ukeys.size
    val = np.zeros((nnzb, 3, 3))
    vab = np.zeros((nnzb, 3, 3))
    np.add.at(val, inv, blk)
    np.add.at(vab, inv, blk_scale)
    brow = (ukeys // n).astype(np.int64)
    bcol = (ukeys % n).astype(np.int32)
    row_ptr = np.zeros(n + 1, np.int64)
    np.add.at(row_ptr, brow + 1, 1)
    row_ptr = np.cumsum(row_ptr).astype(np.int32)
    tm["barrier"] = time.perf_counter() - t1
    res = PassResult(Cset, kl, d, dty, active, F_rest, dbar, dbar_min, energy, e, grad, grad_abs,
                     row_ptr, bcol, val, vab, bool(pen.value))
    if dbar_comp is not None:
        res.fwidth = dbar_comp[topo.comp[stencils(topo, Cset)[:, 0]]] if m else np.zeros(0)
    # (e) CCD step bound
    if ccd:
        t1 = time.perf_counter()
        ck, ckl, tt, it, cs = ccd_bound(scene, topo, x, p, F_rest, mode, core_temp, dbar_min, cull_radius,
                                        paper_literal)
        res.ccd_keys, res.ccd_klass, res.ccd_t, res.ccd_iters, res.ccd_status = ck, ckl, tt, it, cs
        res.alpha = float(min(1.0, tt.min())) if tt.size else 1.0
        tm["ccd"] = time.perf_counter() - t1
    res.timings = tm
    return res


def offsets(scene, paper_literal: bool = False) -> tuple[float, float]:
    """(xi, dhat): the offset and barrier width of a scene.  Default: xi =
    thickness, so the activation a = xi + dhat lies dhat beyond the
    thickness.  paper_literal: the activation is the thickness itself (the
    h of Eq. 1 and Eq. 4) and xi = thickness - dhat (Sec. 3.3: a = eta +
    dhat); a thickness below dhat is an error."""
    th, dhat = float(scene.thickness), float(scene.dhat)
    if not paper_literal:
        return th, dhat
    if th - dhat < 0.0:
        raise ValueError("paper_literal: thickness below dhat")
    return th - dhat, dhat


def ccd_bound(scene, topo, x, p, F_rest, mode="double", core_temp=True, dbar_min=0.0, cull_radius=0,
              paper_literal=False):
    """Swept broad phase with boxes of x and x+p inflated by xi/2, class of each
    pair at x (offset xi for U, 0 for F and C; culled pairs of mode "kaldor"
    do not constrain the step), additive CCD per pair."""
    xi, dhat = offsets(scene, paper_literal)
    off_u = 0.0 if mode == "single" else xi
    keys = broad_phase(topo, x, 0.5 * xi, p=p)
    m = keys.size
    klass_in = np.zeros(m, np.uint8) if mode in ("off", "kaldor") else np.isin(keys, F_rest).astype(np.uint8)
    if mode == "kaldor":
        klass_in[kaldor_culled(topo, keys, cull_radius)] = KLASS_X
    P = _Params(xi, dhat, float(scene.kappa), dbar_min if np.isfinite(dbar_min) else 0.0,
                int(mode == "single"), int(core_temp), 1)
    tc = topo.ctype()
    d = np.zeros(m)
    dty = np.zeros(m, np.int8)
    kl = np.zeros(m, np.uint8)
    act = np.zeros(m, np.uint8)
    pen = C.c_int(0)
    lib().orc_narrow(C.byref(tc), _ptr(x), C.byref(P), m, _ptr(keys), _ptr(klass_in), _ptr(d),
                     _ptr(dty), _ptr(kl), _ptr(act), C.byref(pen))
    t = np.zeros(m)
    it = np.zeros(m, np.int32)
    stt = np.zeros(m, np.int32)
    lib().orc_ccd_pairs(C.byref(tc), _ptr(x), _ptr(p), m, _ptr(keys), _ptr(kl), off_u, ACCD_S,
                        ACCD_INNER, 1.0, ACCD_MAX_ITER, _ptr(t), _ptr(stt), _ptr(it))
    return keys, kl, t, it, stt


def bsr_dense(res: PassResult, n: int) -> np.ndarray:
    """Dense 3n x 3n matrix of the BSR result (small cases only)."""
    A = np.zeros((3 * n, 3 * n))
    for r in range(n):
        for q in range(res.bsr_row_ptr[r], res.bsr_row_ptr[r + 1]):
            c = res.bsr_col[q]
            A[3 * r:3 * r + 3, 3 * c:3 * c + 3] = res.bsr_val[q]
    return A


def total_energy(scene, x, mode="double", core_temp=True, topo=None, filt=None, paper_literal=False) -> float:
    r = contact_pass(scene, mode=mode, core_temp=core_temp, ccd=False, x=x, topo=topo, filt=filt,
                     paper_literal=paper_literal)
    return r.energy
