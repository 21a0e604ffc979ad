"""Thin ctypes binding of libcontact.so (include/contact.h).

Argument marshalling only: every stage of the pass runs in the library's CUDA
kernels.  Device buffers are torch CUDA tensors (FP64, SoA [3][n]); streams are
torch streams.  There is no CPU fallback: if the library cannot be loaded the
import of the pass functions raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcontact.so")
_lib = None

CB_OK, CB_ERR_ARG, CB_ERR_OOM, CB_ERR_CAPACITY, CB_ERR_PENETRATION, CB_ERR_DEGENERATE, \
    CB_ERR_ITER_LIMIT, CB_ERR_CUDA, CB_ERR_TOO_LARGE = range(9)
CB_ROD, CB_SHELL = 0, 1
CB_FILTER_DOUBLE, CB_FILTER_SINGLE, CB_FILTER_OFF, CB_FILTER_KALDOR = 0, 1, 2, 3
CB_THICK_PAPER_LITERAL = 4
CB_NO_CORE_TEMP = 8
CB_DBAR_PER_COMPONENT = 16
CB_EE_MOLLIFIER = 32
CB_PER_STENCIL = 64
CB_DBAR_GEODESIC = 128
PAIRS = {"candidate": 0, "filtered": 1, "core": 2, "active": 3, "ccd": 4, "rest_filtered": 5}
MODES = {"double": CB_FILTER_DOUBLE, "single": CB_FILTER_SINGLE, "off": CB_FILTER_OFF, "kaldor": CB_FILTER_KALDOR}

# names declared in include/contact.h (the tests check the library exports each)
ABI_FUNCTIONS = ["cb_scene_create", "cb_scene_destroy", "contact_build", "contact_filter", "barrier_eval",
                 "ccd_step", "cb_get_pairs", "cb_get_active", "cb_get_ccd", "cb_get_bsr", "cb_bsr_device",
                 "cb_get_stats", "cb_sync_status", "cb_get_stage_ms", "cb_get_stage_times", "cb_set_timing", "cb_status_str",
                 "cb_version", "cb_kernel_launches", "cb_measure_fma_tflops", "cb_batch_create",
                 "cb_batch_offsets", "cb_member_count", "ccd_step_noalloc", "cb_set_tuning",
                 "cb_get_tuning", "barrier_energy", "cb_bsr_spmv", "friction_lag", "friction_eval",
                 "friction_spmv", "cb_get_friction", "cb_server_create", "cb_server_destroy", "cb_batch_admit",
                 "cb_batch_release", "cb_batch_pass", "cb_server_stats", "cb_scene_reserve", "cb_get_rest_filter"]


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    """cb_allocator of the C ABI."""
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("ctx", C.c_void_p)]


_TORCH_ALLOCATORS: dict = {}


def torch_allocator(device=None) -> Allocator:
    """PyTorch's CUDA caching allocator as the library's allocator for one
    device: every device buffer of a scene created with it is a block of
    torch's pool, so torch.cuda.memory_allocated / memory_reserved account for
    it and a budget charged from them sees the library's memory.  The
    callbacks live for the whole process (scenes keep pointers to them)."""
    import torch
    if device is None:
        dev = torch.cuda.current_device()
    elif isinstance(device, int):
        dev = device
    else:
        dev = torch.device(device).index
        if dev is None:
            dev = torch.cuda.current_device()
    got = _TORCH_ALLOCATORS.get(dev)
    if got is not None:
        return got[0]

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(stream or 0))
        except Exception:  # out of memory: the library reports CB_ERR_OOM
            return None

    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    fa, ff = _ALLOC_FN(_alloc), _FREE_FN(_free)
    a = Allocator(fa, ff, None)
    _TORCH_ALLOCATORS[dev] = (a, fa, ff)
    return a


def _allocator_arg(allocator):
    """allocator argument of the create calls: "torch" (default), None (the
    library's own stream-ordered pool) or an Allocator."""
    if allocator is None:
        return None
    if isinstance(allocator, str):
        if allocator != "torch":
            raise ValueError(f"unknown allocator {allocator!r}")
        return C.byref(torch_allocator())
    return C.byref(allocator)


class ContactError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_str(status)} ({status})")


class SceneDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_verts", C.c_int32), ("rest_xyz", C.c_void_p),
                ("n_rods", C.c_int32), ("rod_ptr", C.c_void_p), ("n_tris", C.c_int32),
                ("tris", C.c_void_p), ("thickness", C.c_double), ("dhat", C.c_double),
                ("kappa", C.c_double), ("mode", C.c_int32), ("cull_radius", C.c_int32),
                ("rod_closed", C.c_void_p), ("rest_uv", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [("n_candidates", C.c_int64), ("n_filtered", C.c_int64), ("n_core", C.c_int64),
                ("n_active", C.c_int64), ("n_ccd", C.c_int64), ("nnzb", C.c_int64),
                ("n_rest_filtered", C.c_int64), ("dbar_min", C.c_double), ("offset", C.c_double),
                ("dhat", C.c_double), ("activation", C.c_double), ("status_bits", C.c_int32),
                ("ccd_max_iters", C.c_int32), ("device_bytes", C.c_int64),
                ("n_candidates_fp32", C.c_int64), ("n_fp64_decided", C.c_int64),
                ("n_hess_face", C.c_int64), ("n_hess_pe_frame", C.c_int64), ("n_hess_pe", C.c_int64),
                ("n_pair_overflow", C.c_int64), ("n_mollified", C.c_int64), ("n_stencil_dropped", C.c_int64)]


def build(force: bool = False) -> str:
    from . import build as _b
    return _b.build(force=force)


def lib():
    """Load libcontact.so (raises OSError if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError(f"contact library not built: {LIB_PATH} (run paper_2510_10256_gb300.build)")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        for name in ABI_FUNCTIONS:
            getattr(L, name).restype = i32
        L.cb_status_str.restype = C.c_char_p
        L.cb_status_str.argtypes = [i32]
        L.cb_version.restype = C.c_char_p
        L.cb_kernel_launches.restype = i64
        L.cb_kernel_launches.argtypes = []
        L.cb_measure_fma_tflops.argtypes = [i32, i32, i32, C.POINTER(C.c_double)]
        L.cb_batch_create.argtypes = [C.POINTER(vp), i32, C.POINTER(Allocator), vp, C.POINTER(vp)]
        L.cb_batch_offsets.argtypes = [vp, vp, vp, vp]
        L.cb_member_count.argtypes = [vp]
        L.cb_scene_create.argtypes = [C.POINTER(SceneDesc), C.POINTER(Allocator), vp, C.POINTER(vp)]
        L.cb_scene_destroy.argtypes = [vp]
        L.contact_build.argtypes = [vp, vp, vp]
        L.contact_filter.argtypes = [vp, vp]
        L.barrier_eval.argtypes = [vp, vp, vp, vp, vp]
        L.barrier_energy.argtypes = [vp, vp, vp, vp]
        L.cb_bsr_spmv.argtypes = [vp, vp, vp, C.c_double, vp]
        L.friction_lag.argtypes = [vp, vp, C.c_double, C.c_double, vp]
        L.friction_eval.argtypes = [vp, vp, vp, vp, vp, vp]
        L.friction_spmv.argtypes = [vp, vp, vp, vp]
        L.cb_get_friction.argtypes = [vp, vp, vp, vp, i64, C.POINTER(i64)]
        L.ccd_step.argtypes = [vp, vp, vp, vp, vp]
        L.cb_get_pairs.argtypes = [vp, i32, vp, i64, C.POINTER(i64)]
        L.cb_get_rest_filter.argtypes = [vp, vp, vp, i64, C.POINTER(i64)]
        L.cb_get_active.argtypes = [vp, vp, vp, vp, vp, i64, C.POINTER(i64)]
        L.cb_get_ccd.argtypes = [vp, vp, vp, vp, i64, C.POINTER(i64)]
        L.cb_get_bsr.argtypes = [vp, vp, vp, vp, i64, C.POINTER(i64)]
        L.cb_bsr_device.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(i64)]
        L.cb_get_stats.argtypes = [vp, C.POINTER(Stats)]
        L.cb_sync_status.argtypes = [vp]
        L.cb_get_stage_ms.argtypes = [vp, C.POINTER(C.c_float)]
        L.cb_get_stage_times.argtypes = [vp, C.POINTER(C.c_float), C.c_int32]
        L.cb_set_timing.argtypes = [vp, i32]
        L.ccd_step_noalloc.argtypes = [vp, vp, i32, vp, vp, vp, i64, vp, vp, vp]
        L.cb_set_tuning.argtypes = [vp, i32, C.c_float, i32]
        L.cb_get_tuning.argtypes = [vp, i32, C.POINTER(C.c_float), C.POINTER(i32)]
        L.cb_server_create.argtypes = [i32, i32, i64, C.POINTER(Allocator), C.POINTER(vp)]
        L.cb_server_destroy.argtypes = [vp]
        L.cb_batch_admit.argtypes = [vp, vp, C.POINTER(i32)]
        L.cb_batch_release.argtypes = [vp, i32]
        L.cb_batch_pass.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), vp]
        L.cb_server_stats.argtypes = [vp, C.POINTER(i32), C.POINTER(i64), C.POINTER(i64)]
        L.cb_scene_reserve.argtypes = [vp, i64, i64, i64, vp]
        _lib = L
    return _lib


def kernel_launches() -> int:
    return int(lib().cb_kernel_launches())


def measure_fma_tflops(fp64: bool = True, blocks: int = 152 * 8, iters: int = 4096) -> float:
    """Measured FMA throughput of the current GPU (TFLOP/s)."""
    t = C.c_double()
    _check(lib().cb_measure_fma_tflops(int(fp64), blocks, iters, C.byref(t)), "cb_measure_fma_tflops")
    return t.value


NOALLOC_MAX_STENCILS = 1 << 20
NOALLOC_BAD_STENCIL = 8


def ccd_step_noalloc(x, p, stencils, is_ee, offset, alpha, flags, stream=None):
    """Step bound of an explicit stencil list without any device allocation
    (ccd_step_noalloc of the C ABI).  All arguments are CUDA tensors the caller
    owns: x, p FP64 [3][n]; stencils int32 [m][4]; is_ee uint8 [m]; offset
    FP64 [m]; alpha FP64 [1] and flags int32 [1] receive the results.  Nothing
    is copied or converted here, so non-contiguous or mistyped tensors are
    rejected rather than fixed.  Every tensor must live on one GPU; the call
    runs with that GPU current (and on its current stream unless `stream` is
    given)."""
    import torch

    def need(t, dtype, numel=None):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
            raise TypeError(f"expected a contiguous CUDA {dtype} tensor")
        if t.device != x.device:
            raise ValueError(f"every tensor must be on {x.device}, got one on {t.device}")
        if numel is not None and t.numel() != numel:
            raise ValueError(f"expected {numel} elements, got {t.numel()}")
        return t.data_ptr()

    n = x.numel() // 3
    m = stencils.numel() // 4
    with torch.cuda.device(x.device):
        args = (need(x, torch.float64, 3 * n), need(p, torch.float64, 3 * n), n,
                need(stencils, torch.int32, 4 * m), need(is_ee, torch.uint8, m), need(offset, torch.float64, m),
                m, need(alpha, torch.float64, 1), need(flags, torch.int32, 1), _stream_ptr(stream))
        _check(lib().ccd_step_noalloc(*args), "ccd_step_noalloc")


def status_str(s: int) -> str:
    try:
        return lib().cb_status_str(int(s)).decode()
    except OSError:
        return f"status {s}"


def _check(status: int, where: str):
    if status != CB_OK:
        raise ContactError(status, where)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _dev_ptr(t, n: int | None = None, shape3: bool = True):
    import torch
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous CUDA float64 tensor")
    if shape3 and n is not None and t.numel() != 3 * n:
        raise ValueError(f"expected 3*n = {3 * n} elements, got {t.numel()}")
    return t.data_ptr()


class ContactScene:
    """A scene of the contact library: topology, rest mesh, filter tables and
    the pass buffers, resident on the current CUDA device."""

    def __init__(self, kind: str, rest, thickness: float, dhat: float, rod_ptr=None, tris=None,
                 kappa: float = 1.0, mode: str = "double", paper_literal: bool = False,
                 core_temp: bool = True, cull_radius: int = 0, per_component: bool = False, rod_closed=None,
                 mollifier: bool = False, rest_uv=None, per_stencil: bool = False, rest_geodesic: bool = False,
                 stream=None, allocator="torch"):
        L = lib()
        rest = np.ascontiguousarray(np.asarray(rest, np.float64).reshape(3, -1))
        self.n = rest.shape[1]
        self._keep = [rest]
        d = SceneDesc()
        d.kind = CB_ROD if kind == "rod" else CB_SHELL
        d.n_verts = self.n
        d.rest_xyz = rest.ctypes.data
        if kind == "rod":
            rp = np.ascontiguousarray(np.asarray(rod_ptr, np.int32))
            self._keep.append(rp)
            d.n_rods = rp.size - 1
            d.rod_ptr = rp.ctypes.data
            if rod_closed is not None:
                rc = np.ascontiguousarray(np.asarray(rod_closed, np.uint8).reshape(-1))
                if rc.size != d.n_rods:
                    raise ValueError("rod_closed: one flag per polyline")
                self._keep.append(rc)
                d.rod_closed = rc.ctypes.data
        else:
            tr = np.ascontiguousarray(np.asarray(tris, np.int32).reshape(3, -1))
            self._keep.append(tr)
            d.n_tris = tr.shape[1]
            d.tris = tr.ctypes.data
            if rest_uv is not None:
                uv = np.ascontiguousarray(np.asarray(rest_uv, np.float64).reshape(2, -1))
                if uv.shape[1] != self.n:
                    raise ValueError("rest_uv: (2, n)")
                self._keep.append(uv)
                d.rest_uv = uv.ctypes.data
        d.thickness = float(thickness)
        d.dhat = float(dhat)
        d.kappa = float(kappa)
        d.mode = MODES[mode] | (CB_THICK_PAPER_LITERAL if paper_literal else 0) | \
            (0 if core_temp else CB_NO_CORE_TEMP) | (CB_DBAR_PER_COMPONENT if per_component else 0) | \
            (CB_EE_MOLLIFIER if mollifier else 0) | (CB_PER_STENCIL if per_stencil else 0) | \
            (CB_DBAR_GEODESIC if rest_geodesic else 0)
        d.cull_radius = int(cull_radius)
        h = C.c_void_p()
        _check(L.cb_scene_create(C.byref(d), _allocator_arg(allocator), _stream_ptr(stream), C.byref(h)),
               "cb_scene_create")
        self.h = h
        self.kind = kind
        self._load_layout()

    def _load_layout(self):
        self.count = int(lib().cb_member_count(self.h))
        vo = np.zeros(self.count + 1, np.int64)
        eo = np.zeros(self.count + 1, np.int64)
        to = np.zeros(self.count + 1, np.int64)
        _check(lib().cb_batch_offsets(self.h, vo.ctypes.data, eo.ctypes.data, to.ctypes.data), "cb_batch_offsets")
        self.vert_offsets, self.edge_offsets, self.tri_offsets = vo, eo, to
        self.n = int(vo[-1])

    @classmethod
    def from_scene(cls, sc, mode: str = "double", **kw) -> "ContactScene":
        return cls(sc.kind, sc.rest, sc.thickness, sc.dhat, rod_ptr=sc.rod_ptr, tris=sc.tris,
                   kappa=sc.kappa, mode=mode, rod_closed=getattr(sc, "rod_closed", None),
                   rest_uv=getattr(sc, "rest_uv", None),
                   rest_geodesic=bool(getattr(sc, "rest_geodesic", False)), **kw)

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            lib().cb_scene_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ----------------------------------------------------------- pass calls
    def contact_build(self, x, stream=None):
        _check(lib().contact_build(self.h, _dev_ptr(x, self.n), _stream_ptr(stream)), "contact_build")

    def contact_filter(self, stream=None):
        _check(lib().contact_filter(self.h, _stream_ptr(stream)), "contact_filter")

    def barrier_eval(self, x, energy=None, grad=None, stream=None):
        _check(lib().barrier_eval(self.h, _dev_ptr(x, self.n), _dev_ptr(energy, None, False),
                                  _dev_ptr(grad, self.n), _stream_ptr(stream)), "barrier_eval")

    def barrier_energy(self, x, energy, stream=None):
        """Energy only (no gradient, Hessian or BSR) at x, over the candidates
        of the last contact_build / contact_filter: the line-search call."""
        _check(lib().barrier_energy(self.h, _dev_ptr(x, self.n), _dev_ptr(energy, None, False),
                                    _stream_ptr(stream)), "barrier_energy")

    def bsr_spmv(self, v, y, shift: float = 0.0, stream=None):
        """y = (H + shift I) v with the BSR Hessian of the last barrier_eval."""
        _check(lib().cb_bsr_spmv(self.h, _dev_ptr(v, self.n), _dev_ptr(y, self.n), float(shift),
                                 _stream_ptr(stream)), "cb_bsr_spmv")

    def friction_lag(self, x_lag, mu: float, eps: float, stream=None):
        """Lagged friction data of the active pairs of the last barrier_eval
        (which must have run at x_lag)."""
        _check(lib().friction_lag(self.h, _dev_ptr(x_lag, self.n), float(mu), float(eps), _stream_ptr(stream)),
               "friction_lag")

    def friction_eval(self, x, x_lag, energy, grad=None, stream=None):
        """Adds the friction energy to energy[0] and, with grad, its gradient
        to grad (and keeps the pair Hessians for friction_spmv)."""
        _check(lib().friction_eval(self.h, _dev_ptr(x, self.n), _dev_ptr(x_lag, self.n),
                                   _dev_ptr(energy, None, False),
                                   None if grad is None else _dev_ptr(grad, self.n), _stream_ptr(stream)),
               "friction_eval")

    def friction_spmv(self, v, y, stream=None):
        """y += H_f v (friction Hessian of the last friction_eval with a gradient)."""
        _check(lib().friction_spmv(self.h, _dev_ptr(v, self.n), _dev_ptr(y, self.n), _stream_ptr(stream)),
               "friction_spmv")

    def friction(self, hessian: bool = True) -> dict:
        """The lagged pairs: keys, lam, beta (nf, 4), nrm (nf, 3) and, if asked,
        the packed pair Hessians hw (nf, 6)."""
        cnt = C.c_int64()
        _check(lib().cb_get_friction(self.h, None, None, None, 0, C.byref(cnt)), "cb_get_friction")
        nf = cnt.value
        keys = np.zeros(nf, np.uint64)
        dat = np.zeros((8, nf))
        hw = np.zeros((6, nf)) if hessian else None
        if nf:
            _check(lib().cb_get_friction(self.h, keys.ctypes.data, dat.ctypes.data,
                                         hw.ctypes.data if hessian else None, nf, C.byref(cnt)),
                   "cb_get_friction")
        out = dict(keys=keys, lam=dat[0].copy(), beta=dat[1:5].T.copy(), nrm=dat[5:8].T.copy())
        if hessian:
            out["hw"] = hw.T.copy()
        return out

    def ccd_step(self, x, p, alpha=None, stream=None):
        _check(lib().ccd_step(self.h, _dev_ptr(x, self.n), _dev_ptr(p, self.n),
                              _dev_ptr(alpha, None, False), _stream_ptr(stream)), "ccd_step")

    def reserve(self, n_candidates: int, n_ccd: int, n_active: int, stream=None):
        """Pre-size the pair-list buffers for passes with at most these counts
        (cb_scene_reserve)."""
        _check(lib().cb_scene_reserve(self.h, int(n_candidates), int(n_ccd), int(n_active), _stream_ptr(stream)),
               "cb_scene_reserve")

    def run_pass(self, x, p, energy, grad, alpha, stream=None):
        """Stages a-e in order on one stream."""
        self.contact_build(x, stream)
        self.contact_filter(stream)
        self.barrier_eval(x, energy, grad, stream)
        self.ccd_step(x, p, alpha, stream)

    # -------------------------------------------------------------- getters
    def member_of_keys(self, keys: np.ndarray) -> np.ndarray:
        """member index of each (batch-numbered) pair key"""
        keys = np.asarray(keys, np.uint64)
        ty = (keys >> np.uint64(62)).astype(np.int64)
        i = ((keys >> np.uint64(31)) & np.uint64(0x7FFFFFFF)).astype(np.int64)
        off = np.where(ty == 1, 0, 1)
        m_v = np.searchsorted(self.vert_offsets, i, side="right") - 1
        m_e = np.searchsorted(self.edge_offsets, i, side="right") - 1
        return np.where(off == 0, m_v, m_e)

    def to_member_keys(self, keys: np.ndarray, m: int) -> np.ndarray:
        """batch-numbered keys of member m -> the member's own numbering"""
        keys = np.asarray(keys, np.uint64)
        ty = keys >> np.uint64(62)
        i = (keys >> np.uint64(31)) & np.uint64(0x7FFFFFFF)
        j = keys & np.uint64(0x7FFFFFFF)
        pt = ty == np.uint64(1)
        di = np.where(pt, self.vert_offsets[m], self.edge_offsets[m]).astype(np.uint64)
        dj = np.where(pt, self.tri_offsets[m], self.edge_offsets[m]).astype(np.uint64)
        return (ty << np.uint64(62)) | ((i - di) << np.uint64(31)) | (j - dj)

    def pairs(self, which: str = "candidate") -> np.ndarray:
        cnt = C.c_int64()
        lib().cb_get_pairs(self.h, PAIRS[which], None, 0, C.byref(cnt))
        out = np.zeros(cnt.value, np.uint64)
        _check(lib().cb_get_pairs(self.h, PAIRS[which], out.ctypes.data if out.size else None, out.size,
                                  C.byref(cnt)), "cb_get_pairs")
        return out

    def rest_filter(self) -> tuple[np.ndarray, np.ndarray]:
        """Shells: the rest-filtered stencil pairs (key order) and their reference distances."""
        cnt = C.c_int64()
        lib().cb_get_rest_filter(self.h, None, None, 0, C.byref(cnt))
        keys, dbar = np.zeros(cnt.value, np.uint64), np.zeros(cnt.value)
        _check(lib().cb_get_rest_filter(self.h, keys.ctypes.data if keys.size else None,
                                        dbar.ctypes.data if dbar.size else None, keys.size, C.byref(cnt)),
               "cb_get_rest_filter")
        return keys, dbar

    def active(self) -> dict:
        cnt = C.c_int64()
        lib().cb_get_active(self.h, None, None, None, None, 0, C.byref(cnt))
        m = cnt.value
        k = np.zeros(m, np.uint64)
        d = np.zeros(m)
        c = np.zeros(m, np.uint8)
        t = np.zeros(m, np.int8)
        if m:
            _check(lib().cb_get_active(self.h, k.ctypes.data, d.ctypes.data, c.ctypes.data, t.ctypes.data, m,
                                       C.byref(cnt)), "cb_get_active")
        return dict(keys=k, d=d, klass=c, dtype=t)

    def ccd(self) -> dict:
        cnt = C.c_int64()
        lib().cb_get_ccd(self.h, None, None, None, 0, C.byref(cnt))
        m = cnt.value
        k = np.zeros(m, np.uint64)
        t = np.zeros(m)
        c = np.zeros(m, np.uint8)
        if m:
            _check(lib().cb_get_ccd(self.h, k.ctypes.data, t.ctypes.data, c.ctypes.data, m, C.byref(cnt)),
                   "cb_get_ccd")
        return dict(keys=k, t=t, klass=c)

    def bsr(self):
        cnt = C.c_int64()
        lib().cb_get_bsr(self.h, None, None, None, 0, C.byref(cnt))
        m = cnt.value
        rp = np.zeros(self.n + 1, np.int32)
        col = np.zeros(m, np.int32)
        val = np.zeros((m, 3, 3))
        _check(lib().cb_get_bsr(self.h, rp.ctypes.data, col.ctypes.data if m else None,
                                val.ctypes.data if m else None, m, C.byref(cnt)), "cb_get_bsr")
        return rp, col, val

    def stats(self) -> dict:
        s = Stats()
        _check(lib().cb_get_stats(self.h, C.byref(s)), "cb_get_stats")
        return {f: getattr(s, f) for f, _ in Stats._fields_}

    def sync_status(self) -> int:
        return int(lib().cb_sync_status(self.h))

    def set_tuning(self, phase: int, cell_factor: float, pair_block: int = 256):
        """Broad-phase knobs (phase 0: contact_build, 1: ccd_step); speed only."""
        _check(lib().cb_set_tuning(self.h, int(phase), float(cell_factor), int(pair_block)), "cb_set_tuning")

    def tuning(self, phase: int) -> tuple[float, int]:
        f, b = C.c_float(), C.c_int32()
        _check(lib().cb_get_tuning(self.h, int(phase), C.byref(f), C.byref(b)), "cb_get_tuning")
        return float(f.value), int(b.value)

    def set_timing(self, on: bool = True):
        _check(lib().cb_set_timing(self.h, int(on)), "cb_set_timing")

    def stage_ms(self) -> list[float]:
        """Device ms of the last calls: build, filter, barrier_eval, ccd_step,
        Hessian kernels, and barrier_eval's stage (c) and stage (d) parts."""
        ms = (C.c_float * 7)()
        _check(lib().cb_get_stage_times(self.h, ms, 7), "cb_get_stage_times")
        return [float(v) for v in ms]


class ContactBatch(ContactScene):
    """Several scenes of one kind in one pass (cb_batch_create).  x, p and grad
    span the concatenated vertices (member order); energy and alpha hold one
    value per member."""

    def __init__(self, members: list, stream=None, allocator="torch"):
        L = lib()
        arr = (C.c_void_p * len(members))(*[m.h.value for m in members])
        h = C.c_void_p()
        _check(L.cb_batch_create(arr, len(members), _allocator_arg(allocator), _stream_ptr(stream), C.byref(h)),
               "cb_batch_create")
        self.h = h
        self.kind = members[0].kind
        self._keep = []
        self._load_layout()


class ContactServer:
    """Resident scenes of one kind advanced by one batched pass (the C ABI's
    cb_server: cb_batch_admit / cb_batch_release / cb_batch_pass).  The caller
    keeps its ContactScene objects; release a slot before closing its scene."""

    def __init__(self, kind: str, slots: int, hbm_budget_bytes: int, allocator="torch"):
        h = C.c_void_p()
        _check(lib().cb_server_create(CB_ROD if kind == "rod" else CB_SHELL, int(slots), int(hbm_budget_bytes),
                                      _allocator_arg(allocator), C.byref(h)), "cb_server_create")
        self.h = h
        self.slots = int(slots)
        self.scenes = [None] * self.slots

    def admit(self, scene: "ContactScene") -> int:
        """The slot the scene got; ContactError with CB_ERR_CAPACITY (no free
        slot) or CB_ERR_OOM (over the budget) otherwise."""
        k = C.c_int32()
        _check(lib().cb_batch_admit(self.h, scene.h, C.byref(k)), "cb_batch_admit")
        self.scenes[k.value] = scene
        return int(k.value)

    def release(self, slot: int):
        _check(lib().cb_batch_release(self.h, int(slot)), "cb_batch_release")
        self.scenes[slot] = None

    def run_pass(self, x: dict, p: dict, energy: dict | None = None, grad: dict | None = None,
                 alpha: dict | None = None, stream=None):
        """Stages a-e for every resident scene; each argument maps a slot to
        that scene's CUDA tensor (x, p, grad [3][n]; energy, alpha [1])."""
        def table(d, out):
            arr = (C.c_void_p * self.slots)()
            for k, sc in enumerate(self.scenes):
                if sc is None or d is None or d.get(k) is None:
                    continue
                arr[k] = _dev_ptr(d[k], sc.n if out != "scalar" else None, shape3=out != "scalar")
            return arr
        _check(lib().cb_batch_pass(self.h, table(x, "vec"), table(p, "vec"), table(energy, "scalar"),
                                   table(grad, "vec"), table(alpha, "scalar"), _stream_ptr(stream)), "cb_batch_pass")

    def stats(self) -> dict:
        r, b, c = C.c_int32(), C.c_int64(), C.c_int64()
        _check(lib().cb_server_stats(self.h, C.byref(r), C.byref(b), C.byref(c)), "cb_server_stats")
        return {"resident": int(r.value), "charged_bytes": int(b.value), "n_candidates": int(c.value)}

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            lib().cb_server_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
