"""ccd_step_noalloc (fixed device scratch, no allocation) against ccd_step
and the oracle.

Some callers cannot allocate device memory while they run (a solver that
hands its whole device budget to its own pool, a loop in which an allocation
could stall the device); ccd_step_noalloc serves them from one fixed scratch
array.  The stencil list is the scene's own CCD candidate set, rebuilt on the
host from the pair keys and the edge numbering the C ABI documents; each
stencil keeps the offset of its class.  The step bound must agree with
ccd_step's within the parity tolerance of alpha, and never exceed the
oracle's (alpha <= alpha_oracle, alpha_oracle - alpha <= 1e-9), on
consecutive calls (the scratch is reused, so every call must start from
cleared accumulators).
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_2510_10256_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_10256_gb300 import contact
    contact.build()
    contact.lib()


def _edges(sc):
    if sc.kind == "rod":
        rp = np.asarray(sc.rod_ptr)
        e = [(v, v + 1) for r in range(rp.size - 1) for v in range(rp[r], rp[r + 1] - 1)]
        return np.array(e, np.int64).reshape(-1, 2)
    t = np.asarray(sc.tris)
    e = np.concatenate([np.sort(np.stack([t[a], t[b]], 1), 1) for a, b in ((0, 1), (1, 2), (0, 2))])
    return np.unique(e, axis=0)


def _stencils(sc, keys, klass, offset, single):
    keys = keys.astype(np.uint64)
    ty = (keys >> np.uint64(62)).astype(np.int64)
    i = ((keys >> np.uint64(31)) & np.uint64(0x7FFFFFFF)).astype(np.int64)
    j = (keys & np.uint64(0x7FFFFFFF)).astype(np.int64)
    E = _edges(sc)
    st = np.zeros((keys.size, 4), np.int32)
    pt = ty == 1
    if pt.any():
        T = np.asarray(sc.tris)
        st[pt, 0] = i[pt]
        st[pt, 1:] = T[:, j[pt]].T
    ee = ~pt
    st[ee, :2] = E[i[ee]]
    st[ee, 2:] = E[j[ee]]
    cls = klass & 0x7F
    off = np.where((cls == 0) & (not single), offset, 0.0)
    return st, ee.astype(np.uint8), off


def _reference(sc, mode="double"):
    """ccd_step on the scene; returns alpha and the noalloc inputs."""
    import torch
    from paper_2510_10256_gb300.contact import ContactScene
    dev = torch.device("cuda:0")
    cs = ContactScene.from_scene(sc, mode=mode)
    x = torch.from_numpy(np.ascontiguousarray(sc.x)).to(dev)
    p = torch.from_numpy(np.ascontiguousarray(sc.p)).to(dev)
    energy = torch.zeros(1, dtype=torch.float64, device=dev)
    grad = torch.zeros(3, sc.n, dtype=torch.float64, device=dev)
    alpha = torch.zeros(1, dtype=torch.float64, device=dev)
    cs.run_pass(x, p, energy, grad, alpha)
    torch.cuda.synchronize()
    c = cs.ccd()
    st, ee, off = _stencils(sc, c["keys"], c["klass"], cs.stats()["offset"], mode == "single")
    cs.close()
    return float(alpha.item()), dict(x=x, p=p, st=torch.from_numpy(st).to(dev), ee=torch.from_numpy(ee).to(dev),
                                     off=torch.from_numpy(off).to(dev))


def _noalloc(inp):
    import torch
    from paper_2510_10256_gb300 import contact
    alpha = torch.full((1,), -7.0, dtype=torch.float64, device="cuda:0")
    flags = torch.full((1,), -1, dtype=torch.int32, device="cuda:0")
    contact.ccd_step_noalloc(inp["x"], inp["p"], inp["st"], inp["ee"], inp["off"], alpha, flags)
    torch.cuda.synchronize()
    return float(alpha.item()), int(flags.item())


def test_noalloc_matches_ccd_step_on_consecutive_calls():
    from paper_2510_10256_gb300 import contact
    cases = [S.pleated_sheet(nx=24), S.woven_patch(n_warp=2, n_weft=2, nseg=48), S.tiny_shell(3),
             S.tiny_rods(2)]
    refs = [_reference(sc) for sc in cases]
    orcs = [O.contact_pass(sc).alpha for sc in cases]
    assert len({a for a, _ in refs}) > 1, "cases should have different step bounds"
    assert any(a < 1.0 for a, _ in refs)
    for (alpha_ref, inp), alpha_orc in zip(refs, orcs):
        assert inp["st"].shape[0] > 0
        for _ in range(2):
            n0 = contact.kernel_launches()
            a, f = _noalloc(inp)
            assert contact.kernel_launches() - n0 == 5
            assert f == 0
            assert a <= 1.0 and abs(a - alpha_ref) <= 1e-9, (a, alpha_ref)
            assert a <= alpha_orc and alpha_orc - a <= 1e-9, (a, alpha_orc)


def test_noalloc_empty_bad_full_and_oversized_inputs():
    import torch
    from paper_2510_10256_gb300 import contact
    alpha_ref, inp = _reference(S.pleated_sheet(nx=24))
    m = inp["st"].shape[0]
    assert m > 0
    empty = dict(inp, st=inp["st"][:0], ee=inp["ee"][:0], off=inp["off"][:0])
    assert _noalloc(empty) == (1.0, 0)
    # a vertex id out of range is skipped and reported, never read
    bad = dict(inp, st=inp["st"][:1].clone(), ee=inp["ee"][:1], off=inp["off"][:1])
    bad["st"][0, 2] = inp["x"].shape[1]
    a, f = _noalloc(bad)
    assert a == 1.0 and f & contact.NOALLOC_BAD_STENCIL
    # a non-finite displacement of a stencil vertex: reported, not passed as alpha = 1 silently
    v = int(inp["st"][0, 1].item())
    pn = inp["p"].clone()
    pn[0, v] = float("nan")
    a, f = _noalloc(dict(inp, p=pn, st=inp["st"][:1], ee=inp["ee"][:1], off=inp["off"][:1]))
    assert f & contact.NOALLOC_BAD_STENCIL
    # ... the remaining stencils still bound the step, and the flag says one was skipped
    a, f = _noalloc(dict(inp, p=pn))
    assert f & contact.NOALLOC_BAD_STENCIL and a <= 1.0
    # an output in (device-reachable) pinned host memory is rejected before any launch
    host_alpha = torch.zeros(1, dtype=torch.float64).pin_memory()
    host_flags = torch.zeros(1, dtype=torch.int32).pin_memory()
    n0 = contact.kernel_launches()
    st = contact.lib().ccd_step_noalloc(inp["x"].data_ptr(), inp["p"].data_ptr(), inp["x"].shape[1],
                                        inp["st"].data_ptr(), inp["ee"].data_ptr(), inp["off"].data_ptr(),
                                        m, host_alpha.data_ptr(), host_flags.data_ptr(),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == contact.CB_ERR_ARG and contact.kernel_launches() == n0
    # exactly the maximum: the candidate list repeated
    M = contact.NOALLOC_MAX_STENCILS
    rep = (M + m - 1) // m
    full = dict(inp, st=inp["st"].repeat(rep, 1)[:M].contiguous(), ee=inp["ee"].repeat(rep)[:M].contiguous(),
                off=inp["off"].repeat(rep)[:M].contiguous())
    a, f = _noalloc(full)
    assert f == 0 and abs(a - alpha_ref) <= 1e-9, (a, alpha_ref)
    # one more than the maximum: rejected on the host before any work
    alpha = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    flags = torch.zeros(1, dtype=torch.int32, device="cuda:0")
    st = contact.lib().ccd_step_noalloc(inp["x"].data_ptr(), inp["p"].data_ptr(), inp["x"].shape[1],
                                        full["st"].data_ptr(), full["ee"].data_ptr(), full["off"].data_ptr(),
                                        M + 1, alpha.data_ptr(), flags.data_ptr(),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == contact.CB_ERR_TOO_LARGE
