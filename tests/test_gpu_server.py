"""Serving through the C ABI (cb_server_create / cb_batch_admit /
cb_batch_release / cb_batch_pass / cb_scene_reserve): resident scenes of one
kind are admitted into slots under a device-memory budget charged from their
real bytes and advanced together by one batched pass; each scene's result is
the one its own pass gives (pair counts and alpha exactly, energy and gradient
within the parity tolerance), across admissions and releases."""
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


def _tensors(sc):
    import torch
    dev = torch.device("cuda:0")
    return dict(x=torch.from_numpy(np.ascontiguousarray(sc.x)).to(dev),
                p=torch.from_numpy(np.ascontiguousarray(sc.p)).to(dev),
                e=torch.zeros(1, dtype=torch.float64, device=dev),
                g=torch.zeros(3, sc.n, dtype=torch.float64, device=dev),
                a=torch.zeros(1, dtype=torch.float64, device=dev))


def _alone(sc):
    import torch
    from paper_2510_10256_gb300.contact import ContactScene
    cs = ContactScene.from_scene(sc)
    t = _tensors(sc)
    cs.run_pass(t["x"], t["p"], t["e"], t["g"], t["a"])
    torch.cuda.synchronize()
    out = (float(t["e"].item()), t["g"].cpu().numpy(), float(t["a"].item()), cs.stats()["n_candidates"])
    cs.close()
    return out


def _check_same(sc, t, alone):
    import torch
    torch.cuda.synchronize()
    e0, g0, a0, _ = alone
    orc = O.contact_pass(sc, ccd=False)
    assert float(t["a"].item()) == a0
    assert abs(float(t["e"].item()) - e0) <= 1e-9 * max(abs(e0), 1e-300)
    assert np.all(np.abs(t["g"].cpu().numpy() - g0) <= 1e-9 * orc.grad_abs + 1e-30)


def test_server_pass_equals_each_scene_alone_across_admissions():
    import torch
    from paper_2510_10256_gb300.contact import ContactScene, ContactServer
    scs = [S.tiny_shell(1), S.pleated_sheet(nx=24), S.tiny_shell(2, nx=6, thickness=0.3, dhat=0.07),
           S.graded_disk(target_tris=3000, L0=0.5)]
    alone = [_alone(sc) for sc in scs]
    srv = ContactServer("shell", slots=3, hbm_budget_bytes=64 << 30)
    css = [ContactScene.from_scene(sc) for sc in scs]
    ts = [_tensors(sc) for sc in scs]
    slots = [srv.admit(cs) for cs in css[:3]]
    assert slots == [0, 1, 2] and srv.stats()["resident"] == 3

    def run(resident):
        srv.run_pass({k: ts[i]["x"] for k, i in resident.items()}, {k: ts[i]["p"] for k, i in resident.items()},
                     {k: ts[i]["e"] for k, i in resident.items()}, {k: ts[i]["g"] for k, i in resident.items()},
                     {k: ts[i]["a"] for k, i in resident.items()})
        torch.cuda.synchronize()
        assert srv.stats()["n_candidates"] == sum(alone[i][3] for i in resident.values())
        for k, i in resident.items():
            _check_same(scs[i], ts[i], alone[i])

    run({0: 0, 1: 1, 2: 2})
    run({0: 0, 1: 1, 2: 2})                  # the same batch again
    # the server is full; release slot 1 and admit the fourth scene there
    from paper_2510_10256_gb300.contact import CB_ERR_CAPACITY, ContactError
    with pytest.raises(ContactError) as ei:
        srv.admit(css[3])
    assert ei.value.status == CB_ERR_CAPACITY
    srv.release(1)
    assert srv.admit(css[3]) == 1
    for t in ts:
        t["e"].zero_(); t["g"].zero_(); t["a"].zero_()
    run({0: 0, 1: 3, 2: 2})
    srv.close()
    for cs in css:
        cs.close()


def test_server_budget_and_arguments():
    from paper_2510_10256_gb300.contact import (CB_ERR_ARG, CB_ERR_OOM, ContactError, ContactScene,
                                                ContactServer)
    shell = ContactScene.from_scene(S.pleated_sheet(nx=24))
    rod = ContactScene.from_scene(S.tiny_rods(1))
    held = shell.stats()["device_bytes"]
    small = ContactServer("shell", slots=4, hbm_budget_bytes=held)    # twice its bytes would not fit
    with pytest.raises(ContactError) as ei:
        small.admit(shell)
    assert ei.value.status == CB_ERR_OOM and small.stats()["resident"] == 0
    big = ContactServer("shell", slots=4, hbm_budget_bytes=4 * held)
    big.admit(shell)
    assert big.stats()["charged_bytes"] == held
    for bad in (rod, shell):                  # wrong kind; already resident
        with pytest.raises(ContactError) as ei:
            big.admit(bad)
        assert ei.value.status == CB_ERR_ARG
    big.release(0)
    small.close()
    big.close()
    shell.close()
    rod.close()


def test_reserve_presizes_the_pair_lists():
    """With cb_scene_reserve for (more than) a pass's counts, that pass
    allocates fewer buffers -- none of the pair lists -- and gives the same
    results; counts beyond 2^31 - 1 are refused."""
    import torch
    from paper_2510_10256_gb300 import contact as CT
    calls = {"n": 0}

    def _alloc(nbytes, stream, ctx):
        calls["n"] += 1
        return torch.cuda.caching_allocator_alloc(int(nbytes), 0, int(stream or 0))

    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    fa, ff = CT._ALLOC_FN(_alloc), CT._FREE_FN(_free)
    al = CT.Allocator(fa, ff, None)
    sc = S.pleated_sheet(nx=32)
    out = []
    for reserve in (False, True):
        cs = CT.ContactScene.from_scene(sc, allocator=al)
        if reserve:
            st = out[0][2]
            cs.reserve(2 * st["n_candidates"], 2 * st["n_ccd"], 2 * st["n_active"])
        t = _tensors(sc)
        n0 = calls["n"]
        cs.run_pass(t["x"], t["p"], t["e"], t["g"], t["a"])
        torch.cuda.synchronize()
        out.append((calls["n"] - n0, (float(t["e"].item()), float(t["a"].item())), cs.stats()))
        if reserve:
            with pytest.raises(CT.ContactError) as ei:
                cs.reserve(1 << 31, 0, 0)
            assert ei.value.status == CT.CB_ERR_TOO_LARGE
        cs.close()
    (n_plain, res_plain, st_plain), (n_res, res_res, st_res) = out
    assert n_res < n_plain, (n_res, n_plain)
    assert res_res[1] == res_plain[1] and abs(res_res[0] - res_plain[0]) <= 1e-9 * abs(res_plain[0])
    assert st_res["n_candidates"] == st_plain["n_candidates"]
