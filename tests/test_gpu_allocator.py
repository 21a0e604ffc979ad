"""The caller's allocator (cb_allocator): every device buffer of a scene or a
batch comes from it and goes back to it, and cb_stats.device_bytes is what
the scene holds.  With PyTorch's caching allocator (the binding's default)
torch.cuda.memory_allocated accounts for the library's memory, so a budget
charged from it sees real reservations; the results are unchanged."""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from paper_2510_10256_gb300 import scenes as S
from tests.parity import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_10256_gb300 import contact
    contact.build()
    contact.lib()


def _pass(cs, sc):
    import torch
    dev = torch.device("cuda:0")
    x = torch.from_numpy(np.ascontiguousarray(sc.x)).to(dev)
    p = torch.from_numpy(np.ascontiguousarray(sc.p)).to(dev)
    e = torch.zeros(cs.count, dtype=torch.float64, device=dev)
    g = torch.zeros(3, cs.n, dtype=torch.float64, device=dev)
    a = torch.zeros(cs.count, dtype=torch.float64, device=dev)
    cs.run_pass(x, p, e, g, a)
    torch.cuda.synchronize()
    return x, p, e, g, a


def test_torch_allocator_accounts_for_the_scene():
    import torch
    from paper_2510_10256_gb300.contact import ContactScene
    sc = S.pleated_sheet(nx=48)
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    cs = ContactScene.from_scene(sc)                 # default: torch's caching allocator
    held = cs.stats()["device_bytes"]
    assert held > 0
    d = torch.cuda.memory_allocated() - base
    # torch rounds each block up: to 512 bytes, and blocks of 10 MiB or more to 2 MiB
    assert held <= d <= 1.05 * held + 512 * 200, (held, d)
    keep = _pass(cs, sc)
    held2 = cs.stats()["device_bytes"]
    assert held2 > held                              # the pass buffers
    d2 = torch.cuda.memory_allocated() - base - sum(t.numel() * t.element_size() for t in keep)
    assert held2 <= d2 <= 1.05 * held2 + 512 * 200, (held2, d2)
    assert torch.cuda.memory_reserved() >= base + held2
    # the results are the oracle's
    o = O.contact_pass(sc)
    g = dict(C=cs.pairs("candidate"), F=cs.pairs("filtered"), CC=cs.pairs("core"), A=cs.active(), ccd=cs.ccd(),
             bsr=cs.bsr(), energy=float(keep[2].item()), grad=keep[3].cpu().numpy(), alpha=float(keep[4].item()),
             stats=cs.stats(), status=cs.sync_status(), frest=cs.pairs("rest_filtered"))
    compare(sc, g, o)
    cs.close()
    del keep
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base


def test_library_pool_is_not_torch_memory():
    import torch
    from paper_2510_10256_gb300.contact import ContactScene
    sc = S.tiny_shell(3, nx=6)
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    cs = ContactScene.from_scene(sc, allocator=None)
    assert cs.stats()["device_bytes"] > 0
    assert torch.cuda.memory_allocated() == base
    cs.close()


def test_counting_allocator_gets_every_buffer_back_and_batches_use_theirs():
    import torch
    from paper_2510_10256_gb300 import contact as CT
    live, calls = {}, {"alloc": 0, "free": 0}

    def _alloc(nbytes, stream, ctx):
        ptr = torch.cuda.caching_allocator_alloc(int(nbytes), 0, int(stream or 0))
        live[ptr] = int(nbytes)
        calls["alloc"] += 1
        return ptr

    def _free(ptr, nbytes, stream, ctx):
        assert live.pop(int(ptr)) == int(nbytes)
        calls["free"] += 1
        torch.cuda.caching_allocator_delete(int(ptr))

    fa, ff = CT._ALLOC_FN(_alloc), CT._FREE_FN(_free)
    al = CT.Allocator(fa, ff, None)
    scenes = [S.tiny_shell(1), S.tiny_shell(2, nx=6)]
    members = [CT.ContactScene.from_scene(sc, allocator=al) for sc in scenes]
    member_bytes = sum(m.stats()["device_bytes"] for m in members)
    assert sum(live.values()) == member_bytes
    b = CT.ContactBatch(members, allocator=al)
    for m in members:
        m.close()
    x = np.concatenate([sc.x for sc in scenes], axis=1)
    p = np.concatenate([sc.p for sc in scenes], axis=1)
    sc_all = S.Scene("shell", x, x, p, 0.4, 0.1)
    _pass(b, sc_all)
    assert sum(live.values()) == b.stats()["device_bytes"] > 0
    b.close()
    assert not live and calls["alloc"] == calls["free"] > 0


def test_failing_allocator_reports_oom_and_leaks_nothing():
    import torch
    from paper_2510_10256_gb300 import contact as CT
    live = {}
    budget = {"left": 40}

    def _alloc(nbytes, stream, ctx):
        if budget["left"] <= 0:
            return None                                   # out of memory
        budget["left"] -= 1
        ptr = torch.cuda.caching_allocator_alloc(int(nbytes), 0, int(stream or 0))
        live[ptr] = int(nbytes)
        return ptr

    def _free(ptr, nbytes, stream, ctx):
        live.pop(int(ptr))
        torch.cuda.caching_allocator_delete(int(ptr))

    fa, ff = CT._ALLOC_FN(_alloc), CT._FREE_FN(_free)
    al = CT.Allocator(fa, ff, None)
    with pytest.raises(CT.ContactError) as ei:
        CT.ContactScene.from_scene(S.pleated_sheet(nx=24), allocator=al)
    assert ei.value.status == CT.CB_ERR_OOM
    assert not live
    # with room to spare the same scene works and gives everything back
    budget["left"] = 10 ** 6
    cs = CT.ContactScene.from_scene(S.pleated_sheet(nx=24), allocator=al)
    assert sum(live.values()) == cs.stats()["device_bytes"]
    cs.close()
    assert not live
