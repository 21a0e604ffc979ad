"""GPU-vs-oracle comparison used by the -m gpu tests and by smoke().

Acceptance (per pass):
  * candidate set C, filtered set F, class-C set, CCD candidate set, BSR
    pattern: bit-exact sorted keys;
  * active set: bit-exact except pairs whose oracle distance lies within
    1e-12 (relative) of their activation threshold, where the barrier and its
    derivatives vanish;
  * distances of active pairs: 1e-12 relative;
  * energy: 1e-9 relative;
  * gradient and BSR entries: |gpu - oracle| <= 1e-9 * sum |contributions|
    (+ 1e-30 absolute), allowing for summation order; the BSR comparison
    always runs -- where a tie-band pair is active on one side only, the
    blocks of its stencil are set apart and every other block is compared
    (``bsr_compared`` / ``bsr_blocks_skipped`` in the report);
  * alpha: alpha_gpu <= alpha_oracle and alpha_oracle - alpha_gpu <= 1e-9.
"""
from __future__ import annotations

import numpy as np

import oracle as O


def run_gpu(sc, mode="double", core_temp=True, x=None, p=None, paper_literal=False, cull_radius=0,
            per_component=False, mollifier=False, per_stencil=False):
    import torch
    from paper_2510_10256_gb300.contact import ContactScene
    dev = torch.device("cuda:0")
    cs = ContactScene.from_scene(sc, mode=mode, core_temp=core_temp, paper_literal=paper_literal,
                                 cull_radius=cull_radius, per_component=per_component, mollifier=mollifier,
                                 per_stencil=per_stencil)
    xx = torch.from_numpy(np.ascontiguousarray(sc.x if x is None else x)).to(dev)
    pp = torch.from_numpy(np.ascontiguousarray(sc.p if p is None else p)).to(dev)
    energy = torch.zeros(1, dtype=torch.float64, device=dev)
    grad = torch.zeros(3, sc.n, dtype=torch.float64, device=dev)
    alpha = torch.zeros(1, dtype=torch.float64, device=dev)
    cs.run_pass(xx, pp, energy, grad, alpha)
    torch.cuda.synchronize()
    out = dict(C=cs.pairs("candidate"), F=cs.pairs("filtered"), CC=cs.pairs("core"),
               A=cs.active(), ccd=cs.ccd(), bsr=cs.bsr(), energy=float(energy.item()),
               grad=grad.cpu().numpy(), alpha=float(alpha.item()), stats=cs.stats(),
               status=cs.sync_status(), frest=cs.pairs("rest_filtered"))
    cs.close()
    return out


def threshold_band(sc, orc: O.PassResult, mode="double", paper_literal=False):
    """Candidates whose distance is within 1e-12 of an activity or class
    threshold (their activity / class may legitimately differ by rounding)."""
    xi, dhat = O.offsets(sc, paper_literal)
    a = xi + dhat
    d = orc.d
    thr = []
    if mode != "single":
        thr.append(np.full_like(d, xi))
    fw = orc.fwidth if orc.fwidth is not None else orc.dbar_min
    thr.append(np.where(orc.klass == O.KLASS_F, fw, np.where(
        (orc.klass == O.KLASS_C) | (mode == "single"), a, xi + dhat)))
    band = np.zeros(d.size, bool)
    for t in thr:
        band |= np.abs(d - t) <= 1e-12 * np.maximum(1.0, np.abs(t))
    return band


def compare(sc, g: dict, orc: O.PassResult, mode="double", check_ccd=True, paper_literal=False) -> dict:
    """Raise AssertionError on any violation; return a summary."""
    rep = {}
    assert np.array_equal(g["C"], orc.C), f"candidate sets differ: {g['C'].size} vs {orc.C.size}"
    rep["C"] = int(orc.C.size)
    assert np.array_equal(g["F"], orc.keys_of(O.KLASS_F)), "filtered sets differ"
    rep["F"] = int(g["F"].size)
    if sc.kind == "shell":
        assert np.array_equal(g["frest"], orc.F_rest), "rest-filtered sets differ"
    dm_g, dm_o = g["stats"]["dbar_min"], orc.dbar_min
    assert (np.isinf(dm_g) and np.isinf(dm_o)) or abs(dm_g - dm_o) <= 1e-12 * abs(dm_o), (dm_g, dm_o)
    band = threshold_band(sc, orc, mode, paper_literal)
    band_keys = set(orc.C[band].tolist())
    cc_o = set(orc.keys_of(O.KLASS_C).tolist())
    cc_g = set(g["CC"].tolist())
    assert (cc_o ^ cc_g) <= band_keys, "class-C sets differ outside the threshold band"
    rep["core"] = len(cc_g)
    act_o = set(orc.active_keys.tolist())
    act_g = set(g["A"]["keys"].tolist())
    assert (act_o ^ act_g) <= band_keys, f"active sets differ: {len(act_o ^ act_g)} outside band"
    assert np.all(np.diff(g["A"]["keys"].astype(np.uint64).view(np.int64)) > 0) or g["A"]["keys"].size < 2
    rep["active"] = len(act_g)
    # distances of active pairs
    idx_o = np.searchsorted(orc.C, g["A"]["keys"])
    d_o = orc.d[idx_o]
    rel = np.abs(g["A"]["d"] - d_o) / np.maximum(d_o, 1e-300)
    assert rel.size == 0 or rel.max() <= 1e-12, f"distance rel err {rel.max()}"
    rep["d_relerr"] = float(rel.max()) if rel.size else 0.0
    assert np.array_equal(g["A"]["dtype"], orc.dtype[idx_o]) or (act_o ^ act_g), "distance types differ"
    # energy / gradient / BSR
    if np.isfinite(orc.energy):
        assert abs(g["energy"] - orc.energy) <= 1e-9 * max(abs(orc.energy), 1e-300), (g["energy"], orc.energy)
        gerr = np.abs(g["grad"] - orc.grad)
        assert np.all(gerr <= 1e-9 * orc.grad_abs + 1e-30), f"gradient err {float((gerr / (orc.grad_abs + 1e-300)).max())}"
        rep["grad_relerr"] = float((gerr / (orc.grad_abs + 1e-300)).max()) if gerr.size else 0.0
        rp, col, val = g["bsr"]
        rep.update(_compare_bsr(sc, g, orc, act_o ^ act_g))
        rep["nnzb"] = int(col.size)
    else:
        assert not np.isfinite(g["energy"])
    if check_ccd:
        assert np.array_equal(g["ccd"]["keys"], orc.ccd_keys), "CCD candidate sets differ"
        rep["ccd"] = int(orc.ccd_keys.size)
        assert g["alpha"] <= orc.alpha and orc.alpha - g["alpha"] <= 1e-9, (g["alpha"], orc.alpha)
        kl = g["ccd"]["klass"]
        assert np.array_equal(kl & 0x7F, orc.ccd_klass), "CCD classes differ"
        exact = (kl & 0x80) != 0
        t_g, t_o = g["ccd"]["t"], orc.ccd_t
        assert np.all(np.abs(t_g[exact] - t_o[exact]) <= 1e-12 * np.maximum(t_o[exact], 1e-300)), \
            "exact CCD times differ"
        assert np.all(t_g[~exact] <= t_o[~exact]), "CCD lower bound above the oracle's t"
        assert np.all(t_g[~exact] >= g["alpha"]), "a pruned pair could lower alpha"
        rep["ccd_exact"] = int(exact.sum())
        rep["alpha"] = g["alpha"]
        rep["alpha_oracle"] = orc.alpha
    return rep


def _bsr_keys(row_ptr, col, n):
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(np.asarray(row_ptr, np.int64)))
    return rows * n + np.asarray(col, np.int64)


def _compare_bsr(sc, g, orc: O.PassResult, diff: set) -> dict:
    """BSR pattern and values of the GPU against the oracle.

    Pairs of the tie band whose activity differs between the two sides
    (``diff``) touch the blocks of their stencil vertices on one side only.
    Those blocks are set apart: every other block must be present on both
    sides (bit-exact pattern) and agree within 1e-9 of its scale.  A set-apart
    block may differ only by what a pair within 1e-12 of its activation
    threshold contributes: b'' there is of the order of the threshold's
    relative distance, so such a pair's entries stay below 1e-8 kappa.
    Returns ``bsr_compared`` (blocks checked) and ``bsr_blocks_skipped``."""
    n = sc.n
    rp, col, val = g["bsr"]
    kg = _bsr_keys(rp, col, n)
    ko = _bsr_keys(orc.bsr_row_ptr, orc.bsr_col, n)
    if not diff:
        assert np.array_equal(rp, orc.bsr_row_ptr) and np.array_equal(col, orc.bsr_col), "BSR pattern differs"
        excl = np.zeros(0, np.int64)
    else:
        st = O.stencils(O.topology(sc), np.array(sorted(diff), np.uint64))
        excl = np.unique((st[:, :, None] * n + st[:, None, :]).reshape(-1))
    sg = ~np.isin(kg, excl)
    so = ~np.isin(ko, excl)
    assert np.array_equal(kg[sg], ko[so]), "BSR pattern differs outside the blocks of tie-band pairs"
    vg, vo, va = val[sg], orc.bsr_val[so], orc.bsr_abs[so]
    verr = np.abs(vg - vo)
    if not np.all(verr <= 1e-9 * va + 1e-30):
        ratio = verr / (va + 1e-300)
        q = int(np.argmax(ratio.reshape(ratio.shape[0], -1).max(axis=1)))
        kq = int(kg[sg][q])
        raise AssertionError(
            f"BSR value err {float(ratio.max())} at block (row {kq // n}, col {kq % n}): "
            f"gpu {vg[q].ravel().tolist()} oracle {vo[q].ravel().tolist()} scale {va[q].ravel().tolist()}")
    if excl.size:
        kap = float(sc.kappa)
        # blocks present on one side only: the tie-band pairs' own entries
        for keys, v, sel in ((kg, val, ~sg), (ko, orc.bsr_val, ~so)):
            other = ko[~so] if keys is kg else kg[~sg]
            only = ~np.isin(keys[sel], other)
            assert np.all(np.abs(v[sel][only]) <= 1e-8 * kap), "a tie-band pair's block is not negligible"
        both_g = np.isin(kg, ko[~so]) & ~sg
        both_o = np.isin(ko, kg[~sg]) & ~so
        d = np.abs(val[both_g] - orc.bsr_val[both_o])
        assert np.all(d <= 1e-9 * orc.bsr_abs[both_o] + 1e-8 * kap), "tie-band blocks differ"
    return {"bsr_compared": int(sg.sum()), "bsr_blocks_skipped": int((~sg).sum()),
            "bsr_relerr": float((verr / (va + 1e-300)).max()) if verr.size else 0.0}


def run_gpu_batch(scenes, mode="double", xs=None, ps=None, **kw):
    """One batched pass over several scenes (cb_batch_create); returns one
    result dict per member in run_gpu's format (member-local numbering)."""
    import torch
    from paper_2510_10256_gb300.contact import ContactBatch, ContactScene
    dev = torch.device("cuda:0")
    members = [ContactScene.from_scene(sc, mode=mode, **kw) for sc in scenes]
    dbar = [m.stats()["dbar_min"] for m in members]
    b = ContactBatch(members)
    for m in members:
        m.close()
    xs = xs or [sc.x for sc in scenes]
    ps = ps or [sc.p for sc in scenes]
    x = torch.from_numpy(np.ascontiguousarray(np.concatenate(xs, axis=1))).to(dev)
    p = torch.from_numpy(np.ascontiguousarray(np.concatenate(ps, axis=1))).to(dev)
    M = len(scenes)
    energy = torch.zeros(M, dtype=torch.float64, device=dev)
    grad = torch.zeros(3, b.n, dtype=torch.float64, device=dev)
    alpha = torch.zeros(M, dtype=torch.float64, device=dev)
    b.run_pass(x, p, energy, grad, alpha)
    torch.cuda.synchronize()
    C, F, CC, fr = b.pairs("candidate"), b.pairs("filtered"), b.pairs("core"), b.pairs("rest_filtered")
    A, ccd = b.active(), b.ccd()
    rp, col, val = b.bsr()
    en, al, gr = energy.cpu().numpy(), alpha.cpu().numpy(), grad.cpu().numpy()
    status = b.sync_status()
    out = []
    for m in range(M):
        vo, vn = int(b.vert_offsets[m]), int(b.vert_offsets[m + 1])

        def sel(keys):
            return b.to_member_keys(keys[b.member_of_keys(keys) == m], m) if keys.size else keys

        am = b.member_of_keys(A["keys"]) == m if A["keys"].size else np.zeros(0, bool)
        cm = b.member_of_keys(ccd["keys"]) == m if ccd["keys"].size else np.zeros(0, bool)
        lrp = rp[vo:vn + 1] - rp[vo]
        out.append(dict(
            C=sel(C), F=sel(F), CC=sel(CC), frest=sel(fr),
            A=dict(keys=b.to_member_keys(A["keys"][am], m), d=A["d"][am], klass=A["klass"][am],
                   dtype=A["dtype"][am]),
            ccd=dict(keys=b.to_member_keys(ccd["keys"][cm], m), t=ccd["t"][cm], klass=ccd["klass"][cm]),
            bsr=(lrp, col[rp[vo]:rp[vn]] - vo, val[rp[vo]:rp[vn]]),
            energy=float(en[m]), grad=gr[:, vo:vn], alpha=float(al[m]),
            stats=dict(dbar_min=dbar[m]), status=status))
    b.close()
    return out
