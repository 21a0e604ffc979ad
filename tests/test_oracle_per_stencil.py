"""Per-stencil activation in the oracle (contact_pass(per_stencil=True)):
a filtered candidate whose boxes, inflated by half its own width, do not
overlap is dropped.  Such a pair is farther apart than that width, so it is
inactive; the pass's energy, gradient, BSR and active set must therefore be
identical, only the candidate set shrinks (the paper's remark that
per-stencil hashing would only trim false positives, Sec. 3.3)."""
import numpy as np
import pytest

import oracle as O
from paper_2510_10256_gb300 import scenes as S


@pytest.mark.parametrize("make", [lambda: S.pleated_sheet(nx=40), lambda: S.tiny_shell(3),
                                  lambda: S.woven_patch(n_warp=2, n_weft=2, nseg=48), lambda: S.ring_chain()])
def test_per_stencil_changes_only_the_candidates(make):
    sc = make()
    a = O.contact_pass(sc, ccd=False)
    b = O.contact_pass(sc, ccd=False, per_stencil=True)
    assert set(b.C.tolist()) <= set(a.C.tolist())
    assert np.array_equal(a.C[a.active], b.C[b.active])
    assert a.energy == b.energy
    assert np.array_equal(a.grad, b.grad)
    assert np.array_equal(a.bsr_row_ptr, b.bsr_row_ptr) and np.array_equal(a.bsr_col, b.bsr_col)
    assert np.array_equal(a.bsr_val, b.bsr_val)
    # every dropped pair was filtered and inactive
    dropped = np.setdiff1d(a.C, b.C)
    idx = np.searchsorted(a.C, dropped)
    assert np.all(a.klass[idx] == O.KLASS_F) and not np.any(a.active[idx])


def test_per_stencil_halves_the_pleated_candidates():
    sc = S.pleated_sheet(nx=64)
    a = O.contact_pass(sc, ccd=False)
    b = O.contact_pass(sc, ccd=False, per_stencil=True)
    assert b.C.size < 0.6 * a.C.size
    assert (b.klass == O.KLASS_F).sum() < 0.2 * (a.klass == O.KLASS_F).sum()
