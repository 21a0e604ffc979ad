"""Batched pass (several scenes, one launch per stage) against each member's
own oracle, and each member's result alone vs in the mix."""
import numpy as np
import pytest

import oracle as O
from paper_2510_10256_gb300 import scenes as S
from tests.parity import compare, run_gpu, run_gpu_batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_10256_gb300 import contact
    contact.build()
    contact.lib()


def test_rod_batch_matches_each_oracle():
    scenes = S.config(4, reduced=True) + [S.woven_patch(n_warp=3, n_weft=3, nseg=64), S.tiny_rods(5)]
    res = run_gpu_batch(scenes)
    for sc, g in zip(scenes, res):
        compare(sc, g, O.contact_pass(sc))


def test_shell_batch_matches_each_oracle():
    scenes = [S.tiny_shell(1), S.pleated_sheet(nx=24), S.tiny_shell(2, nx=6, thickness=0.3, dhat=0.07),
              S.graded_disk(target_tris=3000, L0=0.5)]
    res = run_gpu_batch(scenes)
    for sc, g in zip(scenes, res):
        compare(sc, g, O.contact_pass(sc))


def test_alone_equals_in_the_mix():
    """Each member's result in the batch equals its result alone: identical
    pair sets and step bound, numerics within the parity tolerance (the
    oracle's per-entry scale; only the atomic summation order differs)."""
    scenes = [S.tiny_shell(7), S.pleated_sheet(nx=20), S.tiny_shell(8)]
    mix = run_gpu_batch(scenes)
    for sc, g in zip(scenes, mix):
        alone = run_gpu(sc)
        orc = O.contact_pass(sc, ccd=False)
        for k in ("C", "F", "CC"):
            assert np.array_equal(alone[k], g[k])
        assert np.array_equal(alone["A"]["keys"], g["A"]["keys"])
        assert np.array_equal(alone["ccd"]["keys"], g["ccd"]["keys"])
        assert alone["alpha"] == g["alpha"]
        assert abs(alone["energy"] - g["energy"]) <= 1e-9 * max(abs(alone["energy"]), 1e-300)
        assert np.all(np.abs(alone["grad"] - g["grad"]) <= 1e-9 * orc.grad_abs + 1e-30)
        assert np.array_equal(alone["bsr"][0], g["bsr"][0]) and np.array_equal(alone["bsr"][1], g["bsr"][1])
        assert np.all(np.abs(alone["bsr"][2] - g["bsr"][2]) <= 1e-9 * orc.bsr_abs + 1e-30)


def test_single_member_batch():
    sc = S.tiny_shell(4)
    (g,) = run_gpu_batch([sc])
    compare(sc, g, O.contact_pass(sc))


def test_repeated_batches_match_the_oracle():
    """Several consecutive batched passes, each against the oracle.  Guards
    the projection kernel's shared-memory phases: the FP64 matrices share
    bytes with other threads' FP32 work arrays, so no thread may start its
    FP64 stage before the whole block has finished the FP32 one."""
    scenes = [S.tiny_shell(7), S.pleated_sheet(nx=20), S.tiny_shell(8)]
    orcs = [O.contact_pass(sc) for sc in scenes]
    for _ in range(4):
        for sc, g, o in zip(scenes, run_gpu_batch(scenes), orcs):
            compare(sc, g, o)


@pytest.mark.slow
def test_rod_batch_64_full_size():
    """The full 64-scene rod batch (1.09 M vertices) in one batched pass,
    every member against its own oracle."""
    scenes = S.rod_batch()
    res = run_gpu_batch(scenes)
    total = compared = skipped = 0
    for sc, g in zip(scenes, res):
        rep = compare(sc, g, O.contact_pass(sc))
        total += rep["C"]
        compared += rep["bsr_compared"]
        skipped += rep["bsr_blocks_skipped"]
    print("rod batch 64", {"candidates": total, "bsr_compared": compared, "bsr_blocks_skipped": skipped})
    assert total > 5_000_000
    assert compared > 0 and skipped <= 1e-4 * compared, (compared, skipped)
