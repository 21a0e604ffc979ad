"""Autotuner selection and cache logic on the host, with a fake runner whose
stage times are a known function of the knobs."""
import json

import numpy as np

from paper_2510_10256_gb300 import scenes as S
from paper_2510_10256_gb300.tune import Autotuner, mean_edge, scene_key


class FakeRunner:
    def __init__(self):
        self.knobs = {0: (1.0, 256), 1: (1.0, 256)}
        self.passes = 0

    def set_timing(self, on=True):
        pass

    def set_tuning(self, ph, f, b):
        self.knobs[ph] = (f, b)

    def stage_ms(self):
        # phase 0 is fastest at (0.71, 128), phase 1 at (1.41, 256)
        f0, b0 = self.knobs[0]
        f1, b1 = self.knobs[1]
        t0 = 1.0 + abs(np.log2(f0 / 0.71)) + (0.1 if b0 != 128 else 0.0)
        t1 = 2.0 + abs(np.log2(f1 / 1.41)) + (0.1 if b1 != 256 else 0.0)
        return [t0, 0.1, 5.0, t1, 4.0]

    def run(self):
        self.passes += 1


def test_picks_fastest_per_phase_and_caches(tmp_path):
    path = str(tmp_path / "tune.json")
    r = FakeRunner()
    c = Autotuner(path).tune(r, "k", r.run)
    assert not c["cached"]
    assert (c["0"]["cell_factor"], c["0"]["pair_block"]) == (0.71, 128)
    assert (c["1"]["cell_factor"], c["1"]["pair_block"]) == (1.41, 256)
    assert r.knobs == {0: (0.71, 128), 1: (1.41, 256)}
    assert c["0"]["stage_ms"] <= c["0"]["default_ms"]
    assert r.passes == 2 * 7 * 2 * 3
    assert "k" in json.load(open(path))
    # a second tuner reads the cache and applies it without running passes
    r2 = FakeRunner()
    c2 = Autotuner(path).tune(r2, "k", r2.run)
    assert c2["cached"] and r2.passes == 0 and r2.knobs == r.knobs


def test_scene_key_and_mean_edge():
    rod = S.straight_rod(n_seg=10, seg=0.1)
    assert abs(mean_edge(rod) - 0.1) < 1e-12
    grid = S.flat_grid(nx=5)
    assert mean_edge(grid) > 0
    k1 = scene_key([rod], "gpu")
    k2 = scene_key([rod], "gpu")
    assert k1 == k2 and k1.startswith("gpu|rod|m0|")
    assert scene_key([rod, rod], "gpu") != k1
