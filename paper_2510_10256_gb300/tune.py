"""Autotuner for the broad-phase knobs of a scene or batch.

The knobs change speed only, never results: the hash-cell edge (a factor
times the members' mean primitive box extent) and the block size of the
pair-enumeration kernel, separately for contact_build's broad phase (phase 0)
and ccd_step's swept broad phase (phase 1).  Each candidate is timed with the
library's own stage events on passes over the caller's data; the fastest is
kept and cached in a JSON file, keyed by the GPU, the scene kind, the vertex
count (octave) and the ratio of the activation to the mean edge length
(half octave): scenes alike in these have alike hash occupancy.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

FACTORS = (0.5, 0.71, 1.0, 1.41, 2.0, 2.83, 4.0)
BLOCKS = (128, 256)
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tuning.json")
# stage_ms index of the stage that contains each phase's broad phase
_STAGE = {0: 0, 1: 3}


def mean_edge(scene) -> float:
    """Mean edge length of the scene's rest mesh."""
    r = np.asarray(scene.rest)
    if scene.kind == "rod":
        rp = np.asarray(scene.rod_ptr)
        keep = np.ones(r.shape[1] - 1, bool)
        keep[rp[1:-1] - 1] = False  # no edge between consecutive polylines
        e = np.linalg.norm(np.diff(r, axis=1), axis=0)[keep]
    else:
        t = np.asarray(scene.tris)
        e = np.concatenate([np.linalg.norm(r[:, t[a]] - r[:, t[b]], axis=0) for a, b in ((0, 1), (1, 2), (0, 2))])
    return float(e.mean()) if e.size else 1.0


def scene_key(scenes, device_name: str = "") -> str:
    scenes = list(scenes)
    n = sum(sc.n for sc in scenes)
    ratios = sorted((sc.thickness + sc.dhat) / max(mean_edge(sc), 1e-300) for sc in scenes)
    med = ratios[len(ratios) // 2]
    return (f"{device_name}|{scenes[0].kind}|m{len(scenes) > 1:d}|n{int(round(math.log2(max(n, 1))))}"
            f"|a{round(2 * math.log2(max(med, 1e-12))) / 2:g}")


class Autotuner:
    def __init__(self, cache_path: str | None = DEFAULT_CACHE, factors=FACTORS, blocks=BLOCKS, reps: int = 2):
        self.path = cache_path
        self.factors = tuple(factors)
        self.blocks = tuple(blocks)
        self.reps = int(reps)
        self.cache = {}
        if self.path and os.path.exists(self.path):
            try:
                self.cache = json.load(open(self.path))
            except (OSError, ValueError):
                self.cache = {}

    def _save(self):
        if not self.path:
            return
        tmp = f"{self.path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(self.cache, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)

    @staticmethod
    def apply(runner, choice: dict):
        for ph in (0, 1):
            c = choice[str(ph)]
            runner.set_tuning(ph, c["cell_factor"], c["pair_block"])

    def tune(self, runner, key: str, run_pass, force: bool = False) -> dict:
        """Pick the knobs for `runner` (a ContactScene or ContactBatch);
        run_pass() must run one full pass on it.  Returns the choice per phase
        with the measured stage time, and whether it came from the cache."""
        if not force and key in self.cache:
            self.apply(runner, self.cache[key])
            return dict(self.cache[key], cached=True, key=key)
        runner.set_timing(True)
        choice = {}
        for ph in (0, 1):
            trials = []
            for f in self.factors:
                for b in self.blocks:
                    runner.set_tuning(ph, f, b)
                    run_pass()  # buffers settle to this setting's sizes
                    t = []
                    for _ in range(self.reps):
                        run_pass()
                        t.append(runner.stage_ms()[_STAGE[ph]])
                    trials.append((min(t), f, b))
            ms, f, b = min(trials)
            runner.set_tuning(ph, f, b)
            default = next((tm for tm, ff, bb in trials if ff == 1.0 and bb == 256), None)
            choice[str(ph)] = {"cell_factor": f, "pair_block": b, "stage_ms": ms, "default_ms": default,
                               "tried": len(trials)}
        self.cache[key] = choice
        self._save()
        return dict(choice, cached=False, key=key)
