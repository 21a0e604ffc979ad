#!/usr/bin/env python3
"""Contact-pass benchmark: stages a-e (broad phase, filter, distances, barrier +
PSD Hessian + assembly, CCD step bound) of the barrier-filtered contact model on
one synthetic scene per GPU.

Metric: contact pairs/s = |C| / T_pass, where |C| is the broad-phase candidate
count of the pass and T_pass the device time of the whole pass (CUDA events on
the launching stream).  N GPUs run N independent replicas (weak scaling); the
value is the sum over ranks, the time the max over ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl {gb300,reference}]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "contact pairs/s (filter+barrier+Hessian+CCD)"
UNIT = "pairs/s"
# FP64 peak from the part's unit counts and clock: 152 SMs x 2070 MHz x 4 FP64
# flop/clk/SM (2 DFMA) = 1.26 TFLOP/s, the 1.25 TFLOP/s dense FP64 figure.
FP64_PEAK_TFLOPS = 152 * 2.070e9 * 4 / 1e12
# FP64 flop of the stage-(d) kernels per pair each one handles: DADD + DMUL +
# 2 DFMA thread instructions executed, counted by ncu on the 128x128 pleated
# sheet (195,263 active pairs: 30,807 face / line-line, 151,976 point-edge in
# their frame) and divided by the pairs of each kernel.  k_hess_prep per
# active pair, k_hess_proj<9> per face / line-line pair, k_hess_proj_pe per
# point-edge pair in its own frame; k_hess_proj<6> (generic point-edge pairs,
# none in that capture) is scaled from k_hess_proj<9> by (6/9)^3.
HESS_FLOPS = {"prep": 549.1, "face": 11471.0, "pe_frame": 1091.0, "pe": 11471.0 * (6 / 9) ** 3}
# DRAM bytes (read + write) of the stage-(d) kernels per active pair, from one
# ncu capture of a full-size pass (256x256 sheet, 805,423 active pairs):
# k_hess_prep 289.1 MB, k_hess_proj_pe 266.8 MB, k_hess_proj<9> 191.5 MB,
# k_hess_proj<6> 0.1 MB
HESS_DRAM_BYTES_PER_ACTIVE = 747.48e6 / 805423
HESS_TRAFFIC_SOURCE = "ncu dram__bytes_read+write of the four stage-(d) kernels of one 256x256 pass, per active pair"


def hess_flops(st) -> float:
    """FP64 flop of one pass's stage-(d) kernels: per-kernel counts per pair
    times the pairs each kernel handled."""
    return (HESS_FLOPS["prep"] * st["n_active"] + HESS_FLOPS["face"] * st["n_hess_face"]
            + HESS_FLOPS["pe_frame"] * st["n_hess_pe_frame"] + HESS_FLOPS["pe"] * st["n_hess_pe"])
L2_FLUSH_BYTES = 256 << 20


def max_over_ranks(values, dist, device):
    """Element-wise maximum of per-rank timings over all ranks (the slowest
    replica sets the job's time); identity without a process group."""
    if not dist:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def _peaks() -> dict:
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def _edge_count(scenes) -> int:
    import numpy as np
    E = 0
    for sc in scenes:
        if sc.kind == "rod":
            E += sc.n - (len(sc.rod_ptr) - 1)
        else:
            t = np.asarray(sc.tris)
            e = np.concatenate([np.sort(np.stack([t[a], t[b]], 1), 1) for a, b in ((0, 1), (1, 2), (0, 2))])
            E += np.unique(e, axis=0).shape[0]
    return E


def stage_roofline(st: dict, med: list, scenes) -> dict:
    """Per stage: algorithmic bytes (what the method must move: inputs read
    once, outputs written once; no hash, sort or re-gather traffic) over the
    stage's device time, against the measured HBM copy bandwidth; stage (d)
    also against the FP64 peak.  Bytes per stage:
      a  24n + 12T + 8E + 8|C|          (positions, topology, candidate keys)
      b  16|C| + table                  (keys in, classes out; rods 12E, shells 4|F_rest|)
      cd 8|C| + 24n + 8|A| + 24n + 76 nnzb + 4(n+1)  (keys+x in; active, gradient, BSR out)
         of which c: 8|C| + 24n (keys, x in) and d: 8|A| + 24n + 76 nnzb + 4(n+1)
      e  8|C_ccd| + 48n + 8             (keys, x, p in; alpha out)"""
    n = sum(sc.n for sc in scenes)
    T = sum(sc.tris.shape[1] for sc in scenes if sc.kind == "shell")
    E = _edge_count(scenes)
    C, A, nnzb, Cc = st["n_candidates"], st["n_active"], st["nnzb"], st["n_ccd"]
    shell = scenes[0].kind == "shell"
    table = 4 * st["n_rest_filtered"] if shell else 12 * E
    by = {"contact_build": 24 * n + 12 * T + 8 * E + 8 * C,
          "contact_filter": 16 * C + table,
          "barrier_eval": 8 * C + 24 * n + 8 * A + 24 * n + 76 * nnzb + 4 * (n + 1),
          "distances_c": 8 * C + 24 * n,
          "assembly_d": 8 * A + 24 * n + 76 * nnzb + 4 * (n + 1),
          "ccd_step": 8 * Cc + 48 * n + 8}
    hbm = _peaks().get("hbm_gbs")
    out = {"hbm_peak_gbs": hbm, "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy)" if hbm else None}
    idx = {"contact_build": 0, "contact_filter": 1, "barrier_eval": 2, "ccd_step": 3, "distances_c": 5,
           "assembly_d": 6}
    for k, i in idx.items():
        ms = med[i] if i < len(med) else 0.0
        gbs = by[k] / (ms / 1000.0) / 1e9 if ms > 0 else None
        out[k] = {"bytes": int(by[k]), "ms": ms, "gbs": gbs, "hbm_frac": (gbs / hbm) if (gbs and hbm) else None}
    hess = med[4]
    out["hessian_kernels"] = {"ms": hess, "fp64_tflops": hess_flops(st) / (hess / 1000.0) / 1e12 if hess > 0
                              else None}
    if hess > 0:
        out["hessian_kernels"]["fp64_frac"] = out["hessian_kernels"]["fp64_tflops"] / FP64_PEAK_TFLOPS
    return out


def _autotune(args, runner, scenes, run_pass):
    """Broad-phase knobs from the autotuner (cached per GPU and scene class)."""
    if args.no_tune:
        return {"autotuned": False, "cell_factor": [runner.tuning(0)[0], runner.tuning(1)[0]]}
    import torch
    from paper_2510_10256_gb300.tune import Autotuner, scene_key
    key = scene_key(scenes, torch.cuda.get_device_name())
    c = Autotuner().tune(runner, key, run_pass)
    torch.cuda.synchronize()
    return {"autotuned": True, "cached": c["cached"],
            "build": {k: c["0"][k] for k in ("cell_factor", "pair_block", "stage_ms", "default_ms")},
            "ccd": {k: c["1"][k] for k in ("cell_factor", "pair_block", "stage_ms", "default_ms")}}


def _workload(name: str, reduced_nx: int | None = None):
    from paper_2510_10256_gb300 import scenes as S
    if name == "pleated":
        nx = reduced_nx or 256
        sc = S.pleated_sheet(nx=nx)
        desc = f"pleated shell {nx}x{nx} grid ({sc.tris.shape[1]} tris), L 0.5 mm, thickness 1 mm, dhat 0.05 mm"
    elif name == "woven":
        sc = S.woven_patch()
        desc = "woven rod patch 16 x 257 vertices, r 0.1 mm, dhat 0.01 mm"
    elif name == "graded":
        sc = S.graded_disk(target_tris=200_000 if not reduced_nx else 6000, L0=0.1 if not reduced_nx else 0.5)
        desc = f"graded twisted disk ({sc.tris.shape[1]} tris), 0.1-4 mm edges, thickness 1 mm"
    elif name == "chain":
        n_rings = reduced_nx or 2000
        sc = S.ring_chain(n_rings=n_rings, m=96)
        desc = (f"chain of {n_rings} interlocked closed yarn loops x 96 segments ({sc.n} vertices), "
                f"R 1 mm, thickness 0.3 mm, dhat 0.05 mm")
    else:
        raise ValueError(name)
    return sc, desc


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [c.strip() for c in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _oracle_sample(scenes, what: str) -> dict:
    """One full oracle pass (a-e) over each scene, timed on this host's cores."""
    import oracle as O
    O.build()
    t0 = time.perf_counter()
    nc = 0
    for sc in scenes:
        nc += O.contact_pass(sc).C.size
    dt = time.perf_counter() - t0
    return {"value": nc / dt, "unit": UNIT, "cores": O.lib().orc_num_threads(), "kind": "oracle",
            "sample": f"{what} (|C| = {nc}, {dt:.1f} s); brute force O(n^2) pair enumeration"}


def cpu_baseline(workload: str, nx: int) -> dict:
    """The oracle as it stands on this host's cores, on a bounded sample of
    the same workload (seconds of CPU work)."""
    from paper_2510_10256_gb300 import scenes as S
    if workload == "pleated":
        sc, _ = _workload("pleated", reduced_nx=nx)
        return _oracle_sample([sc], f"one oracle pass on the pleated-sheet recipe at {nx}x{nx} vertices")
    if workload == "woven":
        sc, _ = _workload("woven")
        return _oracle_sample([sc], "one oracle pass on the full woven patch")
    if workload == "graded":
        sc = S.graded_disk(target_tris=50_000, L0=0.2)
        return _oracle_sample([sc], f"one oracle pass on the graded-disk recipe at {sc.tris.shape[1]} triangles")
    if workload == "chain":
        sc = S.ring_chain(n_rings=500, m=96)
        return _oracle_sample([sc], "one oracle pass on a 500-loop chain of the same recipe")
    if workload == "knit64":
        scenes = S.rod_batch()[::4]
        return _oracle_sample(scenes, f"one oracle pass on every fourth scene of the batch ({len(scenes)} scenes)")
    if workload == "serve":
        pool = S.serve_pool()
        sample = [min((sc for sc in pool if sc.kind == k), key=lambda sc: sc.n) for k in ("rod", "shell")]
        return _oracle_sample(sample, "one oracle pass on the smallest rod and the smallest shell of the pool")
    raise ValueError(workload)


def run_reference(args, rank: int, world: int):
    """Reference arm: the CPU oracle timed as it stands, rank 0 only."""
    if rank != 0:
        return
    import oracle as O
    O.build()
    nx = args.ref_nx
    sc, desc = _workload("pleated", reduced_nx=nx)
    for _ in range(args.warmup):
        O.contact_pass(sc)
    times, nc = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = O.contact_pass(sc)
        times.append(time.perf_counter() - t0)
        nc = r.C.size
    ms = 1000.0 * statistics.median(times)
    val = nc / (ms / 1000.0)
    cores = O.lib().orc_num_threads()
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{desc} (oracle sample of the pleated 256x256 workload)", "candidates": int(nc)},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"pleated-sheet recipe at {nx}x{nx} vertices per step"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _timed_steps(run, steps, flush, stream):
    """Device time (ms) of each of `steps` calls of run(), L2 flushed before each."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        run()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def bench_batch(args, rank, world, local, dist):
    """64 rod scenes (weave / knit, 1k-64k vertices each): the batched pass (one
    launch per stage for all scenes) against the plain form (one scene per
    launch sequence, the 64 scenes one after another on the same stream)."""
    import numpy as np
    import torch
    from paper_2510_10256_gb300 import contact as CT
    from paper_2510_10256_gb300 import scenes as S
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    scenes = S.rod_batch()
    members = [CT.ContactScene.from_scene(sc) for sc in scenes]
    batch = CT.ContactBatch(members)
    M, N = len(scenes), batch.n
    xs = [torch.from_numpy(sc.x).to(dev) for sc in scenes]
    ps = [torch.from_numpy(sc.p).to(dev) for sc in scenes]
    es = [torch.zeros(1, dtype=torch.float64, device=dev) for _ in scenes]
    gs = [torch.zeros(3, sc.n, dtype=torch.float64, device=dev) for sc in scenes]
    als = [torch.zeros(1, dtype=torch.float64, device=dev) for _ in scenes]
    hx_np = np.ascontiguousarray(np.concatenate([sc.x for sc in scenes], axis=1))
    hp_np = np.ascontiguousarray(np.concatenate([sc.p for sc in scenes], axis=1))
    x = torch.from_numpy(hx_np).to(dev)
    p = torch.from_numpy(hp_np).to(dev)
    energy = torch.zeros(M, dtype=torch.float64, device=dev)
    grad = torch.zeros(3, N, dtype=torch.float64, device=dev)
    alpha = torch.zeros(M, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def run_batched():
        batch.run_pass(x, p, energy, grad, alpha)

    def run_plain():
        for k, m in enumerate(members):
            m.run_pass(xs[k], ps[k], es[k], gs[k], als[k])

    tuning = _autotune(args, batch, scenes, run_batched)
    if not args.no_plain:  # the plain arm uses the same knobs
        for m in members:
            for ph in (0, 1):
                m.set_tuning(ph, *batch.tuning(ph))
    batch.set_timing(True)
    for _ in range(args.warmup):
        run_batched()
        if not args.no_plain:
            run_plain()
    torch.cuda.synchronize()
    st = batch.stats()
    n_cand = int(st["n_candidates"])
    if not args.no_plain:  # the batch forms exactly the members' own pairs
        assert n_cand == sum(int(m.stats()["n_candidates"]) for m in members)
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = CT.kernel_launches()
    stage = []

    def run_b():
        run_batched()
        stage.append(batch.stage_ms())

    b_ms = _timed_steps(run_b, args.steps, flush, stream)
    launches = CT.kernel_launches() - l0
    p_ms = _timed_steps(run_plain, args.steps, flush, stream) if not args.no_plain else [float("nan")]
    clk = clocks.stop()
    ms, pms = statistics.median(b_ms), statistics.median(p_ms)
    ms, pms = max_over_ranks([ms, pms], dist, dev)
    # end to end: pinned host x, p in; energy, alpha, gradient out
    hx, hp = torch.from_numpy(hx_np).pin_memory(), torch.from_numpy(hp_np).pin_memory()
    he = torch.zeros(M, dtype=torch.float64).pin_memory()
    ha = torch.zeros(M, dtype=torch.float64).pin_memory()
    hg = torch.zeros(3, N, dtype=torch.float64).pin_memory()

    def run_e2e():
        x.copy_(hx, non_blocking=True)
        p.copy_(hp, non_blocking=True)
        run_batched()
        he.copy_(energy, non_blocking=True)
        ha.copy_(alpha, non_blocking=True)
        hg.copy_(grad, non_blocking=True)

    e2e_ms = statistics.mean(_timed_steps(run_e2e, max(3, args.steps // 2), flush, stream))
    if rank != 0:
        return
    hess_ms = statistics.mean(s[4] for s in stage)
    med = [statistics.median(s[i] for s in stage) for i in range(7)]
    na = int(st["n_active"])
    achieved = hess_flops(st) / (hess_ms / 1000.0) / 1e12 if hess_ms > 0 else 0.0
    sizes = [sc.n for sc in scenes]
    line = {"metric": METRIC, "value": world * n_cand / (ms / 1000.0), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{M} rod scenes (even: plain weave, odd: helix-loop knit), "
                                   f"{min(sizes)}-{max(sizes)} vertices each, {N} in all, batched",
                       "candidates": n_cand, "active": na, "ccd_pairs": int(st["n_ccd"]), "nnzb": int(st["nnzb"]),
                       "ccd_max_iters": int(st["ccd_max_iters"]), "tuning": tuning,
                       "l2": "flushed (256 MiB write) between steps", "parallelism": f"replicas x{world}"},
            "plain": {"value": world * n_cand / (pms / 1000.0), "unit": UNIT, "ms_per_step": pms,
                      "form": f"{M} single-scene passes in sequence on one stream"},
            "batched_over_plain": pms / ms,
            "stage_roofline": stage_roofline(st, med, scenes),
            "fp32_broad_phase": {"candidates_fp32": st["n_candidates_fp32"], "candidates": n_cand,
                                 "superset_ratio": st["n_candidates_fp32"] / max(1, n_cand),
                                 "fp64_decided": st["n_fp64_decided"]},
            "stage_ms": _stage_dict(med),
            "roofline": {"bound": "alu", "kernel": "k_hess_prep + k_hess_proj<9> + k_hess_proj_pe (FP64 stage d)", "achieved": achieved,
                         "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                         "traffic": None, "flops_per_pass": hess_flops(st), "kernel_ms": hess_ms,
                         "peak_source": "derived: 152 SM x 2070 MHz x 4 FP64 flop/clk/SM"},
            "e2e": {"value": world * n_cand / (e2e_ms / 1000.0), "unit": UNIT, "ms_per_step": e2e_ms,
                    "h2d_bytes_per_step": 2 * 3 * N * 8, "d2h_bytes_per_step": 2 * M * 8 + 3 * N * 8},
            "clocks": clk, "gpu_launches": int(launches), "status": batch.sync_status()}
    if not args.no_cpu_baseline and world == 1:
        try:
            line["cpu_baseline"] = cpu_baseline(args.workload, args.cpu_nx)
        except Exception as e:  # the baseline is context; never fail the bench on it
            line["cpu_baseline"] = {"value": None, "error": str(e)}
    print(json.dumps(line), flush=True)


def _serve_config(pool, n, rate, steps, budget_gb, slots) -> dict:
    rods = [s.n for s in pool if s.kind == "rod"]
    tris = [s.tris.shape[1] for s in pool if s.kind == "shell"]
    return {"workload": f"served stream: {n} Poisson requests at {rate:g}/s, {steps} contact steps each, "
                        f"rods {min(rods)}-{max(rods)} vertices / shells {min(tris)}-{max(tris)} triangles "
                        f"(pool of {len(pool)} seeded scenes), half and half",
            "hbm_budget_gb": budget_gb, "slots": slots}


def serve_measure(eng, pool, n, rate, steps, budget_gb, slots, seed, plain=False) -> dict:
    """One served stream (continuous batching, paper_2510_10256_gb300.serve) or
    its plain form (the same trace FIFO, one single-scene pass per step):
    throughput and per-step latency, with the kernel launches it made."""
    from paper_2510_10256_gb300 import contact as CT
    from paper_2510_10256_gb300.serve import Server, poisson_requests, run_plain
    reqs = poisson_requests(pool, n, rate, steps, seed=seed)
    l0 = CT.kernel_launches()
    if plain:
        rep = run_plain(eng, reqs)
    else:
        rep = Server(eng, hbm_budget=int(budget_gb * (1 << 30)), max_slots=slots).run(reqs)
    launches = CT.kernel_launches() - l0
    lat = rep["step_latency_ms"]
    return {"form": "plain: FIFO, one request at a time, each step a single-scene pass" if plain else
            "served: continuous batching under the HBM budget",
            "rate_per_s": rate, "requests": rep["requests"], "rejected": len(rep["rejected"]),
            "steps": rep["steps"], "pairs": rep["pairs"], "wall_s": rep["wall_s"],
            "pairs_per_s": rep["pairs"] / rep["wall_s"] if rep["wall_s"] > 0 else 0.0,
            "steps_per_s": rep["steps_per_s"], "iterations": rep["iterations"],
            "max_resident": rep["max_resident"], "peak_reserved_gb": rep["peak_reserved_bytes"] / 2 ** 30,
            "latency_ms": {"step_p50": lat["p50"], "step_p99": lat["p99"], "step_mean": lat["mean"],
                           "queue_p50": rep["queue_delay_ms"]["p50"], "queue_p99": rep["queue_delay_ms"]["p99"],
                           "load_p50": rep["load_ms"]["p50"], "load_p99": rep["load_ms"]["p99"]},
            "gpu_launches": int(launches), "_h2d": sum(
                8 * r.scene.rest.size + 8 * r.scene.x.size + 4 * (r.scene.tris.size if r.scene.tris is not None
                                                                  else r.scene.rod_ptr.size) for r in reqs)}


def _serve_engine(local, warmup):
    import torch
    from paper_2510_10256_gb300 import scenes as S
    from paper_2510_10256_gb300.serve import DeviceEngine
    pool = S.serve_pool()
    eng = DeviceEngine(torch.device("cuda", local))
    small = sorted(pool, key=lambda sc: sc.n)
    sample = [next(sc for sc in small if sc.kind == k) for k in ("rod", "shell")]
    sample += [next(sc for sc in small if sc.kind == "shell" and sc.name != sample[1].name)]
    bpv = None
    for _ in range(max(1, warmup // len(sample))):
        bpv = eng.calibrate(sample)
    torch.cuda.synchronize()
    return pool, eng, bpv


def serve_suite(args, local, seed, n_req, sustain_rate, sustain_n) -> dict:
    """The served stream at the configured arrival rate, its plain form on the
    same trace, and the served stream at an arrival rate one GPU sustains."""
    pool, eng, bpv = _serve_engine(local, args.warmup)
    try:
        served = serve_measure(eng, pool, n_req, args.rate, args.req_steps, args.budget_gb, args.slots, seed)
        plain = serve_measure(eng, pool, n_req, args.rate, args.req_steps, args.budget_gb, args.slots, seed,
                              plain=True)
        sustained = serve_measure(eng, pool, sustain_n, sustain_rate, args.req_steps, args.budget_gb, args.slots,
                                  seed + 1)
    finally:
        eng.close()
    for r in (served, plain, sustained):
        r.pop("_h2d", None)
    return {"config": dict(_serve_config(pool, n_req, args.rate, args.req_steps, args.budget_gb, args.slots),
                           bytes_per_vertex_model=bpv),
            "served": served, "plain": plain, "served_over_plain": served["pairs_per_s"] / plain["pairs_per_s"]
            if plain["pairs_per_s"] > 0 else None, "sustained": sustained}


def bench_serve(args, rank, world, local, dist):
    """Served request stream: Poisson arrivals, each request a sequence of
    contact steps on its own scene (rods 5k-200k vertices, shells 10k-500k
    triangles, half and half), admitted under an HBM budget and advanced by
    continuous batching (paper_2510_10256_gb300.serve); beside it the same
    trace in its plain form (FIFO, one single-scene pass per step)."""
    import torch
    from paper_2510_10256_gb300 import scenes as S
    pool, eng, bpv = _serve_engine(local, args.warmup)
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    seed = S.BASE_SEED + 5 + rank
    rep = serve_measure(eng, pool, args.requests, args.rate, args.req_steps, args.budget_gb, args.slots, seed)
    torch.cuda.synchronize()
    clk = clocks.stop()
    wall = max_over_ranks([rep["wall_s"]], dist, torch.device("cuda", local))[0]
    plain = None
    if not args.no_plain:
        plain = serve_measure(eng, pool, args.requests, args.rate, args.req_steps, args.budget_gb, args.slots, seed,
                              plain=True)
        plain.pop("_h2d", None)
    eng.close()
    if rank != 0:
        return
    h2d = rep.pop("_h2d")
    steps = max(1, rep["steps"])
    value = world * rep["pairs"] / wall
    lat = rep["latency_ms"]
    line = {"metric": "served contact pairs/s (filter+barrier+Hessian+CCD); p50/p99 step latency", "value": value,
            "unit": UNIT, "n_gpus": world, "steps": rep["steps"], "warmup": max(3, args.warmup),
            "ms_per_step": lat["step_p50"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": dict(_serve_config(pool, args.requests, args.rate, args.req_steps, args.budget_gb, args.slots),
                           bytes_per_vertex_model=bpv,
                           l2="not flushed: every iteration streams pair lists far larger than L2",
                           parallelism=f"replicas x{world}"),
            "latency_ms": lat, "served": rep,
            "plain": plain, "served_over_plain": (rep["pairs_per_s"] / plain["pairs_per_s"])
            if plain and plain["pairs_per_s"] > 0 else None,
            "roofline": None,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": h2d / steps, "d2h_bytes_per_step": 16,
                    "note": "the served stream is itself end to end: scenes uploaded from host memory at "
                            "admission, step results read back every step"},
            "clocks": clk, "gpu_launches": rep["gpu_launches"]}
    if not args.no_cpu_baseline and world == 1:
        try:
            line["cpu_baseline"] = cpu_baseline(args.workload, args.cpu_nx)
        except Exception as e:  # the baseline is context; never fail the bench on it
            line["cpu_baseline"] = {"value": None, "error": str(e)}
    print(json.dumps(line), flush=True)


def bench_friction(args, rank, world, local, dist):
    """Lagged friction on the pleated sheet: one barrier pass at x, friction_lag
    there (mu 0.4, eps 1e-3 mm), then per step friction_eval (energy, gradient,
    pair Hessians) at a displaced state and one friction_spmv.  Metric: lagged
    pairs per second through both calls."""
    import numpy as np
    import torch
    from paper_2510_10256_gb300 import contact as CT
    sc, desc = _workload("pleated", reduced_nx=args.nx or None)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    cs = CT.ContactScene.from_scene(sc)
    x = torch.from_numpy(sc.x).to(dev)
    energy = torch.zeros(1, dtype=torch.float64, device=dev)
    grad = torch.zeros(3, sc.n, dtype=torch.float64, device=dev)
    cs.contact_build(x)
    cs.contact_filter()
    cs.barrier_eval(x, energy, grad)
    mu, eps = 0.4, 1e-3
    cs.friction_lag(x, mu, eps)
    rng = np.random.default_rng(23)
    x1 = torch.from_numpy(sc.x + rng.normal(0.0, eps, size=sc.x.shape)).to(dev)
    v = torch.from_numpy(rng.normal(size=sc.x.shape)).to(dev)
    y = torch.zeros_like(v)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    fe = torch.zeros(1, dtype=torch.float64, device=dev)

    def step():
        fe.zero_()
        grad.zero_()
        y.zero_()
        cs.friction_eval(x1, x, fe, grad)
        cs.friction_spmv(v, y)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    nf = int(cs.friction(hessian=False)["keys"].size)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = CT.kernel_launches()
    for k in range(args.steps):
        flush.zero_()
        fe.zero_()
        grad.zero_()
        y.zero_()
        ev[k][0].record(stream)
        cs.friction_eval(x1, x, fe, grad)
        ev[k][1].record(stream)
        cs.friction_spmv(v, y)
        ev[k][2].record(stream)
    torch.cuda.synchronize()
    launches = CT.kernel_launches() - l0
    clk = clocks.stop()
    eval_ms = statistics.mean(a.elapsed_time(b) for a, b, _ in ev)
    spmv_ms = statistics.mean(b.elapsed_time(c) for _, b, c in ev)
    ms = max_over_ranks([eval_ms + spmv_ms], dist, dev)[0]
    # end to end: displaced state from pinned host memory, energy and gradient back
    hx = torch.from_numpy(x1.cpu().numpy()).pin_memory()
    he = torch.zeros(1, dtype=torch.float64).pin_memory()
    hg = torch.zeros(3, sc.n, dtype=torch.float64).pin_memory()
    e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(max(3, args.steps // 2))]
    for a, b in e_ev:
        flush.zero_()
        a.record(stream)
        x1.copy_(hx, non_blocking=True)
        fe.zero_()
        grad.zero_()
        y.zero_()
        cs.friction_eval(x1, x, fe, grad)
        cs.friction_spmv(v, y)
        he.copy_(fe, non_blocking=True)
        hg.copy_(grad, non_blocking=True)
        b.record(stream)
        stream.synchronize()
    e2e_ms = max_over_ranks([statistics.mean(a.elapsed_time(b) for a, b in e_ev)], dist, dev)[0]
    status = cs.sync_status()
    cs.close()
    if rank != 0:
        return
    # friction_eval's algorithmic bytes: per pair the stencil (16 B), lagged
    # data (64 B) and packed Hessian written (48 B); per vertex x and x_lag
    # read (48 B) and the gradient read and written (48 B)
    bytes_eval = nf * (16 + 64 + 48) + sc.n * (48 + 48)
    hbm = _peaks().get("hbm_gbs") or 6800.0
    achieved = bytes_eval / (eval_ms / 1000.0) / 1e9
    line = {"metric": "lagged friction pairs per second (friction_eval + friction_spmv)",
            "value": world * nf / (ms / 1000.0), "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"lagged friction on the {desc} (mu {mu}, eps {eps} mm, displaced by N(0, eps))",
                       "friction_pairs": nf, "l2": "flushed (256 MiB write) between steps",
                       "parallelism": f"replicas x{world}"},
            "stage_ms": {"friction_eval": eval_ms, "friction_spmv": spmv_ms},
            "roofline": {"bound": "hbm", "kernel": "k_fric_eval", "achieved": achieved, "peak": hbm,
                         "unit": "GB/s", "frac": achieved / hbm, "traffic": None,
                         "algorithmic_bytes": bytes_eval, "kernel_ms": eval_ms,
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy)"},
            "e2e": {"value": world * nf / (e2e_ms / 1000.0), "unit": "pairs/s",
                    "h2d_bytes_per_step": 3 * sc.n * 8, "d2h_bytes_per_step": 8 + 3 * sc.n * 8,
                    "ms_per_step": e2e_ms},
            "clocks": clk, "gpu_launches": int(launches), "status": status}
    if not args.no_cpu_baseline and world == 1:
        try:
            line["cpu_baseline"] = _friction_cpu_baseline(args.cpu_nx)
        except Exception as e:
            line["cpu_baseline"] = {"value": None, "error": str(e)}
    print(json.dumps(line), flush=True)


def _friction_cpu_baseline(nx: int) -> dict:
    """The friction oracle (lag + one evaluation) on a smaller pleated sheet."""
    import numpy as np
    import oracle as O
    import oracle.friction as Fr
    from paper_2510_10256_gb300 import scenes as S
    nx = min(nx, 48)
    sc = S.pleated_sheet(nx=nx)
    res = O.contact_pass(sc, ccd=False)
    L = Fr.lag(sc, res, sc.x, 0.4, 1e-3)
    rng = np.random.default_rng(23)
    x1 = sc.x + rng.normal(0.0, 1e-3, size=sc.x.shape)
    t0 = time.perf_counter()
    ev = Fr.evaluate(L, x1, sc.x)
    Fr.hessian_matvec(L, ev.Hw, rng.normal(size=sc.x.shape))
    dt = time.perf_counter() - t0
    return {"value": L.keys.size / dt, "unit": "pairs/s", "cores": 1, "kind": "oracle",
            "sample": f"friction oracle evaluate + Hessian product on the pleated recipe at {nx}x{nx} "
                      f"({L.keys.size} lagged pairs, {dt:.2f} s), one Python thread"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="pleated",
                    choices=["pleated", "woven", "graded", "knit64", "serve", "friction", "chain"])
    ap.add_argument("--requests", type=int, default=1000, help="serve: requests in the stream")
    ap.add_argument("--rate", type=float, default=200.0, help="serve: Poisson arrival rate (requests/s)")
    ap.add_argument("--req-steps", type=int, default=10, help="serve: contact steps per request")
    ap.add_argument("--budget-gb", type=float, default=150.0, help="serve: HBM admission budget")
    ap.add_argument("--slots", type=int, default=16, help="serve: most requests resident at once")
    ap.add_argument("--nx", type=int, default=0, help="pleated grid size (default: the full 256); chain: loops")
    ap.add_argument("--cpu-nx", type=int, default=128, help="grid size of the oracle baseline sample")
    ap.add_argument("--ref-nx", type=int, default=96, help="grid size of a reference-arm step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true",
                    help="knit64 / serve: skip the one-scene-per-launch (plain) arm")
    ap.add_argument("--no-tune", action="store_true", help="keep the default broad-phase knobs")
    ap.add_argument("--mollifier", action="store_true", help="single-scene workloads: IPC's edge-edge mollifier")
    ap.add_argument("--no-extras", action="store_true",
                    help="pleated: skip the graded disk and the served stream that the default line carries")
    ap.add_argument("--extra-requests", type=int, default=100, help="default line: requests of each served stream")
    ap.add_argument("--sustain-rate", type=float, default=10.0,
                    help="default line: arrival rate (requests/s) of the sustained served stream")
    ap.add_argument("--sustain-requests", type=int, default=100)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2510_10256_gb300 import build as B
    if rank == 0:
        B.build()
    if dist:
        dist.barrier()
    from paper_2510_10256_gb300 import contact as CT

    if args.workload == "knit64":
        bench_batch(args, rank, world, local, dist)
        return
    if args.workload == "serve":
        bench_serve(args, rank, world, local, dist)
        return
    if args.workload == "friction":
        bench_friction(args, rank, world, local, dist)
        return
    res = measure_single(args, args.workload, args.steps, local, dist, nx=args.nx or None,
                         mollifier=args.mollifier)
    extras = (args.workload == "pleated" and not args.nx and not args.no_extras and not args.mollifier)
    extra = {}
    if extras:
        # the larger single scene of the metric's configs, and the served stream
        g = measure_single(args, "graded", max(5, args.steps // 2), local, dist, clocks=False)
        extra["graded"] = _single_summary(g, world)
        from paper_2510_10256_gb300 import scenes as S
        extra["serve"] = serve_suite(args, local, S.BASE_SEED + 5 + rank, args.extra_requests, args.sustain_rate,
                                     args.sustain_requests)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    line = _single_line(args, res, world)
    if extras:
        sv = extra["serve"]["served"]
        line["latency_ms"] = {"step_p50": sv["latency_ms"]["step_p50"], "step_p99": sv["latency_ms"]["step_p99"],
                              "source": "the served stream in extra.serve.served"}
        line["extra"] = extra
    if not args.no_cpu_baseline and world == 1:
        try:
            line["cpu_baseline"] = cpu_baseline(args.workload, args.cpu_nx)
            if args.workload == "pleated":
                line["cpu_baseline"]["one_core"] = one_core_baselines()
        except Exception as e:  # the baseline is context; never fail the bench on it
            line["cpu_baseline"] = {"value": None, "error": str(e)}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def one_core_baselines() -> dict:
    """The oracle on one host core: the full woven rod patch and the pleated
    recipe at 64 x 64 (brute force, so a full 256 x 256 pass would take
    minutes)."""
    import oracle as O
    from paper_2510_10256_gb300 import scenes as S
    prev = O.set_num_threads(1)
    try:
        out = {}
        for key, sc, what in (("woven", S.woven_patch(), "one oracle pass on the full woven patch, 1 core"),
                              ("pleated", S.pleated_sheet(nx=64), "one oracle pass on the pleated recipe at 64x64, 1 core")):
            out[key] = _oracle_sample([sc], what)
        return out
    finally:
        O.set_num_threads(prev)


def measure_single(args, name, steps, local, dist, nx=None, mollifier=False, clocks=True) -> dict:
    """One scene of the named workload: autotuned broad-phase knobs, W warm-up
    passes, then `steps` passes timed on the device (L2 flushed before each),
    the per-stage times of each pass, and an end-to-end leg through the C ABI
    with host buffers (copies inside the timed region)."""
    import torch
    from paper_2510_10256_gb300 import contact as CT
    sc, desc = _workload(name, reduced_nx=nx)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    cs = CT.ContactScene.from_scene(sc, mollifier=mollifier)
    x = torch.from_numpy(sc.x).to(dev)
    p = torch.from_numpy(sc.p).to(dev)
    energy = torch.zeros(1, dtype=torch.float64, device=dev)
    grad = torch.zeros(3, sc.n, dtype=torch.float64, device=dev)
    alpha = torch.zeros(1, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    tuning = _autotune(args, cs, [sc], lambda: cs.run_pass(x, p, energy, grad, alpha))
    cs.set_timing(True)
    for _ in range(args.warmup):
        cs.run_pass(x, p, energy, grad, alpha)
    torch.cuda.synchronize()
    st = cs.stats()
    # ---- device-resident timed region
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    stage = []
    clk_s = ClockSampler(local) if clocks else None
    if clk_s:
        clk_s.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = CT.kernel_launches()
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        cs.run_pass(x, p, energy, grad, alpha)
        ev[k][1].record(stream)
        stage.append(cs.stage_ms())
    torch.cuda.synchronize()
    launches = CT.kernel_launches() - l0
    if dist:
        dist.barrier()
    clk = clk_s.stop() if clk_s else None
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = max_over_ranks([statistics.median(step_ms)], dist, dev)[0]
    status = cs.sync_status()
    # ---- end to end through the C ABI with host buffers (copies timed)
    hx = torch.from_numpy(sc.x).pin_memory()
    hp = torch.from_numpy(sc.p).pin_memory()
    he = torch.zeros(1, dtype=torch.float64).pin_memory()
    ha = torch.zeros(1, dtype=torch.float64).pin_memory()
    hg = torch.zeros(3, sc.n, dtype=torch.float64).pin_memory()
    e2e_steps = max(3, steps // 2)
    torch.cuda.synchronize()
    e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(e2e_steps)]
    for k in range(e2e_steps):
        flush.zero_()
        e_ev[k][0].record(stream)
        x.copy_(hx, non_blocking=True)
        p.copy_(hp, non_blocking=True)
        cs.run_pass(x, p, energy, grad, alpha)
        he.copy_(energy, non_blocking=True)
        ha.copy_(alpha, non_blocking=True)
        hg.copy_(grad, non_blocking=True)
        e_ev[k][1].record(stream)
        stream.synchronize()
    e2e_ms = max_over_ranks([statistics.median(a.elapsed_time(b) for a, b in e_ev)], dist, dev)[0]
    cs.close()
    return {"sc": sc, "desc": desc, "st": st, "step_ms": step_ms, "ms": ms, "stage": stage, "e2e_ms": e2e_ms,
            "launches": launches, "tuning": tuning, "clocks": clk, "status": status, "steps": steps,
            "h2d": 2 * 3 * sc.n * 8, "d2h": 8 + 8 + 3 * sc.n * 8}


def _stage_dict(med) -> dict:
    return {"contact_build": med[0], "contact_filter": med[1], "barrier_eval": med[2], "ccd_step": med[3],
            "hessian_kernel": med[4], "distances_c": med[5], "assembly_d": med[6]}


def _single_summary(r, world) -> dict:
    st = r["st"]
    med = [statistics.median(s[i] for s in r["stage"]) for i in range(7)]
    return {"workload": r["desc"], "value": world * st["n_candidates"] / (r["ms"] / 1000.0), "unit": UNIT,
            "ms_per_step": r["ms"], "ms_mean": statistics.mean(r["step_ms"]), "steps": r["steps"],
            "candidates": int(st["n_candidates"]), "filtered": st["n_filtered"], "active": int(st["n_active"]),
            "ccd_pairs": st["n_ccd"], "nnzb": st["nnzb"], "stage_ms": _stage_dict(med),
            "stage_roofline": stage_roofline(st, med, [r["sc"]]),
            "e2e": {"value": world * st["n_candidates"] / (r["e2e_ms"] / 1000.0), "unit": UNIT,
                    "ms_per_step": r["e2e_ms"], "h2d_bytes_per_step": r["h2d"], "d2h_bytes_per_step": r["d2h"]},
            "tuning": r["tuning"], "gpu_launches": int(r["launches"]), "status": r["status"]}


def _single_line(args, r, world) -> dict:
    """The JSON line of a single-scene workload, with the roofline of the
    dominant (FP64 stage-d) kernels."""
    from paper_2510_10256_gb300 import contact as CT
    st, sc = r["st"], r["sc"]
    n_cand = st["n_candidates"]
    med = [statistics.median(s[i] for s in r["stage"]) for i in range(7)]
    hess_ms = statistics.mean(s[4] for s in r["stage"])
    na = st["n_active"]
    achieved = hess_flops(st) / (hess_ms / 1000.0) / 1e12 if hess_ms > 0 else 0.0
    try:
        fp64_meas = CT.measure_fma_tflops(True)
        fp32_meas = CT.measure_fma_tflops(False, iters=65536)
    except Exception:
        fp64_meas = fp32_meas = None
    roofline = {"bound": "alu", "kernel": "k_hess_prep + k_hess_proj<9> + k_hess_proj_pe (FP64 stage d)",
                "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "peak_fp64_fma_measured": fp64_meas, "peak_fp32_fma_measured": fp32_meas,
                "traffic": HESS_DRAM_BYTES_PER_ACTIVE * na if HESS_DRAM_BYTES_PER_ACTIVE else None,
                "traffic_source": HESS_TRAFFIC_SOURCE,
                "flops_per_pass": hess_flops(st), "active_pairs": na,
                "pairs_per_kernel": {"face": st["n_hess_face"], "pe_frame": st["n_hess_pe_frame"],
                                     "pe": st["n_hess_pe"]},
                "kernel_ms": hess_ms, "peak_source": "derived: 152 SM x 2070 MHz x 4 FP64 flop/clk/SM"}
    return {"metric": METRIC, "value": world * n_cand / (r["ms"] / 1000.0), "unit": UNIT, "n_gpus": world,
            "steps": r["steps"], "warmup": args.warmup, "ms_per_step": r["ms"],
            "ms_mean": statistics.mean(r["step_ms"]), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": r["desc"], "candidates": int(n_cand), "filtered": st["n_filtered"],
                       "core": st["n_core"], "active": int(na), "ccd_pairs": st["n_ccd"], "nnzb": st["nnzb"],
                       "dbar_min": st["dbar_min"], "seed": sc.seed, "tuning": r["tuning"],
                       "mollifier": bool(args.mollifier), "mollified_pairs": st["n_mollified"],
                       "l2": "flushed (256 MiB write) between steps", "timing": "median of the timed passes",
                       "parallelism": f"replicas x{world}"},
            "stage_ms": _stage_dict(med),
            "roofline": roofline,
            "stage_roofline": stage_roofline(st, med, [sc]),
            "fp32_broad_phase": {"candidates_fp32": st["n_candidates_fp32"], "candidates": int(n_cand),
                                 "superset_ratio": st["n_candidates_fp32"] / max(1, n_cand),
                                 "fp64_decided": st["n_fp64_decided"]},
            "e2e": {"value": world * n_cand / (r["e2e_ms"] / 1000.0), "unit": UNIT,
                    "h2d_bytes_per_step": r["h2d"], "d2h_bytes_per_step": r["d2h"], "ms_per_step": r["e2e_ms"]},
            "clocks": r["clocks"], "gpu_launches": int(r["launches"]), "status": r["status"]}


if __name__ == "__main__":
    main()
