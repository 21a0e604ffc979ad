"""Served request stream: continuous batching of contact passes on one GPU.

A request is a scene plus a sequence of contact steps.  Each step runs one
contact pass (stages a-e) at the request's current positions x with a fresh
seeded search direction p, then moves x <- x + alpha p by the pass's step
bound alpha.

Scheduling is iteration-level ("continuous batching"):
  * arrivals join a FIFO queue;
  * at every iteration boundary, queued requests are admitted while a slot is
    free and their estimated device footprint fits the HBM budget; a loader
    thread creates their scenes on the device (upload, filter tables) on its
    own stream, overlapping the running iteration;
  * one iteration advances every resident request by one step: the resident
    scenes of each kind form one batch (one launch per stage for all of them,
    rebuilt only when membership changes), and the rod and shell batches run
    on two streams at once;
  * finished requests leave, freeing their slot and budget.

Per-step latency runs from the step becoming runnable (the previous step's
result, or the scene being ready) to its alpha and gradient being ready;
queueing delay (arrival to admission) and load time (admission to ready) are
reported separately.

The scheduler (Server) only talks to an engine: footprint(req) -> bytes,
create(req) -> handle, run_step(kind, handles) -> (per-handle results, pairs
of the pass), release(handle).
DeviceEngine is the GPU engine on the contact library; tests drive the same
scheduler with a host-only fake engine.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import dataclasses
import math
import statistics
import threading
import time

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float            # seconds after the stream starts
    scene: object             # scenes.Scene (host arrays; may be shared by requests)
    steps: int = 10
    seed: int = 0             # seed of the request's search directions
    sigma: float = 0.1        # std of each coordinate of p

    @property
    def kind(self) -> str:
        return self.scene.kind


@dataclasses.dataclass
class StepResult:
    energy: float
    alpha: float


@dataclasses.dataclass
class _Slot:
    req: Request
    handle: object
    reserved: int
    admitted: float
    ready: float
    runnable: float
    step: int = 0


def poisson_requests(pool: list, n: int, rate: float, steps: int, seed: int) -> list[Request]:
    """n requests with exponential inter-arrival times (mean 1/rate), the first
    at t = 0; each draws rod or shell with probability 1/2 and then a scene of
    that kind from the pool uniformly."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, n)
    t = np.concatenate([[0.0], np.cumsum(gaps[1:])])
    by_kind = {"rod": [s for s in pool if s.kind == "rod"], "shell": [s for s in pool if s.kind == "shell"]}
    out = []
    for i in range(n):
        kind = "rod" if rng.random() < 0.5 else "shell"
        cands = by_kind[kind] or by_kind["shell" if kind == "rod" else "rod"]
        sc = cands[int(rng.integers(len(cands)))]
        sigma = float(sc.meta.get("sigma", 0.0)) if sc.meta else 0.0
        if not sigma > 0.0:
            sigma = float(np.std(sc.p)) if sc.p.size else 0.0
        out.append(Request(rid=i, arrival=float(t[i]), scene=sc, steps=steps, seed=seed * 1000 + i, sigma=sigma))
    return out


def _pct(v, q):
    if not v:
        return None
    s = sorted(v)
    k = min(len(s) - 1, max(0, int(math.ceil(q / 100.0 * len(s))) - 1))
    return s[k]


class Server:
    """Iteration-level scheduler over an engine (see the module docstring)."""

    def __init__(self, engine, hbm_budget: int, max_slots: int = 16, keep_results: bool = False,
                 clock=time.perf_counter, sleep=time.sleep):
        self.engine = engine
        self.budget = int(hbm_budget)
        self.max_slots = int(max_slots)
        self.keep = keep_results
        self.clock = clock
        self.sleep = sleep

    def run(self, requests: list[Request]) -> dict:
        eng = self.engine
        clock = self.clock
        pending = collections.deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
        waiting: collections.deque = collections.deque()
        loading: dict = {}                      # future -> (request, reserved bytes, admission time)
        resident = {"rod": [], "shell": []}     # kind -> slots
        inflight: dict = {}                     # kind -> (future, slots of the running iteration)
        used = peak_used = peak_real = 0
        live_bytes = getattr(eng, "live_bytes", None)
        lat, queue, load = [], [], []
        results = collections.defaultdict(list) if self.keep else None
        rejected = []
        steps_done = pairs = iters = max_resident = 0
        loader = cf.ThreadPoolExecutor(max_workers=1)
        workers = cf.ThreadPoolExecutor(max_workers=2)
        t0 = clock()

        def timed(kind, handles):
            res, npairs = eng.run_step(kind, handles)
            return res, npairs, clock() - t0

        try:
            while pending or waiting or loading or inflight or resident["rod"] or resident["shell"]:
                now = clock() - t0
                while pending and pending[0].arrival <= now:
                    waiting.append(pending.popleft())
                # admission: FIFO while a slot is free and the footprint fits the budget.
                # What is charged is the larger of the footprint estimates of everything
                # admitted and, where the engine can tell, the device memory it really
                # holds now (plus the estimates of the scenes still loading).
                n_res = len(resident["rod"]) + len(resident["shell"])
                charged = used
                if live_bytes is not None:
                    real = int(live_bytes()) + sum(v[1] for v in loading.values())
                    peak_real = max(peak_real, real)
                    charged = max(used, real)
                while waiting and n_res + len(loading) < self.max_slots:
                    req = waiting[0]
                    need = int(eng.footprint(req))
                    if need > self.budget:
                        rejected.append(waiting.popleft().rid)
                        continue
                    if charged + need > self.budget:
                        break
                    charged += need
                    waiting.popleft()
                    used += need
                    peak_used = max(peak_used, used)
                    loading[loader.submit(eng.create, req)] = (req, need, clock() - t0)
                # loaded scenes become resident (runnable from now)
                for fut in [f for f in loading if f.done()]:
                    req, need, adm = loading.pop(fut)
                    h = fut.result()
                    ready = clock() - t0
                    queue.append(adm - req.arrival)
                    load.append(ready - adm)
                    resident[req.kind].append(_Slot(req, h, need, adm, ready, ready))
                # finished iterations: record, advance, retire
                for kind in [k for k, (f, _) in inflight.items() if f.done()]:
                    fut, group = inflight.pop(kind)
                    res, npairs, done_t = fut.result()
                    iters += 1
                    pairs += int(npairs)
                    for sl, r in zip(group, res):
                        lat.append(done_t - sl.runnable)
                        sl.runnable = done_t
                        sl.step += 1
                        steps_done += 1
                        if self.keep:
                            results[sl.req.rid].append(r)
                    keep = []
                    for sl in resident[kind]:
                        if sl.step >= sl.req.steps:
                            eng.release(sl.handle)
                            used -= sl.reserved
                        else:
                            keep.append(sl)
                    resident[kind] = keep
                max_resident = max(max_resident, len(resident["rod"]) + len(resident["shell"]))
                # idle kinds start their next iteration over every resident request
                for kind in ("rod", "shell"):
                    if kind not in inflight and resident[kind]:
                        group = list(resident[kind])
                        inflight[kind] = (workers.submit(timed, kind, [sl.handle for sl in group]), group)
                # wait for an iteration, a load or the next arrival
                futs = [f for f, _ in inflight.values()] + list(loading)
                timeout = 0.05
                if pending:
                    timeout = max(0.0, min(timeout, pending[0].arrival - (clock() - t0)))
                if futs:
                    cf.wait(futs, timeout=timeout, return_when=cf.FIRST_COMPLETED)
                elif pending or waiting:
                    self.sleep(timeout if pending else 0.001)
        finally:
            loader.shutdown(wait=True)
            workers.shutdown(wait=True)
        wall = clock() - t0
        rep = {"wall_s": wall, "steps": steps_done, "pairs": pairs, "iterations": iters,
               "pairs_per_s": pairs / wall if wall > 0 else 0.0, "steps_per_s": steps_done / wall if wall > 0 else 0.0,
               "requests": len(requests) - len(rejected), "rejected": rejected,
               "step_latency_ms": {"p50": _ms(_pct(lat, 50)), "p99": _ms(_pct(lat, 99)),
                                   "mean": _ms(statistics.mean(lat)) if lat else None},
               "queue_delay_ms": {"p50": _ms(_pct(queue, 50)), "p99": _ms(_pct(queue, 99))},
               "load_ms": {"p50": _ms(_pct(load, 50)), "p99": _ms(_pct(load, 99))},
               "peak_reserved_bytes": peak_used, "peak_live_bytes": peak_real if live_bytes is not None else None,
               "max_resident": max_resident}
        if self.keep:
            rep["results"] = dict(results)
        return rep


def _ms(v):
    return None if v is None else 1000.0 * v


class DeviceEngine:
    """The GPU engine: scenes of the contact library, one batch per kind.

    Every device buffer of its scenes and batches comes from PyTorch's caching
    allocator, so live_bytes() -- torch's allocated bytes on the device since
    the engine started -- is what the resident requests really hold; the
    scheduler charges the budget from it.  Footprint model (the estimate a
    request is admitted on, before it holds anything): device bytes per
    vertex of each kind, measured by calibrate() on sample scenes (scene +
    batch copy + pass buffers), times a safety factor."""

    def __init__(self, device=None, mode: str = "double", safety: float = 1.25):
        import torch
        from . import contact as CT
        self.torch = torch
        self.CT = CT
        self.dev = torch.device(device or "cuda")
        self.mode = mode
        self.safety = safety
        self.streams = {"rod": torch.cuda.Stream(self.dev), "shell": torch.cuda.Stream(self.dev),
                        "load": torch.cuda.Stream(self.dev)}
        self.batches = {}
        self.bytes_per_vertex = {"rod": 4096.0, "shell": 16384.0}
        self.lock = threading.Lock()
        torch.cuda.synchronize(self.dev)
        self.base_bytes = torch.cuda.memory_allocated(self.dev)

    def live_bytes(self) -> int:
        """Device memory allocated since the engine started: the scenes,
        batches and step tensors of the resident requests."""
        return max(0, self.torch.cuda.memory_allocated(self.dev) - self.base_bytes)

    # -- footprint
    def calibrate(self, scenes: list):
        """Device bytes per vertex of each kind: the largest ratio over the
        sample scenes of (scene after one pass alone) x 2.  A batched member
        holds its static data twice (its own scene and the batch copy) and the
        pass buffers once, so twice the alone figure bounds it."""
        best = {}
        for sc in scenes:
            h = self.create(Request(-1, 0.0, sc, 1, 0, float(np.std(sc.p))))
            self.run_step(sc.kind, [h])
            per = 2.0 * h.cs.stats()["device_bytes"] / max(1, sc.n)
            self.release(h)
            best[sc.kind] = max(best.get(sc.kind, 0.0), per)
        self.bytes_per_vertex.update(best)
        return dict(self.bytes_per_vertex)

    def footprint(self, req: Request) -> int:
        return int(self.safety * self.bytes_per_vertex[req.kind] * req.scene.n)

    # -- lifecycle
    def create(self, req: Request):
        torch = self.torch
        st = self.streams["load"]
        with torch.cuda.stream(st):
            cs = self.CT.ContactScene.from_scene(req.scene, mode=self.mode, stream=st)
            x = torch.from_numpy(np.ascontiguousarray(req.scene.x)).to(self.dev, non_blocking=False)
            gen = torch.Generator(device=self.dev)
            gen.manual_seed(int(req.seed))
        st.synchronize()
        return _Handle(cs, x, gen, req.sigma, req.scene.n)

    def release(self, h):
        for k in list(self.batches):
            if any(m is h for m in self.batches[k][0]):
                self._drop_batch(k)
        h.cs.close()

    def _drop_batch(self, kind):
        old = self.batches.pop(kind, None)
        if old is not None and old[1] is not None:
            self.streams[kind].synchronize()
            old[1].close()

    # -- one step of every handle of one kind
    def run_step(self, kind: str, handles: list):
        torch = self.torch
        st = self.streams[kind]
        with torch.cuda.stream(st):
            cur = self.batches.get(kind)
            if cur is None or len(cur[0]) != len(handles) or any(a is not b for a, b in zip(cur[0], handles)):
                self._drop_batch(kind)
                b = self.CT.ContactBatch([h.cs for h in handles], stream=st) if len(handles) > 1 else None
                self.batches[kind] = (list(handles), b)
            runner = self.batches[kind][1] or handles[0].cs
            M = len(handles)
            x = torch.cat([h.x for h in handles], dim=1) if M > 1 else handles[0].x.contiguous()
            p = torch.cat([torch.randn(3, h.n, generator=h.gen, device=self.dev, dtype=torch.float64) * h.sigma
                           for h in handles], dim=1)
            energy = torch.zeros(M, dtype=torch.float64, device=self.dev)
            grad = torch.zeros(3, x.shape[1], dtype=torch.float64, device=self.dev)
            alpha = torch.zeros(M, dtype=torch.float64, device=self.dev)
            runner.run_pass(x, p, energy, grad, alpha, stream=st)
            sizes = torch.tensor([h.n for h in handles], device=self.dev)
            xn = x + torch.repeat_interleave(alpha, sizes)[None, :] * p
            off = 0
            for h in handles:
                h.x = xn[:, off:off + h.n]
                off += h.n
            e_h, a_h = energy.cpu().numpy(), alpha.cpu().numpy()
            npairs = int(runner.stats()["n_candidates"])
        return [StepResult(float(e_h[i]), float(a_h[i])) for i in range(M)], npairs

    def close(self):
        for k in list(self.batches):
            self._drop_batch(k)


@dataclasses.dataclass
class _Handle:
    cs: object
    x: object
    gen: object
    sigma: float
    n: int


def run_plain(engine, requests: list[Request], clock=time.perf_counter, sleep=time.sleep) -> dict:
    """The plain form of a request stream, for comparison with Server: the
    same requests in arrival order (FIFO), one at a time, each step a plain
    single-scene pass; nothing overlaps.  Reports like Server.run (step
    latency from the step becoming runnable to its result, queueing delay
    from arrival to the start of the request's scene creation)."""
    lat, queue, load = [], [], []
    steps_done = pairs = 0
    t0 = clock()
    for req in sorted(requests, key=lambda r: (r.arrival, r.rid)):
        now = clock() - t0
        if req.arrival > now:
            sleep(req.arrival - now)
        adm = clock() - t0
        queue.append(adm - req.arrival)
        h = engine.create(req)
        ready = clock() - t0
        load.append(ready - adm)
        runnable = ready
        for _ in range(req.steps):
            _, npairs = engine.run_step(req.kind, [h])
            done = clock() - t0
            lat.append(done - runnable)
            runnable = done
            steps_done += 1
            pairs += int(npairs)
        engine.release(h)
    wall = clock() - t0
    return {"wall_s": wall, "steps": steps_done, "pairs": pairs, "iterations": steps_done,
            "pairs_per_s": pairs / wall if wall > 0 else 0.0, "steps_per_s": steps_done / wall if wall > 0 else 0.0,
            "requests": len(requests), "rejected": [],
            "step_latency_ms": {"p50": _ms(_pct(lat, 50)), "p99": _ms(_pct(lat, 99)),
                                "mean": _ms(statistics.mean(lat)) if lat else None},
            "queue_delay_ms": {"p50": _ms(_pct(queue, 50)), "p99": _ms(_pct(queue, 99))},
            "load_ms": {"p50": _ms(_pct(load, 50)), "p99": _ms(_pct(load, 99))},
            "peak_reserved_bytes": 0, "max_resident": 1}


def run_alone(engine, req: Request) -> list[StepResult]:
    """The same request with nothing else on the device: its steps one after
    another, each a plain single-scene pass."""
    h = engine.create(req)
    out = [engine.run_step(req.kind, [h])[0][0] for _ in range(req.steps)]
    engine.release(h)
    return out
