"""Rest-force sweep (Fig. 3): the norm of the contact-only force at the rest
configuration, with the barrier filter (Eq. 4) and with the plain barrier
(no filter), over mesh resolution and thickness.

With the filter every stencil neighbour closer than the activation at rest is
class F, with offset 0 and width dbar_min, the smallest such rest distance, so
at rest it sits at or beyond its width and exerts nothing: the force is
exactly zero at every resolution.  Without the filter those neighbours are
active at rest (closer than the thickness they take the temporary zero offset
of class C, Sec. 3.4) and the rest force grows as the mesh is refined.

Scenes: a straight polyline of segment length L (the rod of the figure's left
panel) and a flat regular grid of edge length L (shells), where the rest
distance of every stencil pair equals its reference distance.  (A rod's
reference distance is the arc-length gap, which a curved rest shape's chord
undercuts: `turn` > 0 bends the polyline by seeded angles, and then the pairs
nearest dbar_min keep a residual force at rounding level, ~1e-31 here.)
Thicknesses are chosen off the multiples of L, so that no rest distance sits
on the offset itself, where rounding would decide the class.  Every number comes from the GPU pass (contact_build,
contact_filter, barrier_eval at x = rest).

    python -m paper_2510_10256_gb300.restforce          # prints the sweep as JSON lines
"""
from __future__ import annotations

import json

import numpy as np

from . import scenes as S


def rod_at_rest(n_seg: int, length: float = 2.0, thickness: float = 0.23, dhat: float = 0.01,
                turn: float = 0.0, seed: int = 3) -> S.Scene:
    """Planar polyline of n_seg segments (total length `length`), straight, or
    with seeded turning angles in [-turn, turn] rad; current = rest."""
    rng = np.random.default_rng(seed)
    seg = length / n_seg
    ang = np.cumsum(rng.uniform(-turn, turn, n_seg)) if turn > 0 else np.zeros(n_seg)
    pts = np.zeros((3, n_seg + 1))
    pts[0, 1:] = np.cumsum(seg * np.cos(ang))
    pts[1, 1:] = np.cumsum(seg * np.sin(ang))
    return S.Scene("rod", pts.copy(), pts.copy(), np.zeros_like(pts), thickness, dhat,
                   rod_ptr=np.array([0, n_seg + 1], np.int32), name="rod_at_rest")


def shell_at_rest(nx: int, size: float = 4.0, thickness: float = 1.0, dhat: float = 0.05) -> S.Scene:
    """Flat nx x nx grid of side `size`, current = rest."""
    return S.flat_grid(nx=nx, L=size / (nx - 1), thickness=thickness, dhat=dhat)


def rest_force(sc: S.Scene, mode: str, keep_grad: bool = False) -> dict:
    """Energy, force norm and active pairs of the contact pass at x = rest
    (keep_grad: also the gradient itself, [3][n] on the host)."""
    import torch
    from .contact import ContactScene
    dev = torch.device("cuda:0")
    cs = ContactScene.from_scene(sc, mode=mode)
    x = torch.from_numpy(np.ascontiguousarray(sc.rest)).to(dev)
    energy = torch.zeros(1, dtype=torch.float64, device=dev)
    grad = torch.zeros(3, sc.n, dtype=torch.float64, device=dev)
    cs.contact_build(x)
    cs.contact_filter()
    cs.barrier_eval(x, energy, grad)
    torch.cuda.synchronize()
    st = cs.stats()
    out = {"energy": float(energy.item()), "force_norm": float(torch.linalg.vector_norm(grad).item()),
           "force_max": float(grad.abs().max().item()), "active": int(st["n_active"]),
           "filtered": int(st["n_filtered"]), "candidates": int(st["n_candidates"])}
    if keep_grad:
        out["grad"] = grad.cpu().numpy()
    cs.close()
    return out


def sweep(rod_segments=(20, 40, 80, 160), rod_thickness=(0.13, 0.23), shell_nx=(9, 17, 33, 65),
          shell_thickness=(0.55, 1.05)) -> list[dict]:
    rows = []
    for th in rod_thickness:
        for ns in rod_segments:
            sc = rod_at_rest(ns, thickness=th)
            for mode in ("double", "off"):
                rows.append({"kind": "rod", "segments": ns, "L": 2.0 / ns, "thickness": th, "mode": mode,
                             **rest_force(sc, mode)})
    for th in shell_thickness:
        for nx in shell_nx:
            sc = shell_at_rest(nx, thickness=th)
            for mode in ("double", "off"):
                rows.append({"kind": "shell", "nx": nx, "L": 4.0 / (nx - 1), "thickness": th, "mode": mode,
                             **rest_force(sc, mode)})
    return rows


if __name__ == "__main__":
    from . import contact
    contact.build()
    for r in sweep():
        print(json.dumps(r))
