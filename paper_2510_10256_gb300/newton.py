"""Contact-only Newton driver: the consumer of the pass's gradient, Hessian,
step bound and energy (the paper minimises each implicit step with projected
Newton, App. A; its line search starts from the CCD bound, Sec. 3.3).

It minimises  Phi(x) = |x - x_target|^2 / (2 h^2) + E(x)  (a unit lumped
mass and time step h: the inertia term of an implicit step with no elastic
energy) from a penetration-free x.  Each iteration:

  1. contact_build, contact_filter, barrier_eval at x: E, g = grad E, H (BSR,
     PSD-projected per pair);
  2. the Newton direction D solves (I / h^2 + H) D = -grad Phi by conjugate
     gradients (H is PSD, so the system is SPD), with products from
     cb_bsr_spmv;
  3. alpha_max = ccd_step(x, D) (<= 1, conservative: no pair reaches its
     offset along [x, x + alpha_max D]);
  4. Armijo backtracking from alpha_max with energy-only passes
     (contact_build, contact_filter, barrier_energy at each trial point).

With friction=(mu, eps), Phi gains the lagged friction potential D(x) of
the active pairs at x0 (friction_lag after the first barrier_eval; App. A:
the paper's solver uses IPC's friction with the contact barrier): its
energy and gradient come from friction_eval and its Hessian products from
friction_spmv, added to the barrier's in every step above.

Vector algebra of the solve (dot products, axpys) runs as torch operations on
the device; every contact quantity comes from the library.  Stops when
|grad Phi| <= tol |grad Phi_0| or after max_iters.
"""
from __future__ import annotations

import dataclasses

import torch


@dataclasses.dataclass
class NewtonIter:
    phi: float
    grad_norm: float
    alpha_max: float
    alpha: float
    cg_iters: int
    line_search_trials: int
    active: int


def _phi(cs, x, x_target, h2, energy, build=True, x_lag=None):
    if build:
        cs.contact_build(x)
        cs.contact_filter()
    cs.barrier_energy(x, energy)
    if x_lag is not None:
        cs.friction_eval(x, x_lag, energy)
    e = float(energy.sum().item())
    return 0.5 * float(torch.sum((x - x_target) ** 2).item()) / h2 + e


def cg(cs, rhs, shift, tol=1e-10, max_iters=500, friction=False):
    """Solve (H + shift I) d = rhs (H: the scene's BSR of the last
    barrier_eval, plus the friction Hessian of the last friction_eval when
    friction is set) by conjugate gradients with a Jacobi-free start d = 0."""
    d = torch.zeros_like(rhs)
    r = rhs.clone()
    p = r.clone()
    Ap = torch.empty_like(rhs)
    rr = torch.sum(r * r)
    stop = (tol * tol) * rr
    it = 0
    while it < max_iters and rr > stop:
        cs.bsr_spmv(p, Ap, shift)
        if friction:
            cs.friction_spmv(p, Ap)
        a = rr / torch.sum(p * Ap)
        d.add_(a * p)
        r.sub_(a * Ap)
        rr_new = torch.sum(r * r)
        p.mul_(rr_new / rr).add_(r)
        rr = rr_new
        it += 1
    return d, it


def minimize(cs, x0, x_target, h: float, tol: float = 1e-8, max_iters: int = 30, armijo: float = 1e-4,
             friction: tuple[float, float] | None = None):
    """Newton iterations from x0 (device [3][n] FP64); returns (x, history).
    friction = (mu, eps): lagged friction of the active pairs at x0."""
    dev = x0.device
    x = x0.clone()
    h2 = h * h
    shift = 1.0 / h2
    M = cs.count if hasattr(cs, "count") else 1
    energy = torch.zeros(M, dtype=torch.float64, device=dev)
    alpha_t = torch.zeros(M, dtype=torch.float64, device=dev)
    grad = torch.zeros_like(x)
    hist: list[NewtonIter] = []
    g0 = None
    x_lag = x0.clone() if friction is not None else None
    for it in range(max_iters):
        cs.contact_build(x)
        cs.contact_filter()
        cs.barrier_eval(x, energy, grad)
        if friction is not None:
            if it == 0:
                cs.friction_lag(x_lag, friction[0], friction[1])
            cs.friction_eval(x, x_lag, energy, grad)
        gphi = (x - x_target) / h2 + grad
        gn = float(torch.linalg.vector_norm(gphi).item())
        phi = 0.5 * float(torch.sum((x - x_target) ** 2).item()) / h2 + float(energy.sum().item())
        if g0 is None:
            g0 = gn
        if gn <= tol * g0:
            hist.append(NewtonIter(phi, gn, 0.0, 0.0, 0, 0, int(cs.stats()["n_active"])))
            break
        active = int(cs.stats()["n_active"])
        D, k = cg(cs, -gphi, shift, friction=friction is not None)
        slope = float(torch.sum(gphi * D).item())
        cs.ccd_step(x, D, alpha_t)
        a_max = float(alpha_t.min().item())
        a = a_max
        trials = 0
        while True:
            trials += 1
            phi_t = _phi(cs, x + a * D, x_target, h2, energy, x_lag=x_lag)
            if phi_t <= phi + armijo * a * slope or trials >= 40:
                break
            a *= 0.5
        x = x + a * D
        hist.append(NewtonIter(phi, gn, a_max, a, k, trials, active))
    return x, hist
