"""Host logic of the Newton driver (newton.py) on a fake scene, no GPU: with
no contact and a quadratic stand-in for the friction potential,
D(x) = k/2 |x - x_lag|^2, Phi = |x - x_t|^2 / (2 h^2) + D has the closed-form
minimiser (x_t / h^2 + k x_0) / (1 / h^2 + k), which one Newton step must
reach only if the driver lags at x_0 once and feeds D's energy, gradient and
Hessian products into every part of the step."""
import numpy as np
import torch

from paper_2510_10256_gb300.newton import minimize


class FakeScene:
    count = 1

    def __init__(self, k=0.0):
        self.k = k
        self.lags = []
        self.spmv_calls = 0

    def contact_build(self, x):
        pass

    def contact_filter(self):
        pass

    def barrier_eval(self, x, energy, grad):
        energy.zero_()
        grad.zero_()

    def barrier_energy(self, x, energy):
        energy.zero_()

    def bsr_spmv(self, v, y, shift=0.0):
        y.copy_(shift * v)

    def ccd_step(self, x, p, alpha):
        alpha.fill_(1.0)

    def stats(self):
        return {"n_active": 0}

    def friction_lag(self, x_lag, mu, eps):
        self.lags.append(x_lag.clone())

    def friction_eval(self, x, x_lag, energy, grad=None):
        dx = x - x_lag
        energy[0] += 0.5 * self.k * float(torch.sum(dx * dx))
        if grad is not None:
            grad.add_(self.k * dx)

    def friction_spmv(self, v, y):
        self.spmv_calls += 1
        y.add_(self.k * v)


def _case(seed=0):
    rng = np.random.default_rng(seed)
    x0 = torch.from_numpy(rng.normal(size=(3, 20)))
    xt = x0 + torch.from_numpy(rng.normal(size=(3, 20)))
    return x0, xt


def test_newton_with_friction_reaches_the_closed_form_minimiser():
    x0, xt = _case()
    h, k = 0.1, 250.0
    cs = FakeScene(k)
    x, hist = minimize(cs, x0, xt, h, tol=1e-12, max_iters=5, friction=(0.5, 1e-3))
    want = (xt / h ** 2 + k * x0) / (1.0 / h ** 2 + k)
    assert torch.max(torch.abs(x - want)) < 1e-10
    assert len(cs.lags) == 1 and torch.equal(cs.lags[0], x0)
    assert cs.spmv_calls > 0
    assert hist[0].alpha == 1.0 and hist[-1].grad_norm <= 1e-12 * hist[0].grad_norm


def test_newton_without_friction_never_touches_it():
    x0, xt = _case(1)
    cs = FakeScene(k=1e9)  # would dominate if it were used
    x, hist = minimize(cs, x0, xt, 0.1, tol=1e-12, max_iters=5)
    assert torch.max(torch.abs(x - xt)) < 1e-10
    assert not cs.lags and cs.spmv_calls == 0
