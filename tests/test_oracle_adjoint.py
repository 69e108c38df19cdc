"""Pins of the oracle's adjoint (gradients of a plane loss with respect to eps_r and sigma).

The oracle obtains the transpose of a step by probing its own forward collision. These tests check
that against the forward step alone. The dot-product identity <lambda, G v> = <G^T lambda, v> must
hold for the step's linear part G. Central differences of the forward step, and of the whole loss,
must match the parameter gradients. Double precision throughout; no GPU.
"""
import numpy as np
import pytest

from helpers import oracle_from_workload
from oracle import OracleLattice, TimeFn
from paper_2309_08068_gb300 import workloads as wl

MODELS = ("mm", "hv")


def lattice(model, seed, shape=(5, 4, 3), sources=True):
    w, f = wl.random_state(model, shape, seed=seed, media="random", n_sources=2 if sources else 0)
    L = oracle_from_workload(w, init=False, threads=4)
    L.set_populations(f, 6)
    return w, L, f


@pytest.mark.parametrize("model", MODELS)
def test_adjoint_step_is_the_transpose(model):
    """<lambda, step(f + v) - step(f)> = <adjoint(lambda), v> for random f, v, lambda, with random
    media, a current source and an imposed source (the affine parts cancel in the difference)."""
    w, L, f = lattice(model, 71)
    rng = np.random.default_rng(72)
    v = rng.standard_normal(f.shape)
    lam = rng.standard_normal(f.shape)
    L.set_populations(f + v, 6)
    L.step(1)
    a = L.populations()
    L.set_populations(f, 6)
    L.step(1)
    b = L.populations()
    lhs = float(np.sum(lam * (a - b)))
    rhs = float(np.sum(L.adjoint_step(7, lam, f) * v))
    assert abs(lhs - rhs) <= 1e-11 * max(1.0, abs(lhs))


@pytest.mark.parametrize("model", MODELS)
def test_adjoint_step_parameter_gradient_matches_finite_differences(model):
    """d/d eps_r(c) and d/d sigma(c) of <lambda, step(f)> against central differences of the forward
    step, at a source cell, an imposed cell and an ordinary cell."""
    w, L, f = lattice(model, 73)
    rng = np.random.default_rng(74)
    lam = rng.standard_normal(f.shape)
    ge = np.zeros(w.n)
    gs = np.zeros(w.n)
    L.adjoint_step(7, lam, f, ge, gs)
    cells = [int(w.sources[0].cells[0]), int(w.sources[1].cells[0]), 11]
    for which, grad in (("eps_r", ge), ("sigma", gs)):
        for c in cells:
            vals = []
            for sgn in (+1, -1):
                w2 = wl.Workload(w.name, w.model, w.shape, 0, eps_r=w.eps_r.copy(), mu_r=w.mu_r, sigma=w.sigma.copy(),
                                 sources=w.sources)
                arr = w2.eps_r if which == "eps_r" else w2.sigma
                h = 1e-5 * max(abs(arr[c]), 1e-2)
                arr[c] += sgn * h
                L2 = oracle_from_workload(w2, init=False)
                L2.set_populations(f, 6)
                L2.step(1)
                vals.append(float(np.sum(lam * L2.populations())))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - grad[c]) <= 1e-6 * max(1.0, abs(fd)), (which, c, fd, grad[c])


@pytest.mark.parametrize("model", MODELS)
def test_loss_gradient_matches_finite_differences(model):
    """L = sum_{t=1..T} sum_{plane x = 2} |E(t)|^2 over T = 12 steps of a 6 x 5 x 4 lattice with
    per-cell eps_r and sigma and a dipole-like current: the adjoint gradient against central
    differences of L at several cells. The gradient is taken at fixed starting populations (the
    finite differences restart from the same f^0, not from a re-initialisation that would itself
    depend on eps_r)."""
    rng = np.random.default_rng(75)
    shape = (6, 5, 4)
    n = 120
    eps = rng.uniform(1.0, 3.0, n)
    sig = rng.uniform(0.0, 0.3, n)
    w = wl.Workload("adj", model, shape, 0, eps_r=eps, sigma=sig)
    cells = np.array([3 + 6 * (2 + 5 * 1), 4 + 6 * (2 + 5 * 2)])
    w.sources = [wl.Source("current", cells, wl.TimeFunction("sin", 1.0, 7.0, 0.3),
                           w=rng.standard_normal((2, 3)))]
    f0 = rng.standard_normal((wl.POPULATIONS[model], n)) * 0.1

    def run(eps_r, sigma, grad=False):
        w2 = wl.Workload("adj", model, shape, 0, eps_r=eps_r, sigma=sigma, sources=w.sources)
        L = oracle_from_workload(w2, init=False)
        L.set_populations(f0, 0)
        if grad:
            return L.loss_and_gradient(12, 0, 2)
        loss = 0.0
        for t in range(1, 13):
            L.step(1)
            loss += L.plane_loss(t, L.populations(), 0, 2)
        return loss

    loss, ge, gs = run(eps, sig, grad=True)
    assert abs(loss - run(eps, sig)) <= 1e-12 * loss
    for c in (2, 17, 40, 77, 101):
        for arr, grad in ((eps, ge), (sig, gs)):
            h = 1e-5 * max(arr[c], 1e-2)
            up, dn = arr.copy(), arr.copy()
            up[c] += h
            dn[c] -= h
            fd = (run(up, sig) - run(dn, sig)) / (2 * h) if arr is eps else (run(eps, up) - run(eps, dn)) / (2 * h)
            assert abs(fd - grad[c]) <= 1e-5 * max(abs(fd), 1e-3 * loss), (c, fd, grad[c])
