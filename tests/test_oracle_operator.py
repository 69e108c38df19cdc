"""The stepping oracle (oracle/lbm_oracle.c) against the brute-force operator (oracle/operator.py).
No GPU.

The two share no code: the C oracle loops over cells and populations in the order of the Appendix B
loop body, while operator.py rebuilds the vector sets from the trigonometric formulas and writes each
cell's collision as a small matrix, then assembles the global affine map. Agreement to rounding on
small lattices with random media, currents and imposed fields pins every term of the step in both:
a dropped term, a wrong coefficient, sign or index, or a transposed advection in either one shows
up here as an O(1) difference.
"""
import numpy as np
import pytest

from helpers import oracle_from_workload
from oracle import OracleLattice
from oracle import operator as O2
from paper_2309_08068_gb300 import workloads as wl


def _run_both(model, shape, w, f, steps):
    L = oracle_from_workload(w, init=False)
    L.set_populations(f, 0)
    x = f.reshape(-1).copy()
    worst = 0.0
    for t in range(1, steps + 1):
        G, b = O2.step_operator(model, shape, t, w.eps_r, w.mu_r, w.sigma, w.sources)
        x = G @ x + b
        L.step(1)
        ref = L.populations().reshape(-1)
        worst = max(worst, float(np.linalg.norm(x - ref) / np.linalg.norm(ref)))
    return worst


@pytest.mark.parametrize("model", ["mm", "hv"])
@pytest.mark.parametrize("shape", [(3, 3, 3), (1, 1, 16), (4, 3, 2)])
def test_oracle_equals_brute_force_operator(model, shape):
    """50 steps from random populations with per-cell random eps_r, mu_r, sigma (half the cells
    conducting), a sinusoidal current and an imposed source (Section II/III step, Appendix B)."""
    w, f = wl.random_state(model, shape, seed=11, media="random", n_sources=2)
    assert {s.kind for s in w.sources} == {"current", "impose"}
    assert _run_both(model, shape, w, f, 50) < 1e-13


@pytest.mark.parametrize("model", ["mm", "hv"])
def test_oracle_equals_brute_force_operator_with_table_and_constant_sources(model):
    """The table and constant time functions, and two sources on one cell (their currents and
    imposed fields add)."""
    shape = (3, 2, 3)
    w, f = wl.random_state(model, shape, seed=12, media="few", n_sources=0)
    rng = np.random.default_rng(13)
    table = rng.standard_normal(20)  # shorter than the run: the source stops after t = 19
    w.sources = [
        wl.Source("current", np.array([1, 4]), wl.TimeFunction("table", 0.7, table=table),
                  w=rng.standard_normal((2, 3))),
        wl.Source("current", np.array([4, 9]), wl.TimeFunction("const", -0.3), w=rng.standard_normal((2, 3))),
        wl.Source("impose", np.array([7]), wl.TimeFunction("table", 1.3, table=table),
                  E0=tuple(rng.standard_normal(3)), B0=tuple(rng.standard_normal(3))),
        wl.Source("impose", np.array([7, 12]), wl.TimeFunction("sin", 0.9, 7.0, 0.4),
                  E0=tuple(rng.standard_normal(3)), B0=tuple(rng.standard_normal(3))),
    ]
    assert _run_both(model, shape, w, f, 30) < 1e-13


@pytest.mark.parametrize("model", ["mm", "hv"])
def test_brute_force_linear_part_matches_unit_responses(model):
    """Column c of the operator is the oracle's step of unit vector c (vacuum, no sources): the
    linear part alone, element by element."""
    shape = (2, 3, 2)
    G, b = O2.step_operator(model, shape, 1)
    assert not b.any()
    L = OracleLattice(model, shape)
    N = G.shape[0]
    worst = 0.0
    for c in range(0, N, 7):
        u = np.zeros(N)
        u[c] = 1.0
        L.set_populations(u.reshape(L.q, L.n), 0)
        L.step(1)
        worst = max(worst, float(np.abs(L.populations().reshape(-1) - G[:, c]).max()))
    assert worst < 1e-14
