"""The paper's experiments on the GPU against the same experiments on the FP64 oracle: the
measured errors and costs must agree (the GPU run differs from the oracle only by FP32 rounding),
and the errors must fall when the grid is refined (Section IV-A: a power law)."""
import math

import numpy as np
import pytest

from helpers import oracle_from_workload
from paper_2309_08068_gb300 import experiments as ex

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

MODELS = ("mm", "hv")


def oracle_series(w, steps, window, picks):
    O = oracle_from_workload(w, threads=8)
    O.step(steps - window)
    rows = [[] for _ in picks]
    for _ in range(window):
        O.step(1)
        F = O.fields()
        for k, (name, comp, cells) in enumerate(picks):
            rows[k].append(F[name][comp][np.asarray(cells)])
    return [np.array(r) for r in rows]


def close(gpu, cpu, rel):
    return abs(gpu - cpu) <= rel * abs(cpu) + 1e-6


@pytest.mark.parametrize("model", MODELS)
def test_pulse_interface_matches_the_oracle(model):
    rec = ex.pulse_interface(model, 512, repeats=1)
    w, alpha = ex.pulse_interface_setup(model, 512)
    O = oracle_from_workload(w, threads=8)
    O.step(w.steps)
    err_r, err_t = ex.pulse_interface_errors(O.fields()["E"][0], 512, alpha)
    assert close(rec["error_reflected"], err_r, 1e-3) and close(rec["error_transmitted"], err_t, 1e-3)
    assert rec["gpu_ms"] > 0 and rec["steps"] == w.steps


@pytest.mark.parametrize("model", MODELS)
def test_multi_interface_matches_the_oracle(model):
    from paper_2309_08068_gb300 import workloads as wl
    rec = ex.multi_interface(model, 1000, repeats=1)
    w = wl.multi_interface_1d(model, 1000)
    O = oracle_from_workload(w, threads=8)
    O.step(ex.multi_interface_steps(model, 1000))
    assert close(rec["error_transmitted"], ex.multi_interface_error(O.fields()["E"][0], 1000), 1e-3)


@pytest.mark.parametrize("model", MODELS)
def test_skin_effect_matches_the_oracle(model):
    rec = ex.skin_effect(model, 500, repeats=1)
    w, period, sigma = ex.skin_effect_setup(model, 500)
    (series,) = oracle_series(w, w.steps, int(math.ceil(2 * period)), [("E", 0, np.arange(500))])
    amp = ex.sinusoid_amplitude(series, 2 * math.pi / period)
    cost, err_delta, _ = ex.skin_effect_errors(model, amp, 500, period, sigma)
    assert close(rec["cost"], cost, 1e-3) and close(rec["error_delta"], err_delta, 1e-3)


@pytest.mark.parametrize("model", MODELS)
def test_dipole_matches_the_oracle(model):
    rec = ex.dipole(model, 32, repeats=1)
    w, period, r_max = ex.dipole_setup(model, 32)
    r, line = ex.dipole_line(32, r_max)
    ez, by = oracle_series(w, w.steps, int(math.ceil(period)), [("E", 2, line), ("B", 1, line)])
    om = 2 * math.pi / period
    costs = ex.dipole_errors(model, ex.sinusoid_amplitude(ez, om), ex.sinusoid_amplitude(by, om), r, period)
    for key in ("cost_E", "cost_B", "cost_E_form_factor", "cost_B_form_factor"):
        assert close(rec[key], costs[key], 1e-3), key


@pytest.mark.parametrize("model", MODELS)
def test_interface_errors_fall_under_refinement(model):
    coarse = ex.pulse_interface(model, 512, repeats=1)
    fine = ex.pulse_interface(model, 2048, repeats=1)
    assert fine["error_reflected"] < coarse["error_reflected"]
    assert fine["error_transmitted"] < coarse["error_transmitted"]
