"""The error measures of the paper's experiments (paper_2309_08068_gb300.experiments), pinned on
CPU to facts outside the code: energy balance at an interface, the limits of the skin depth and of
the dipole field, a brute-force lattice sum for the Gaussian source's form factor, and exact
recovery of a sampled sinusoid and parabola. No GPU."""
import math

import numpy as np
import pytest

from paper_2309_08068_gb300 import experiments as ex
from paper_2309_08068_gb300 import workloads as wl


@pytest.mark.parametrize("r", [1.3, 2.5, 9.0])
def test_fresnel_conserves_energy(r):
    R, T = ex.fresnel(r)
    assert R < 0 < T
    assert R * R + math.sqrt(r) * T * T == pytest.approx(1.0, rel=1e-14)  # |R|^2 + n2/n1 |T|^2 = 1
    assert 1.0 + R == pytest.approx(T)  # E tangential is continuous


def test_skin_depth_limits():
    eps, mu, om = 3.0, 3.0, 0.01
    good = ex.skin_depth(1e4, eps, mu, om)  # sigma >> omega eps
    assert good == pytest.approx(math.sqrt(2.0 / (1e4 * mu * om)), rel=1e-5)
    low = ex.skin_depth(1e-6, eps, mu, om)  # sigma << omega eps: delta = (2 / sigma) sqrt(eps / mu)
    assert low == pytest.approx(2.0 / 1e-6 * math.sqrt(eps / mu), rel=1e-6)


@pytest.mark.parametrize("model", ["mm", "hv"])
def test_dipole_amplitudes_limits(model):
    eps0, mu0 = ex.UNITS[model]
    c = 1.0 / math.sqrt(eps0 * mu0)
    p, om = 2.0, 0.3
    k = om / c
    far = np.array([1e4 / k])
    e, b = ex.dipole_amplitudes(far, p, om, eps0, mu0)
    assert e[0] == pytest.approx(p * k * k / (4 * math.pi * eps0 * far[0]), rel=1e-7)
    assert b[0] == pytest.approx(e[0] / c, rel=1e-7)
    near = np.array([1e-4 / k])
    e, b = ex.dipole_amplitudes(near, p, om, eps0, mu0)
    assert e[0] == pytest.approx(p / (4 * math.pi * eps0 * near[0] ** 3), rel=1e-6)  # static dipole
    assert b[0] == pytest.approx(mu0 * om * p / (4 * math.pi * near[0] ** 2), rel=1e-6)  # Biot-Savart, I dl = omega p


@pytest.mark.parametrize("k", [0.14, 0.5, 1.1])
def test_gaussian_source_form_factor_by_lattice_sum(k):
    """Outside a spherically symmetric source the l = 0 term alone survives, weighting each source
    point by j0(k r'). Summed over the lattice for the dipole's weights exp(-0.5 r^2), that gives
    (pi / alpha)^1.5 exp(-k^2 / (4 alpha)), the factor the dipole costs use."""
    cells, W = wl.dipole_cells((40, 40, 40), (20, 20, 20), alpha=0.5, r2_max=300.0)
    z, y, x = np.divmod(cells, 1600)[0], (cells // 40) % 40, cells % 40
    r = np.sqrt((x - 20.0) ** 2 + (y - 20.0) ** 2 + (z - 20.0) ** 2)
    j0 = np.where(r > 0, np.sin(k * r) / np.where(r > 0, k * r, 1.0), 1.0)
    total = float(np.sum(W[:, 2] * j0))
    # the lattice sum differs from the integral by aliased terms of relative size about
    # exp(-(2 pi - k)^2 / (4 alpha)), 1.5e-6 at k = 1.1 (Poisson summation)
    assert total == pytest.approx((math.pi / 0.5) ** 1.5 * math.exp(-k * k / 2.0), rel=1e-5)


def test_sinusoid_amplitude_is_exact_for_a_sampled_sinusoid():
    period = 8.3
    om = 2 * math.pi / period
    t = np.arange(17)[:, None]
    A = np.array([1.0, 0.25, 3.0])
    y = A * np.cos(om * t + np.array([0.3, 2.0, -1.0])) + np.array([0.1, -0.2, 0.0])
    assert np.allclose(ex.sinusoid_amplitude(y, om), A, rtol=1e-12)
    assert np.max(np.abs(y[:9, 0] - 0.1)) < 1.0  # a sampled maximum misses the amplitude


def test_peak_parabola_and_cost():
    z = np.arange(3.0, 12.0)
    y = -(2.0 - 0.05 * (z - 7.3) ** 2)
    assert ex.peak_parabola(y) == pytest.approx(-2.0, rel=1e-12)
    assert ex.relative_cost([1.0, 2.0], [1.0, 2.0]) == 0.0
    assert ex.relative_cost([1.1, 1.8], [1.0, 2.0]) == pytest.approx(0.01 + 0.01)


@pytest.mark.parametrize("model", ["mm", "hv"])
def test_setups_follow_the_paper(model):
    c = wl.LIGHT_SPEED[model]
    w, alpha = ex.pulse_interface_setup(model, 600)
    assert alpha == pytest.approx(0.05 * 600 / math.sqrt(2))
    assert w.eps_r[299] == 1.0 and w.eps_r[300] == 2.5
    assert int(np.argmax(w.E[0])) == 200
    w, period, sigma = ex.skin_effect_setup(model, 1000)
    eps0, _ = ex.UNITS[model]
    assert period == pytest.approx(17.68e-3 * 1000 / c)
    assert sigma == pytest.approx(0.1 * eps0 / period)
    assert w.sigma[249] == 0.0 and w.sigma[250] == pytest.approx(sigma)
    assert w.steps >= 2 * 1000 / c
    w, period, r_max = ex.dipole_setup(model, 64)
    assert period == pytest.approx(0.1768 * 64 / c)
    assert w.steps == round(period * 70 / 25)
    assert 3 < r_max < 32 - 3  # inside the wave front, away from the periodic images
