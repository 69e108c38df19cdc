"""Pins of the FP64 oracle's three-dimensional radiation against electromagnetism. No GPU.

The Gaussian current of Section IV-C radiates as a Hertz dipole. Outside a spherically symmetric
source the field is exactly a point dipole's, with moment p = (J0 / omega)(pi / alpha)^1.5 times
the form factor exp(-k^2 / (4 alpha)). These tests check the oracle's field against that closed
form: its angular pattern, its 1/r amplitude and its absolute size, which depends on the model's
mu0 and on how the current enters Ampere's law. They also check that B stays nearly solenoidal
(div B is not exactly zero on the lattice, but small). Mistakes these catch include a wrong sign or axis in a magnetic vector b, a wrong mu0
or eps0, a current entering with the wrong factor, and a transposed advection.
"""
import math

import numpy as np
import pytest

from helpers import oracle_from_workload
from paper_2309_08068_gb300 import experiments as ex
from paper_2309_08068_gb300 import workloads as wl

UNITS = {"mm": (1.0, 2.0), "hv": (3.0, 3.0)}
ALPHA = 0.5  # the Gaussian's exponent, Section IV-C


def point_dipole_e(r, theta, p, k, eps0):
    """|E_theta| and |E_r| of an oscillating point dipole p (along z) at distance r and polar angle
    theta: (p k^3 / 4 pi eps0) sin(theta) |1/(kr) + i/(kr)^2 - 1/(kr)^3| and
    (p k^3 / 4 pi eps0) 2 cos(theta) |i/(kr)^2 - 1/(kr)^3|."""
    kr = k * r
    a = p * k ** 3 / (4.0 * math.pi * eps0)
    e_t = a * math.sin(theta) * math.hypot(1.0 / kr - 1.0 / kr ** 3, 1.0 / kr ** 2)
    e_r = a * 2.0 * math.cos(theta) * math.hypot(1.0 / kr ** 2, 1.0 / kr ** 3)
    return e_t, e_r


# Sample points in the x-z plane through the source: (dx, dz) from it.
POINTS = [(19, 0), (14, 0), (17, 10), (14, 14), (10, 17)]
# Lattice, period (about 11 cells per wavelength) and sampling window for each model: the window
# starts a period after the wave has passed the farthest point and ends before the first wave from
# a periodic image of the source arrives (it travels n - 20 cells).
SETUP = {"mm": dict(n=80, period=16.0, first=48, window=32), "hv": dict(n=80, period=32.0, first=100, window=64)}


@pytest.fixture(scope="module", params=["mm", "hv"])
def dipole_run(request):
    model = request.param
    s = SETUP[model]
    n, period = s["n"], s["period"]
    c = wl.LIGHT_SPEED[model]
    assert s["first"] > 20.0 / c + period and s["first"] + s["window"] < (n - 20) / c
    w = wl.hertz_dipole(model, n=n, period=period, j0=1e-4)
    O = oracle_from_workload(w, threads=16)
    O.step(s["first"])
    ctr = n // 2
    cells = [(ctr + dx) + n * (ctr + n * (ctr + dz)) for dx, dz in POINTS]
    rows = []
    for _ in range(s["window"]):
        O.step(1)
        E = O.fields()["E"]
        rows.append(E[:, cells])
    series = np.array(rows)  # window x 3 x points
    omega = 2.0 * math.pi / period
    return model, series, omega


def projected_amplitudes(series, omega):
    """Fitted amplitudes of E . theta_hat and E . r_hat at each sample point."""
    out = []
    for k, (dx, dz) in enumerate(POINTS):
        r = math.hypot(dx, dz)
        th = math.atan2(dx, dz)  # polar angle from +z
        ex_, ez = series[:, 0, k], series[:, 2, k]
        e_theta = ex_ * math.cos(th) - ez * math.sin(th)
        e_r = ex_ * math.sin(th) + ez * math.cos(th)
        a_t = float(ex.sinusoid_amplitude(e_theta[:, None], omega)[0])
        a_r = float(ex.sinusoid_amplitude(e_r[:, None], omega)[0])
        out.append((r, th, a_t, a_r))
    return out


def test_dipole_field_matches_a_point_dipole(dipole_run):
    """Section IV-C source, Hertz-dipole closed form: |E_theta| within 10 % at every point. The
    absolute amplitude fixes mu0, eps0 and the current's normalisation (a wrong mu0 is a factor 2
    or 3). Measured: 0.95-1.02 of the closed form (MM), 0.99-1.08 (HV); at about 11 cells per
    wavelength the lattice's anisotropy accounts for the rest."""
    model, series, omega = dipole_run
    eps0, mu0 = UNITS[model]
    k = omega * math.sqrt(eps0 * mu0)
    p = (1e-4 / omega) * (math.pi / ALPHA) ** 1.5 * math.exp(-k * k / (4.0 * ALPHA))
    for r, th, a_t, _ in projected_amplitudes(series, omega):
        e_t, _ = point_dipole_e(r, th, p, k, eps0)
        assert abs(a_t / e_t - 1.0) < 0.10, (model, r, math.degrees(th), a_t, e_t)


def test_dipole_pattern_is_sin_theta_over_r(dipole_run):
    """The shape alone, normalised by the point at 90 degrees and 19 cells: the ratios follow
    sin(theta) and 1/r (with the near-field terms of the closed form) within 10 % (measured: up to
    6 % for MM and 8 % for HV, at 45 degrees). A sin^2 pattern would be 50 % off at 30 degrees."""
    model, series, omega = dipole_run
    eps0, mu0 = UNITS[model]
    k = omega * math.sqrt(eps0 * mu0)
    amps = projected_amplitudes(series, omega)
    r0, th0, a0, _ = amps[0]
    e0, _ = point_dipole_e(r0, th0, 1.0, k, eps0)
    for r, th, a_t, _ in amps[1:]:
        e_t, _ = point_dipole_e(r, th, 1.0, k, eps0)
        assert abs((a_t / a0) / (e_t / e0) - 1.0) < 0.10, (model, r, math.degrees(th))


def test_radial_field_is_a_near_field(dipole_run):
    """E_r of a dipole falls like 1/r^2 and vanishes at 90 degrees: on the equator it is below 5 % of
    E_theta, and off the equator the ratio E_r / E_theta matches the closed form's to 0.03
    (measured: within 0.02)."""
    model, series, omega = dipole_run
    eps0, mu0 = UNITS[model]
    k = omega * math.sqrt(eps0 * mu0)
    amps = projected_amplitudes(series, omega)
    assert amps[0][3] < 0.05 * amps[0][2]
    for r, th, a_t, a_r in amps[2:]:
        e_t, e_r = point_dipole_e(r, th, 1.0, k, eps0)
        assert abs(a_r / a_t - e_r / e_t) < 0.03, (model, r, math.degrees(th), a_r / a_t, e_r / e_t)


def div_and_curl_norms(B, n, exclude_r=6.0):
    """Central-difference div B and curl B on a periodic n^3 lattice, as L2 norms over the cells
    farther than exclude_r from the centre."""
    b = [B[a].reshape(n, n, n) for a in range(3)]  # index [z, y, x]

    def d(f, axis):  # axis 0 = x, 1 = y, 2 = z
        ax = 2 - axis
        return 0.5 * (np.roll(f, -1, axis=ax) - np.roll(f, 1, axis=ax))

    div = d(b[0], 0) + d(b[1], 1) + d(b[2], 2)
    curl = [d(b[2], 1) - d(b[1], 2), d(b[0], 2) - d(b[2], 0), d(b[1], 0) - d(b[0], 1)]
    g = np.arange(n) - n // 2
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    far = x * x + y * y + z * z > exclude_r * exclude_r
    return float(np.linalg.norm(div[far])), float(np.linalg.norm(np.stack([c[far] for c in curl])))


@pytest.mark.parametrize("model", ["mm", "hv"])
def test_magnetic_field_stays_nearly_solenoidal(model):
    """div B of the radiated field is not round-off zero on the lattice, but it stays small next to
    curl B: below 5 % outside the source's support, at periods 24 and 48 (32^3, 40 and 80 steps).
    Measured: MM 0.97 % and 1.5 %, HV 3.2 % and 1.6 %. HV's ratio halves when the wavelength
    doubles; MM's stays near 1 %, set by the sharp Gaussian source's near field, which does not
    scale with the wavelength. A magnetic vector with a wrong sign or axis breaks this."""
    n = 32
    for period, steps in ((24.0, 40), (48.0, 80)):
        w = wl.hertz_dipole(model, n=n, period=period, j0=1e-4)
        O = oracle_from_workload(w, threads=16)
        O.step(steps)
        div, curl = div_and_curl_norms(O.fields()["B"], n)
        assert div / curl < 5e-2, (model, period, div / curl)
