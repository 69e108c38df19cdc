"""Physics pins of the oracle's reported fields and of its source time argument. No GPU.

Two conventions of the oracle are not visible in E and B alone:
  * the magnetic field it reports, H = B / (mu0 mu_r) (Section II-A units for MM: eps0 = 1, mu0 = 2;
    Section III-A for HV: eps0 mu0 = 9), and D = eps0 eps_r E;
  * the time argument of a source: iteration t of the Appendix B loop (t = 1 .. t_max) evaluates the
    source at s(t), and the sin and table forms of s agree.
Both are checked here against what Maxwell's equations fix: the electromagnetic energy
(1/2) sum (E.D + B.H) of a lossless run is conserved and splits equally between E and B in a
travelling wave, and the wave radiated by a current sheet is the retarded current.
"""
import numpy as np
import pytest

from oracle import OracleLattice, TimeFn
from paper_2309_08068_gb300 import workloads as wl

C = wl.LIGHT_SPEED
UNITS = {"mm": (1.0, 2.0), "hv": (3.0, 3.0)}  # (eps0, mu0) of each model


def _energies(F):
    return 0.5 * float(np.sum(F["E"] * F["D"])), 0.5 * float(np.sum(F["B"] * F["H"]))


@pytest.mark.parametrize("model", ["mm", "hv"])
@pytest.mark.parametrize("medium", ["vacuum", "dielectric", "magnetic"])
def test_field_energy_is_conserved_and_equipartitioned(model, medium):
    """A Gaussian E_x with B = 0 (no charge, no current, sigma = 0) splits into two one-way pulses.
    With the D and H the oracle reports, (1/2) sum (E.D + B.H) must stay at its initial, purely
    electric, value (Poynting's theorem on the periodic lattice), and after the split the electric and
    magnetic halves must be equal, as in any plane wave with B = E / c. The slab 400 <= z <= 700 has
    eps_r = 2.5 or mu_r = 2.5, and the pulses are inside it at the later checks.

    A factor mu0 missing from H (H = B / mu_r, eq. MacroscopicBMiller read literally) gives 3/4 of
    the energy for MM; H without mu_r, or D without eps0 or eps_r, breaks conservation inside the
    slab or at t = 0."""
    n = 1024
    z = np.arange(n, dtype=np.float64)
    slab = np.where((z >= 400) & (z <= 700), 2.5, 1.0)
    eps_r = slab if medium == "dielectric" else None
    mu_r = slab if medium == "magnetic" else None
    E, _ = wl.gaussian_pulse_fields(model, z, 200.0, 20.0, 1.0)
    L = OracleLattice(model, (1, 1, n), eps_r=eps_r, mu_r=mu_r, threads=4)
    L.init_fields(E, np.zeros_like(E))
    ue0, ub0 = _energies(L.fields())
    eps0, _ = UNITS[model]
    assert ub0 < 1e-20 * ue0
    assert abs(ue0 - 0.5 * eps0 * np.sum(E[0] ** 2)) < 1e-12 * ue0
    split = {"mm": 200, "hv": 300}[model]      # both pulses in vacuum, 100+ cells apart
    checks = {"mm": (100, 200, 400, 600), "hv": (100, 300, 800, 1000)}[model]
    inside = 0.0
    for t in checks:
        L.step(t - L.time)
        F = L.fields()
        ue, ub = _energies(F)
        assert abs((ue + ub) / ue0 - 1.0) < 1e-3, (t, ue / ue0, ub / ue0)
        if t == split:
            assert abs(ue - ub) < 1e-3 * ue0, (t, ue / ue0, ub / ue0)
        dens = F["E"][0] * F["D"][0] + F["B"][1] * F["H"][1]
        inside = max(inside, float(dens[400:701].sum() / dens.sum()))
    if medium != "vacuum":
        assert inside > 0.3  # a pulse was inside the slab at one of the checks


def _phase_lead(model, period, phase, dzs=(40, 80, 120, 160)):
    """Current sheet J_x = s(t) at z_s in a 1 x 1 x 1600 vacuum lattice. Fits E_x(z_s + dz, t) over
    two periods to A sin(w t + phi) and returns, per |dz|, the lead delta in
    E_x(z, t) = -(Z/2) s(t + delta - |dz| / C)."""
    nz, zs, t_end = 1600, 800, 700
    L = OracleLattice(model, (1, 1, nz), threads=4)
    L.init_fields(np.zeros((3, nz)), np.zeros((3, nz)))
    L.add_current([zs], np.array([[1.0, 0.0, 0.0]]), TimeFn("sin", 1.0, period, phase))
    span = 2 * int(period)
    L.step(t_end - span)
    rec, ts = [], []
    for _ in range(span):
        L.step(1)
        rec.append(L.fields()["E"][0].copy())
        ts.append(L.time)
    rec = np.array(rec)
    ts = np.array(ts, dtype=np.float64)
    w = 2.0 * np.pi / period
    M = np.stack([np.sin(w * ts), np.cos(w * ts), np.ones_like(ts)], axis=1)
    eps0, mu0 = UNITS[model]
    out = []
    for sign in (1, -1):
        for dz in dzs:
            a, b, _ = np.linalg.lstsq(M, rec[:, zs + sign * dz], rcond=None)[0]
            amp, phi = np.hypot(a, b), np.arctan2(b, a)
            assert abs(amp / (0.5 * np.sqrt(mu0 / eps0)) - 1.0) < 0.03  # 13+ cells per wavelength
            # -sin(x) = sin(x + pi): phi = w (delta - |dz|/C) + phase + pi (mod 2 pi)
            delta = (phi - np.pi - phase) / w + dz / C[model]
            delta = (delta + period / 2) % period - period / 2
            out.append((dz, delta))
    return out


@pytest.mark.parametrize("model,lead", [("mm", 1.0), ("hv", 0.5)])
@pytest.mark.parametrize("period,phase", [(80.0, 1.0), (40.0, -0.7)])
def test_sheet_radiation_follows_the_source_time_argument(model, lead, period, phase):
    """A sheet current radiates E_x(z, t) = -(Z/2) J(t - |z - z_s| / c) both ways (Maxwell's
    equations, Section I-B). Iteration t of the Appendix B loop takes the lattice from time t - 1 to
    t with the current s(t), so the lattice's J(t) is s(t) shifted by how the step applies it:
      * HV: the source term of iteration t moves D by -s(t) (Appendix A, sum_i T_i = -J), all of it
        within the step that ends at t: the current is centred half a step before its label, and
        the field leads s by 1/2 step;
      * MM: D' moves by -s(t) in the same way, and the reported D = D' - mu0 J/4 takes the next
        iteration's current, so D moves by -(s(t) + s(t + 1))/2 per step: centred one step before
        the label, the field leads s by 1 step.
    The phase of the far field, extrapolated to the sheet (the lattice's dispersion adds a delay
    that grows linearly with distance), must show this lead within 0.1 step on both sides. Evaluating
    the source at s(t - 1) or s(t + 1) moves it by a whole step, and a wrong sign of the phase by
    2 |phase| period / (2 pi) steps."""
    pts = _phase_lead(model, period, phase)
    d = np.array([p[0] for p in pts], dtype=np.float64)
    delta = np.array([p[1] for p in pts])
    slope, intercept = np.polyfit(d, delta, 1)
    assert abs(intercept - lead) < 0.1, (intercept, pts)
    assert np.abs(delta - (intercept + slope * d)).max() < 0.02  # same law on both sides
    assert abs(slope) < 0.02  # the dispersion delay stays small at these wavelengths


@pytest.mark.parametrize("model", ["mm", "hv"])
def test_table_source_equals_the_sine_it_tabulates(model):
    """s(t) = amp table[t] (zero past the table) and s(t) = amp sin(2 pi t / T + phase) must drive
    the same run when table[t] holds that sine: with iteration t using s(t) in both, the populations
    agree up to rounding through t = len - 1 and differ from t = len on, when the table has run
    out. A table read at t - 1 or t + 1 breaks the first; a source that does not stop breaks the
    second."""
    nz, zs, period, phase, length = 256, 128, 24.0, 0.9, 60
    rng = np.random.default_rng(7)
    wvec = rng.standard_normal((3, 3))
    cells = [zs - 1, zs, zs + 1]
    t = np.arange(length)
    table = np.sin(2.0 * np.pi * t / period + phase)
    runs = {}
    for kind in ("sin", "table"):
        L = OracleLattice(model, (1, 1, nz), threads=2)
        L.init_fields(np.zeros((3, nz)), np.zeros((3, nz)))
        fn = TimeFn("sin", 1.7, period, phase) if kind == "sin" else TimeFn("table", 1.7, table=table)
        L.add_current(cells, wvec, fn)
        L.step(length - 1)
        before = L.populations()
        L.step(1)
        runs[kind] = (before, L.populations())
    scale = np.abs(runs["sin"][0]).max()
    assert scale > 0
    assert np.abs(runs["sin"][0] - runs["table"][0]).max() < 1e-13 * scale
    assert np.abs(runs["sin"][1] - runs["table"][1]).max() > 1e-3 * scale
