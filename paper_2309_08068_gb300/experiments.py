"""The paper's four numerical experiments (Section IV), re-run on the GPU as refinement sweeps.

Each experiment keeps its physical setup fixed in units of the lattice length and refines the grid.
It reports the error measure the paper uses, and the GPU time of the time stepping alone (the paper
times only the integration of Maxwell's equations, not the set-up or the output). Both models run
the same sizes:

* ``pulse_interface``  Section IV-A: Gaussian pulse from vacuum into eps_r = 2.5; relative errors of
  the reflected and transmitted amplitudes against Fresnel's (sqrt r - 1)/(sqrt r + 1) and
  2/(sqrt r + 1).
* ``skin_effect``      Section IV-B: plane wave imposed at z = 0 into a conductor (z >= Lz/4,
  sigma = 0.1 eps / T, T = 17.68e-3 Lz / C); the cost C = sum over conductor cells of
  ((A_sim - A_theo) / A_theo)^2 with A_theo = A0 exp(-z/delta) and the paper's lossy-medium delta.
* ``dipole``           Section IV-C: Gaussian current J0 exp(-alpha |x - x_d|^2) sin(wt) z on an L^3
  lattice, T = 0.1768 Lz / C, run to t_max = 70 T / 25; the cost C of the E and B amplitudes along a
  line through the dipole perpendicular to it, against the Hertz dipole's exact amplitudes.
* ``multi_interface``  Section IV-D: pulse through permittivities 1, 1.3, 2, 3; relative error of the
  transmitted amplitude against the product of the three Fresnel transmissions.

The set-ups come from ``workloads``; the lattices run through the library (``lbm.Lattice``), timed
with CUDA events while ``lbm.Batch`` replays a captured CUDA graph of the steps.
Run ``python -m paper_2309_08068_gb300.experiments`` for every sweep (one JSON record per run).
"""
from __future__ import annotations

import argparse
import json
import math
import sys

import numpy as np

from . import workloads as wl

# Vacuum constants of each model (Section II-A for MM; HV: eps0 = mu0 = 3, the library default).
UNITS = {"mm": (1.0, 2.0), "hv": (3.0, 3.0)}

SIZES = {
    "pulse_interface": (256, 512, 1024, 2048, 4096, 8192),
    "skin_effect": (500, 1000, 2000, 4000, 8000),
    "dipole": (32, 48, 64, 96, 128, 192, 256),
    "multi_interface": (500, 1000, 2000, 3000, 4000, 6000, 8000),
}


# --- error measures (numpy, on fields read back from the GPU) ---------------------------------
def peak_parabola(y) -> float:
    """Signed value at the sample of largest |y|, refined by the parabola through it and its two
    neighbours (the sample itself at either end)."""
    y = np.asarray(y, dtype=np.float64)
    i = int(np.argmax(np.abs(y)))
    if i == 0 or i == y.size - 1:
        return float(y[i])
    a, b, c = y[i - 1], y[i], y[i + 1]
    curv = a - 2.0 * b + c
    if curv == 0.0:
        return float(b)
    s = 0.5 * (a - c) / curv  # offset of the vertex from sample i
    return float(b - 0.25 * (a - c) * s)


def fresnel(r: float):
    """Normal-incidence amplitude ratios of E from vacuum into relative permittivity r (mu_r = 1):
    reflected -(sqrt r - 1)/(sqrt r + 1) (E flips sign), transmitted 2/(sqrt r + 1)."""
    n = math.sqrt(r)
    return -(n - 1.0) / (n + 1.0), 2.0 / (n + 1.0)


def skin_depth(sigma: float, eps: float, mu: float, omega: float) -> float:
    """delta = sqrt(2 / (sigma mu omega)) sqrt(sqrt(1 + (omega eps / sigma)^2) + omega eps / sigma),
    the lossy-medium skin thickness of Section IV-B."""
    q = omega * eps / sigma
    return math.sqrt(2.0 / (sigma * mu * omega)) * math.sqrt(math.sqrt(1.0 + q * q) + q)


def dipole_amplitudes(r, p: float, omega: float, eps0: float, mu0: float):
    """|E| and |B| at distance r in the plane perpendicular to an oscillating dipole of amplitude p
    (near, intermediate and radiation terms). In that plane E = (p / 4 pi eps0) e^{ikr}
    (k^2/r - 1/r^3 + i k/r^2) along -p, and B = (mu0 c k^2 p / 4 pi r) e^{ikr} (1 + i/(kr)) around it,
    with k = omega / c, c = 1 / sqrt(eps0 mu0)."""
    r = np.asarray(r, dtype=np.float64)
    c = 1.0 / math.sqrt(eps0 * mu0)
    k = omega / c
    e = p / (4.0 * math.pi * eps0) * np.sqrt((k * k / r - 1.0 / r ** 3) ** 2 + (k / r ** 2) ** 2)
    b = mu0 * c * k * k * p / (4.0 * math.pi * r) * np.sqrt(1.0 + 1.0 / (k * r) ** 2)
    return e, b


def relative_cost(sim, theo) -> float:
    """The paper's cost: C = sum_j ((A_sim - A_theo) / A_theo)^2."""
    sim = np.asarray(sim, dtype=np.float64)
    theo = np.asarray(theo, dtype=np.float64)
    return float(np.sum(((sim - theo) / theo) ** 2))


# --- GPU runs --------------------------------------------------------------------------------
def _stream():
    import torch
    return torch.cuda.Stream()


def _lattice(w, stream):
    import torch
    from .lbm import lattice_from_workload
    with torch.cuda.stream(stream):
        return lattice_from_workload(w, stream=stream)


def _reinit(L, w):
    zeros = np.zeros((3, w.n), np.float32)
    L.init_fields(zeros if w.E is None else w.E, zeros if w.B is None else w.B)


GRAPH_STEPS = 2048


def time_steps(w, steps: int, repeats: int = 3):
    """GPU time of `steps` steps of workload w from its initial state. The steps run as replays of
    one captured CUDA graph of GRAPH_STEPS steps (lbm.Batch), and the remainder as plain launches.
    One untimed run first captures the graph, then each of `repeats` runs starts from a fresh
    initialisation and is timed with CUDA events. Returns (mean ms, sample standard deviation ms)."""
    import torch
    from .lbm import Batch
    stream = _stream()
    L = _lattice(w, stream)
    B = Batch([L])
    chunk = min(steps, GRAPH_STEPS)
    whole, rest = divmod(steps, chunk)

    def run():
        for _ in range(whole):
            B.step(chunk)
        if rest:
            L.step(rest)

    run()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    for _ in range(repeats):
        _reinit(L, w)
        torch.cuda.synchronize()
        e0.record(stream)
        run()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    B.close()
    L.close()
    mean = float(np.mean(times))
    std = float(np.std(times, ddof=1)) if len(times) > 1 else 0.0
    return mean, std


def _run_fields(w, steps: int, names: str = "E"):
    """Fields after `steps` steps (host arrays)."""
    stream = _stream()
    L = _lattice(w, stream)
    L.step(steps)
    out = L.fields_host(names)
    L.close()
    return out


def sinusoid_amplitude(series, omega: float):
    """Amplitude of a(t) = A cos(omega t + phi) + c fitted by least squares to samples t = 0, 1, ...
    (rows of `series`, one column per cell). A sampled maximum would underestimate A by up to
    1 - cos(pi / samples per period), 8 % at 8 samples."""
    y = np.asarray(series, dtype=np.float64)
    t = np.arange(y.shape[0], dtype=np.float64)
    X = np.stack([np.cos(omega * t), np.sin(omega * t), np.ones_like(t)], axis=1)
    coef, *_ = np.linalg.lstsq(X, y.reshape(y.shape[0], -1), rcond=None)
    return np.hypot(coef[0], coef[1]).reshape(y.shape[1:])


def _series(w, steps: int, window: int, picks):
    """Field samples of the last `window` of `steps` steps: picks is a list of (field letter,
    component, cell indices); returns one (window, len(cells)) array per pick."""
    import torch
    stream = _stream()
    L = _lattice(w, stream)
    L.step(steps - window)
    names = "".join(sorted({p[0] for p in picks}, key="EBDHJ".index))
    idx = [torch.as_tensor(np.asarray(c, dtype=np.int64), device=L.device) for _, _, c in picks]
    rows = [[] for _ in picks]
    with torch.cuda.stream(stream):  # the gathers follow the library's field kernel on its stream
        for _ in range(window):
            L.step(1)
            f = L.fields(names)
            for k, (name, comp, _) in enumerate(picks):
                rows[k].append(f[name][comp].index_select(0, idx[k]))
        out = [torch.stack(r).cpu().numpy() for r in rows]
    L.close()
    return out


def pulse_interface_setup(model: str, lz: int):
    """Section IV-A on a 1 x 1 x Lz lattice: E_x Gaussian (eq. Initialpulse) of unit amplitude at
    z0 = Lz/2 - Lz/6 with alpha = 0.05 Lz / sqrt 2; eps_r = 2.5 for z >= Lz/2. The fields are read
    0.3 Lz / C after the pulse centre reaches the interface."""
    c = wl.LIGHT_SPEED[model]
    z = np.arange(lz, dtype=np.float64)
    alpha = 0.05 * lz / math.sqrt(2.0)
    E, B = wl.gaussian_pulse_fields(model, z, lz / 2 - lz / 6, alpha, 1.0)
    steps = int(round((lz / 6) / c + 0.3 * lz / c))
    w = wl.Workload("pulse_interface", model, (1, 1, lz), steps, eps_r=np.where(z >= lz / 2, 2.5, 1.0), E=E, B=B)
    return w, alpha


def pulse_interface_errors(ex, lz: int, alpha: float):
    R, T = fresnel(2.5)
    a_r = peak_parabola(ex[: lz // 2 - int(2 * alpha)])
    a_t = peak_parabola(ex[lz // 2 + int(alpha):])
    return abs(a_r - R) / abs(R), abs(a_t - T) / T


def pulse_interface(model: str, lz: int, repeats: int = 3) -> dict:
    w, alpha = pulse_interface_setup(model, lz)
    ex = _run_fields(w, w.steps)["E"][0]
    err_r, err_t = pulse_interface_errors(ex, lz, alpha)
    ms, sd = time_steps(w, w.steps, repeats)
    return {"experiment": "pulse_interface", "model": model, "lz": lz, "cells": w.n, "steps": w.steps,
            "gpu_ms": ms, "gpu_ms_std": sd, "error_reflected": err_r, "error_transmitted": err_t}


def skin_effect_setup(model: str, lz: int):
    """Section IV-B on a 1 x 1 x Lz lattice: E = E0 sin(wt) x, B = E0/C sin(wt) y imposed at z = 0
    (E0 = 1), T = 17.68e-3 Lz / C, conductor for z >= Lz/4 with sigma = 0.1 eps0 / T (eps_r = 1).
    The run lasts 2 Lz / C (the transmitted wave crosses the conductor) rounded up to whole periods;
    the amplitude is fitted to the last two periods."""
    c = wl.LIGHT_SPEED[model]
    eps0, _ = UNITS[model]
    period = 17.68e-3 * lz / c
    sigma = 0.1 * eps0 / period
    z = np.arange(lz)
    src = wl.Source("impose", np.array([0], dtype=np.int64), wl.TimeFunction("sin", 1.0, period, 0.0),
                    E0=(1.0, 0.0, 0.0), B0=(0.0, 1.0 / c, 0.0))
    steps = int(math.ceil(2.0 * lz / c / period) * period)
    w = wl.Workload("skin_effect", model, (1, 1, lz), steps, sigma=np.where(z >= lz // 4, sigma, 0.0),
                    sources=[src])
    return w, period, sigma


def skin_effect_errors(model: str, amp, lz: int, period: float, sigma: float):
    eps0, mu0 = UNITS[model]
    omega = 2.0 * math.pi / period
    delta = skin_depth(sigma, eps0, mu0, omega)
    zc = lz // 4
    z = np.arange(zc, lz, dtype=np.float64)
    a = np.asarray(amp[zc:], dtype=np.float64)
    theo = a[0] * np.exp(-(z - zc) / delta)  # A0: the amplitude where the conductor begins
    fit = np.arange(zc + 2, min(lz - 1, int(zc + 2 * delta)))
    slope = np.polyfit(fit, np.log(np.asarray(amp, dtype=np.float64)[fit]), 1)[0]
    return relative_cost(a, theo), abs(-1.0 / slope - delta) / delta, delta


def skin_effect(model: str, lz: int, repeats: int = 3) -> dict:
    w, period, sigma = skin_effect_setup(model, lz)
    window = int(math.ceil(2 * period))
    (ex,) = _series(w, w.steps, window, [("E", 0, np.arange(lz))])
    amp = sinusoid_amplitude(ex, 2.0 * math.pi / period)
    cost, err_delta, delta = skin_effect_errors(model, amp, lz, period, sigma)
    ms, sd = time_steps(w, w.steps, repeats)
    return {"experiment": "skin_effect", "model": model, "lz": lz, "cells": w.n, "steps": w.steps,
            "gpu_ms": ms, "gpu_ms_std": sd, "cost": cost, "error_delta": err_delta, "delta_cells": delta}


def dipole_setup(model: str, n: int):
    """Section IV-C on an n^3 lattice: J0 = 1e-4, alpha = 0.5 at the centre, T = 0.1768 n / C,
    t_max = 70 T / 25. The line runs along +x from the dipole, from r = 3 (outside the source's
    support) to c (t_max - T), where the field has oscillated for a whole period. The amplitude is
    fitted to the last period (the run is only 2.8 periods long)."""
    c = wl.LIGHT_SPEED[model]
    period = 0.1768 * n / c
    steps = int(round(period * 70.0 / 25.0))
    w = wl.hertz_dipole(model, n=n, period=period, j0=1e-4, steps=steps)
    r_max = int(c * (steps - period))
    return w, period, r_max


def dipole_line(n: int, r_max: int):
    """Distances 3 .. r_max and cell indices of the line along +x from the centre cell."""
    ctr = n // 2
    r = np.arange(3, r_max + 1)
    return r, (ctr + r) + n * (ctr + n * ctr)


def dipole_errors(model: str, amp_e, amp_b, r, period: float, alpha: float = 0.5):
    """Costs of |E_z| and |B_y| along the line against the Hertz dipole with the paper's moment
    p = (J0 / omega)(pi / alpha)^1.5, and against the same with the source's form factor
    exp(-k^2 / (4 alpha)): outside a spherically symmetric Gaussian current the field is exactly a
    point dipole's with that factor on p (only the l = 0 term of the Green's function survives)."""
    eps0, mu0 = UNITS[model]
    omega = 2.0 * math.pi / period
    p = (1e-4 / omega) * (math.pi / alpha) ** 1.5
    k = omega * math.sqrt(eps0 * mu0)
    e_theo, b_theo = dipole_amplitudes(r, p, omega, eps0, mu0)
    ff = math.exp(-k * k / (4.0 * alpha))
    return {"cost_E": relative_cost(amp_e, e_theo), "cost_B": relative_cost(amp_b, b_theo),
            "cost_E_form_factor": relative_cost(amp_e, ff * e_theo),
            "cost_B_form_factor": relative_cost(amp_b, ff * b_theo), "form_factor": ff}


def dipole(model: str, n: int, repeats: int = 3) -> dict:
    w, period, r_max = dipole_setup(model, n)
    r, line = dipole_line(n, r_max)
    window = int(math.ceil(period))
    ez, by = _series(w, w.steps, window, [("E", 2, line), ("B", 1, line)])
    omega = 2.0 * math.pi / period
    costs = dipole_errors(model, sinusoid_amplitude(ez, omega), sinusoid_amplitude(by, omega), r, period)
    ms, sd = time_steps(w, w.steps, repeats)
    return {"experiment": "dipole", "model": model, "n": n, "cells": w.n, "steps": w.steps, "gpu_ms": ms,
            "gpu_ms_std": sd, "line_cells": int(r.size), **costs}


def multi_interface_steps(model: str, lz: int) -> int:
    """Time for the pulse centre to cross the three interfaces and run 0.05 Lz into eps_r = 3."""
    c = wl.LIGHT_SPEED[model]
    d = lz / 20.0
    return int((lz / 30.0) / c + d * math.sqrt(1.3) / c + 2 * d * math.sqrt(2.0) / c + 0.05 * lz * math.sqrt(3.0) / c)


def multi_interface_error(ex, lz: int) -> float:
    theory = 1.0
    for e1, e2 in ((1.0, 1.3), (1.3, 2.0), (2.0, 3.0)):
        theory *= 2.0 / (1.0 + math.sqrt(e2 / e1))
    a = np.asarray(ex[int(lz / 2.0 + 3 * lz / 20.0) + 1:], dtype=np.float64)
    return abs(float(a[np.argmax(np.abs(a))]) - theory) / theory


def multi_interface(model: str, lz: int, repeats: int = 3) -> dict:
    w = wl.multi_interface_1d(model, lz)
    steps = multi_interface_steps(model, lz)
    ex = _run_fields(w, steps)["E"][0]
    ms, sd = time_steps(w, steps, repeats)
    return {"experiment": "multi_interface", "model": model, "lz": lz, "cells": w.n, "steps": steps,
            "gpu_ms": ms, "gpu_ms_std": sd, "error_transmitted": multi_interface_error(ex, lz)}


EXPERIMENTS = {"pulse_interface": pulse_interface, "skin_effect": skin_effect, "dipole": dipole,
               "multi_interface": multi_interface}


def sweep(name: str, models=("mm", "hv"), sizes=None, repeats: int = 3):
    """One record per model and size of experiment `name`."""
    fn = EXPERIMENTS[name]
    return [fn(m, s, repeats) for m in models for s in (sizes or SIZES[name])]


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--experiment", choices=sorted(EXPERIMENTS) + ["all"], default="all")
    ap.add_argument("--repeats", type=int, default=3)
    ap.add_argument("--out", default=None, help="also write the records to this JSON file")
    args = ap.parse_args(argv)
    names = sorted(EXPERIMENTS) if args.experiment == "all" else [args.experiment]
    records = []
    for name in names:
        for rec in sweep(name, repeats=args.repeats):
            print(json.dumps(rec), flush=True)
            records.append(rec)
    if args.out:
        with open(args.out, "w") as fh:
            json.dump(records, fh, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
