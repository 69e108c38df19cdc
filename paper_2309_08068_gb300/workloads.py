"""Seeded synthetic inputs for the MM and HV lattice-Boltzmann Maxwell solvers.

This module only builds inputs: media arrays, initial E and B fields, and source descriptions
(cells, weights, time functions). It contains none of the schemes' arithmetic, so the GPU path and
the FP64 oracle can both take their inputs from it. The setups restate the paper's tests
(arXiv 2309.08068, Section IV) at the sizes used by the benchmark and the parity tests:

* ``dielectric_pulse_1d``  - Section IV-A, Gaussian pulse (eq. Initialpulse) into a dielectric slab.
* ``hertz_dipole``         - Section IV-C, Gaussian current J0 exp(-alpha |x - x_d|^2) sin(wt) z.
* ``slab_pulse``           - plane pulse through 64 random dielectric slabs (many interfaces, 3-D).
* ``multi_interface_1d``   - Section IV-D, pulse through permittivities 1, 1.3, 2, 3.
* ``skin_effect_1d``       - Section IV-B, plane wave imposed at z = 0 into a conductor.
* ``skin_effect_3d``, ``refinement_batch`` - the same on N^3 lattices, N = 32 ... 272 (the
  mesh-refinement sweep run as one batch).
* ``random_medium_dipole`` - dipole in a per-cell random permittivity.
* ``random_state``         - random populations and media for element-wise parity tests.

Cell index is ``x + nx * (y + ny * z)`` (x fastest); vector fields are ``(3, n)`` component-major.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Vacuum light speed of each model in lattice units: 1/sqrt(2) for MM (Section II-A, eps0 = 1,
# mu0 = 2) and 1/3 for HV (Section III-A).
LIGHT_SPEED = {"mm": 1.0 / np.sqrt(2.0), "hv": 1.0 / 3.0}
# Populations per cell the paper counts (Section II: 50, Section III: 36).
POPULATIONS = {"mm": 50, "hv": 36}


@dataclass
class TimeFunction:
    """s(t): ``sin`` -> amplitude sin(2 pi t / period + phase); ``table`` -> amplitude table[t]
    (zero outside the table); ``const`` -> amplitude."""
    kind: str = "sin"
    amplitude: float = 1.0
    period: float = 1.0
    phase: float = 0.0
    table: np.ndarray | None = None


@dataclass
class Source:
    """``current``: J_ext(x, t) += w(x) s(t) at ``cells`` (w is (n_cells, 3)).
    ``impose``: after each collision the cells are set to f_eq(E0 s(t), B0 s(t), J = 0)."""
    kind: str
    cells: np.ndarray
    fn: TimeFunction
    w: np.ndarray | None = None
    E0: tuple = (0.0, 0.0, 0.0)
    B0: tuple = (0.0, 0.0, 0.0)


@dataclass
class Workload:
    name: str
    model: str
    shape: tuple  # (nx, ny, nz)
    steps: int
    eps_r: np.ndarray | None = None  # per cell, float64, or None for 1
    mu_r: np.ndarray | None = None   # per cell, or None for 1
    sigma: np.ndarray | None = None  # per cell, or None for 0
    E: np.ndarray | None = None      # (3, n) initial field, or None for zero
    B: np.ndarray | None = None
    sources: list = field(default_factory=list)

    @property
    def n(self) -> int:
        nx, ny, nz = self.shape
        return nx * ny * nz


def _grid(shape):
    nx, ny, nz = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.reshape(-1), y.reshape(-1), z.reshape(-1)


def gaussian_pulse_fields(model: str, coord: np.ndarray, center: float, width: float, amplitude: float,
                          axis: str = "z", local_speed: np.ndarray | float | None = None):
    """eq. Initialpulse: E = E0 exp(-(s - s0)^2 / (2 alpha^2)) along the first transverse axis and
    B = E / c along the second, so that E x B points along +axis. ``local_speed`` is the wave speed
    at each cell (the model's C / sqrt(eps_r mu_r)); default: the vacuum speed."""
    c = LIGHT_SPEED[model] if local_speed is None else local_speed
    g = amplitude * np.exp(-((coord - center) ** 2) / (2.0 * width ** 2))
    n = coord.size
    E = np.zeros((3, n))
    B = np.zeros((3, n))
    e_ax, b_ax = {"z": (0, 1), "x": (1, 2), "y": (2, 0)}[axis]
    E[e_ax] = g
    B[b_ax] = g / c
    return E, B


def dielectric_pulse_1d(model: str, nz: int = 1024, steps: int = 1500) -> Workload:
    """Pulse through a dielectric slab on a 1 x 1 x nz periodic lattice (Section IV-A geometry at the
    benchmark's size): vacuum for z < 400 and z > 700, eps_r = 2.5 for 400 <= z <= 700; E_x Gaussian
    centred at z = 200, width 20 cells, amplitude 1e-4; B_y = E_x / C."""
    z = np.arange(nz, dtype=np.float64)
    eps = np.where((z >= 400) & (z <= 700), 2.5, 1.0)
    E, B = gaussian_pulse_fields(model, z, 200.0, 20.0, 1e-4)
    return Workload("dielectric_pulse_1d", model, (1, 1, nz), steps, eps_r=eps, E=E, B=B)


def multi_interface_1d(model: str, lz: int) -> Workload:
    """Section IV-D: permittivities 1, 1.3, 2, 3 with interfaces at z0, z0 + d, z0 + 3d (z0 = Lz/2,
    d = Lz/20); pulse of unit amplitude at z0 - Lz/30 with alpha = Lz/(100 sqrt 2)."""
    z = np.arange(lz, dtype=np.float64)
    z0, d = lz / 2.0, lz / 20.0
    eps = np.ones(lz)
    eps[z >= z0] = 1.3
    eps[z >= z0 + d] = 2.0
    eps[z >= z0 + 3 * d] = 3.0
    E, B = gaussian_pulse_fields(model, z, z0 - lz / 30.0, lz / (100.0 * np.sqrt(2.0)), 1.0)
    return Workload("multi_interface_1d", model, (1, 1, lz), 0, eps_r=eps, E=E, B=B)


def dipole_cells(shape, center, alpha: float = 0.5, r2_max: float = 36.0):
    """Cells and weights exp(-alpha |x - x_d|^2) of the Section IV-C Gaussian current, truncated at
    |x - x_d|^2 <= r2_max (the weight there is below 2e-8 of the peak). Periodic wrap."""
    nx, ny, nz = shape
    r = int(np.floor(np.sqrt(r2_max)))
    cells, w = [], []
    cx, cy, cz = center
    for dz in range(-r, r + 1):
        for dy in range(-r, r + 1):
            for dx in range(-r, r + 1):
                d2 = dx * dx + dy * dy + dz * dz
                if d2 > r2_max:
                    continue
                x, y, z = (cx + dx) % nx, (cy + dy) % ny, (cz + dz) % nz
                cells.append(x + nx * (y + ny * z))
                w.append(np.exp(-alpha * d2))
    cells = np.asarray(cells, dtype=np.int64)
    order = np.argsort(cells, kind="stable")
    cells = cells[order]
    wz = np.asarray(w)[order]
    if np.unique(cells).size != cells.size:
        raise ValueError("dipole support overlaps itself; lattice too small for r2_max")
    W = np.zeros((cells.size, 3))
    W[:, 2] = wz
    return cells, W


def hertz_dipole(model: str, n: int = 256, period: float = 32.0, j0: float = 1e-4, steps: int = 2000,
                 r2_max: float = 36.0, nz: int | None = None) -> Workload:
    """Hertz dipole in an n^3 vacuum lattice (Section IV-C source at the benchmark's size): current
    J0 exp(-0.5 |x - x_d|^2) sin(2 pi t / period) z at the centre cell, truncated at |x - x_d|^2 <=
    r2_max, zero initial fields. nz, when given, makes the lattice n x n x nz (a thinner copy of the
    same problem for profiling)."""
    shape = (n, n, n if nz is None else nz)
    cells, W = dipole_cells(shape, (n // 2, n // 2, shape[2] // 2), r2_max=r2_max)
    src = Source("current", cells, TimeFunction("sin", j0, period, 0.0), w=W)
    return Workload("hertz_dipole", model, shape, steps, sources=[src])


def slab_pulse(model: str, shape=(512, 64, 64), seed: int = 3, steps: int = 3000) -> Workload:
    """Plane pulse through 64 dielectric slabs along x (8 cells each), eps_r per slab uniform in
    [1, 8) from numpy's default_rng(seed); E_y Gaussian centred at x = 64, width 16 cells, amplitude
    1e-4, uniform in y and z; B_z = E_y / c_local with the slab's local speed."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    nslab = 64
    slab_eps = rng.uniform(1.0, 8.0, nslab)
    x, _, _ = _grid(shape)
    eps = slab_eps[np.minimum(x * nslab // nx, nslab - 1)].astype(np.float64)
    c_local = LIGHT_SPEED[model] / np.sqrt(eps)
    E, B = gaussian_pulse_fields(model, x.astype(np.float64), 64.0, 16.0, 1e-4, axis="x", local_speed=c_local)
    return Workload("slab_pulse", model, shape, steps, eps_r=eps, E=E, B=B)


def skin_effect_1d(model: str, nz: int, sigma: float, periods: float = 12.0, e0: float = 1e-4) -> Workload:
    """Section IV-B in 1-D: conductor (sigma) for z >= nz/4, plane wave E_x = e0 sin(2 pi t / T),
    B_y = E_x / C imposed at z = 0 with period T = 1.25 nz."""
    z = np.arange(nz)
    sig = np.where(z >= nz // 4, float(sigma), 0.0)
    period = 1.25 * nz
    c = LIGHT_SPEED[model]
    src = Source("impose", np.array([0], dtype=np.int64), TimeFunction("sin", 1.0, period, 0.0),
                 E0=(e0, 0.0, 0.0), B0=(0.0, e0 / c, 0.0))
    return Workload("skin_effect_1d", model, (1, 1, nz), int(periods * period), sigma=sig, sources=[src])


# Mesh-refinement sizes of the batched skin-effect sweep: N = 16 k for k = 2 .. 17 (32 ... 272).
REFINEMENT_SIZES = tuple(16 * k for k in range(2, 18))


def skin_effect_3d(model: str, n: int, sigma: float, e0: float = 1e-4) -> Workload:
    """Section IV-B on an n^3 lattice: conductor (sigma) for z >= n/4, plane wave E_x = e0 sin(2 pi t /
    T), B_y = E_x / C imposed on the whole z = 0 plane, T = 1.25 n, 10 n steps. Media and source are
    uniform in x and y, so every (x, y) column evolves like the 1 x 1 x n lattice."""
    cells_per_plane = n * n
    z = np.repeat(np.arange(n), cells_per_plane)
    sig = np.where(z >= n // 4, float(sigma), 0.0)
    period = 1.25 * n
    c = LIGHT_SPEED[model]
    src = Source("impose", np.arange(cells_per_plane, dtype=np.int64), TimeFunction("sin", 1.0, period, 0.0),
                 E0=(e0, 0.0, 0.0), B0=(0.0, e0 / c, 0.0))
    return Workload("skin_effect_3d", model, (n, n, n), 10 * n, sigma=sig, sources=[src])


def refinement_batch(model: str, sigma: float, sizes=REFINEMENT_SIZES) -> list:
    """The batched skin-effect refinement sweep: one ``skin_effect_3d`` lattice per size."""
    return [skin_effect_3d(model, n, sigma) for n in sizes]


def random_medium_dipole(model: str, n: int = 128, seed: int = 5, period: float = 24.0, j0: float = 1e-4,
                         steps: int = 1000, r2_max: float = 36.0) -> Workload:
    """Dipole (as ``hertz_dipole``, period 24) in an n^3 lattice whose eps_r is uniform in [1, 4) per
    cell from numpy's default_rng(seed)."""
    rng = np.random.default_rng(seed)
    eps = rng.uniform(1.0, 4.0, n * n * n)
    w = hertz_dipole(model, n, period, j0, steps, r2_max=r2_max)
    w.name = "random_medium_dipole"
    w.eps_r = eps
    return w


def random_state(model: str, shape, seed: int, media: str = "random", n_sources: int = 2,
                 amplitude: float = 1.0):
    """Random test case for element-wise parity: random populations (q, n) in canonical order,
    random media (``media`` = ``random`` | ``vacuum`` | ``few`` materials), and random current and
    imposed sources on a few cells. Returns (Workload, populations)."""
    nx, ny, nz = shape
    n = nx * ny * nz
    rng = np.random.default_rng(seed)
    q = POPULATIONS[model]
    f = amplitude * rng.standard_normal((q, n))
    eps = mu = sig = None
    if media == "random":
        eps = rng.uniform(1.0, 4.0, n)
        mu = rng.uniform(1.0, 2.0, n)
        sig = rng.uniform(0.0, 0.5, n) * (rng.random(n) < 0.5)
    elif media == "few":
        table = rng.uniform(1.0, 4.0, (5, 3))
        table[:, 2] = [0.0, 0.0, 0.1, 0.3, 1.0]
        ids = rng.integers(0, 5, n)
        eps, mu, sig = table[ids, 0], table[ids, 1] * 0.5 + 0.5, table[ids, 2]
    sources = []
    for k in range(n_sources):
        m = max(1, min(n // 7, 5))
        cells = np.sort(rng.choice(n, size=m, replace=False)).astype(np.int64)
        if k % 2 == 0:
            fn = TimeFunction("sin", rng.uniform(0.5, 2.0), rng.uniform(5.0, 40.0), rng.uniform(0, 6.28))
            sources.append(Source("current", cells, fn, w=rng.standard_normal((m, 3))))
        else:
            fn = TimeFunction("sin", rng.uniform(0.5, 2.0), rng.uniform(5.0, 40.0), rng.uniform(0, 6.28))
            sources.append(Source("impose", cells, fn, E0=tuple(rng.standard_normal(3)),
                                  B0=tuple(rng.standard_normal(3))))
    w = Workload("random_state", model, (nx, ny, nz), 0, eps_r=eps, mu_r=mu, sigma=sig, sources=sources)
    return w, f


def slab_case(model: str, shape, seed: int, media: str = "random", amplitude: float = 1.0):
    """``random_state`` plus sources on two z-columns, so that every plane, and so every slab's
    boundary planes, holds source cells: a current on the column (1, 2, z) for all z, and imposed
    fields on (nx - 2, ny - 1, z) for every third z. Returns (Workload, populations)."""
    nx, ny, nz = shape
    w, f = random_state(model, shape, seed, media=media, amplitude=amplitude)
    rng = np.random.default_rng(seed + 1000)
    z = np.arange(nz, dtype=np.int64)
    col = (1 % nx) + nx * ((2 % ny) + ny * z)
    w.sources.append(Source("current", col, TimeFunction("sin", 1.0, 13.0, 0.7), w=rng.standard_normal((nz, 3))))
    zi = z[::3]
    imp = ((nx - 2) % nx) + nx * ((ny - 1) + ny * zi)
    w.sources.append(Source("impose", imp, TimeFunction("sin", 0.8, 17.0, 0.2), E0=tuple(rng.standard_normal(3)),
                            B0=tuple(rng.standard_normal(3))))
    return w, f
