"""FP64 CPU oracle for the MM and modified-HV lattice-Boltzmann Maxwell schemes (arXiv 2309.08068).

TEST INFRASTRUCTURE. Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The GPU library never calls it, and the two share no code:
the oracle is ``lbm_oracle.c`` (plain loops, double precision, the paper's order of steps), loaded
here with ctypes.

Arrays crossing this wrapper are float64, cell index ``x + nx * (y + ny * z)`` (x fastest), and
vector fields are component-major ``(3, n)``. Populations use the canonical index documented in
``lbm_oracle.c``: MM ``k = r*24 + p*8 + (i-1)*2 + j`` plus the rest populations 48, 49; HV
``k = r*18 + (i-1)*3 + c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liblbm_oracle.so")

MM, HV = 0, 1
FN_SIN, FN_TABLE, FN_CONST = 0, 1, 2
SRC_CURRENT, SRC_IMPOSE = 0, 1
Q = {MM: 50, HV: 36}
FIELD_NAMES = ("E", "B", "D", "H", "J")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add contraction, so x86 and Arm agree)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    D = ctypes.POINTER(ctypes.c_double)
    I64 = ctypes.c_int64
    lib.or_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, D, D, D, ctypes.c_double,
                              ctypes.c_double, ctypes.POINTER(P)]
    lib.or_create.restype = ctypes.c_int
    lib.or_destroy.argtypes = [P]
    lib.or_set_threads.argtypes = [P, ctypes.c_int]
    lib.or_max_threads.restype = ctypes.c_int
    lib.or_time.argtypes = [P]
    lib.or_time.restype = I64
    lib.or_eps0.argtypes = [P]
    lib.or_eps0.restype = ctypes.c_double
    lib.or_mu0.argtypes = [P]
    lib.or_mu0.restype = ctypes.c_double
    lib.or_clear_sources.argtypes = [P]
    lib.or_add_source.argtypes = [P, ctypes.c_int, I64, ctypes.POINTER(I64), D, D, D, ctypes.c_int, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, D, I64]
    lib.or_add_source.restype = ctypes.c_int
    lib.or_init_fields.argtypes = [P, D, D]
    lib.or_step.argtypes = [P, I64]
    lib.or_fields.argtypes = [P, D]
    lib.or_charge.argtypes = [P, D]
    lib.or_get_populations.argtypes = [P, D]
    lib.or_set_populations.argtypes = [P, D, I64]
    lib.or_tables.argtypes = [P, D, D, D]
    lib.or_adjoint_step.argtypes = [P, I64, D, D, D, D, D]
    lib.or_plane_loss.argtypes = [P, I64, D, ctypes.c_int, ctypes.c_int, D, D, D]
    lib.or_plane_loss.restype = ctypes.c_double
    _lib = lib
    return lib


def _dptr(a: np.ndarray | None):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, shape=None) -> np.ndarray:
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        arr = arr.reshape(shape)
    return arr


@dataclass
class TimeFn:
    """Source time dependence s(t): ``sin``: amp sin(2 pi t / period + phase); ``table``: amp table[t]
    (0 outside the table); ``const``: amp."""
    kind: str = "sin"
    amplitude: float = 1.0
    period: float = 1.0
    phase: float = 0.0
    table: np.ndarray | None = None


class OracleLattice:
    """One periodic lattice of the FP64 oracle. ``model`` is ``"mm"`` or ``"hv"``."""

    def __init__(self, model: str, shape, eps_r=None, mu_r=None, sigma=None, eps0: float = 0.0, mu0: float = 0.0,
                 threads: int = 1):
        self.lib = _load()
        self.model = {"mm": MM, "hv": HV}[model]
        nx, ny, nz = (int(s) for s in shape)
        self.shape = (nx, ny, nz)
        self.n = nx * ny * nz
        self.q = Q[self.model]
        media = [None if m is None else _f64(m).reshape(-1) for m in (eps_r, mu_r, sigma)]
        for m in media:
            if m is not None and m.size != self.n:
                raise ValueError("media arrays must have one value per cell")
        self._media = media
        h = ctypes.c_void_p()
        rc = self.lib.or_create(self.model, nx, ny, nz, *(_dptr(m) for m in media), float(eps0), float(mu0),
                                ctypes.byref(h))
        if rc != 0:
            raise RuntimeError(f"or_create failed ({rc})")
        self.h = h
        self.lib.or_set_threads(self.h, int(threads))

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            self.lib.or_destroy(h)
            self.h = None

    @property
    def time(self) -> int:
        return int(self.lib.or_time(self.h))

    @property
    def eps0(self) -> float:
        return float(self.lib.or_eps0(self.h))

    @property
    def mu0(self) -> float:
        return float(self.lib.or_mu0(self.h))

    def set_threads(self, threads: int) -> None:
        self.lib.or_set_threads(self.h, int(threads))

    def _add(self, kind, cells, w, E0, B0, fn: TimeFn):
        cells = np.ascontiguousarray(np.asarray(cells, dtype=np.int64).reshape(-1))
        fk = {"sin": FN_SIN, "table": FN_TABLE, "const": FN_CONST}[fn.kind]
        table = None if fn.table is None else _f64(fn.table).reshape(-1)
        w = None if w is None else _f64(w).reshape(-1)
        E0 = None if E0 is None else _f64(E0).reshape(3)
        B0 = None if B0 is None else _f64(B0).reshape(3)
        rc = self.lib.or_add_source(self.h, kind, cells.size, cells.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                    _dptr(w), _dptr(E0), _dptr(B0), fk, float(fn.amplitude), float(fn.period),
                                    float(fn.phase), _dptr(table), 0 if table is None else table.size)
        if rc != 0:
            raise ValueError(f"or_add_source rejected the source ({rc})")

    def add_current(self, cells, w, fn: TimeFn) -> None:
        """J_ext(x, t) += w(x) s(t) at the listed cells; w is (n_cells, 3)."""
        self._add(SRC_CURRENT, cells, w, None, None, fn)

    def add_impose(self, cells, E0, B0, fn: TimeFn) -> None:
        """After each collision, the listed cells are set to f_eq(E0 s(t), B0 s(t), J = 0)."""
        self._add(SRC_IMPOSE, cells, None, E0, B0, fn)

    def clear_sources(self) -> None:
        self.lib.or_clear_sources(self.h)

    def init_fields(self, E, B) -> None:
        E = _f64(E, (3, self.n))
        B = _f64(B, (3, self.n))
        self.lib.or_init_fields(self.h, _dptr(E), _dptr(B))

    def step(self, n: int = 1) -> None:
        self.lib.or_step(self.h, int(n))

    def fields(self) -> dict:
        out = np.empty((15, self.n), dtype=np.float64)
        self.lib.or_fields(self.h, _dptr(out))
        return {name: out[3 * i:3 * i + 3] for i, name in enumerate(FIELD_NAMES)}

    def charge(self) -> np.ndarray:
        out = np.empty(self.n, dtype=np.float64)
        self.lib.or_charge(self.h, _dptr(out))
        return out

    def populations(self) -> np.ndarray:
        out = np.empty((self.q, self.n), dtype=np.float64)
        self.lib.or_get_populations(self.h, _dptr(out))
        return out

    def set_populations(self, f, t: int = 0) -> None:
        f = _f64(f, (self.q, self.n))
        self.lib.or_set_populations(self.h, _dptr(f), int(t))

    def adjoint_step(self, iteration: int, g_next, f_n, grad_eps_r=None, grad_sigma=None):
        """dL/df^n from dL/df^{n+1} through forward iteration `iteration` (sources s(iteration)),
        adding dL/d eps_r and dL/d sigma into the given float64 arrays (n values each)."""
        g_next = _f64(g_next, (self.q, self.n))
        f_n = _f64(f_n, (self.q, self.n))
        out = np.empty((self.q, self.n), dtype=np.float64)
        self.lib.or_adjoint_step(self.h, int(iteration), _dptr(g_next), _dptr(f_n), _dptr(out), _dptr(grad_eps_r),
                                 _dptr(grad_sigma))
        return out

    def plane_loss(self, t: int, f_t, axis: int, index: int, g=None, grad_eps_r=None, grad_sigma=None) -> float:
        """sum over the plane cells of |E(f_t)|^2 at time t; adds its derivatives when arrays are given."""
        f_t = _f64(f_t, (self.q, self.n))
        return float(self.lib.or_plane_loss(self.h, int(t), _dptr(f_t), int(axis), int(index), _dptr(g),
                                            _dptr(grad_eps_r), _dptr(grad_sigma)))

    def loss_and_gradient(self, steps: int, axis: int, index: int):
        """From the current state: run `steps` steps, return L = sum_{t=1..steps} plane_loss(t) and
        dL/d eps_r, dL/d sigma by the adjoint recursion (all states kept; small lattices only)."""
        t0 = self.time
        states = [self.populations()]
        for _ in range(steps):
            self.step(1)
            states.append(self.populations())
        ge = np.zeros(self.n)
        gs = np.zeros(self.n)
        g = np.zeros((self.q, self.n))
        loss = self.plane_loss(t0 + steps, states[steps], axis, index, g, ge, gs)
        for k in range(steps - 1, -1, -1):
            g = self.adjoint_step(t0 + k + 1, g, states[k], ge, gs)
            if k >= 1:
                loss += self.plane_loss(t0 + k, states[k], axis, index, g, ge, gs)
        return loss, ge, gs

    def tables(self):
        v = np.zeros((12, 3))
        e = np.zeros((24, 3))
        b = np.zeros((24, 3))
        self.lib.or_tables(self.h, _dptr(v), _dptr(e), _dptr(b))
        if self.model == HV:
            return v[:6].copy()
        return v, e, b


def max_threads() -> int:
    return int(_load().or_max_threads())
