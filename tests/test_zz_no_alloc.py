"""lbm_reduce_noalloc: the reduction entry point for callers that cannot allocate device memory
(their memory belongs to a pool of their own, or their loop cannot take cudaMalloc's implicit
synchronisation). It keeps its partial sums in a static device array instead of a buffer that
lbm_reduce allocates. Checked through the C ABI against lbm_reduce, on two calls in a row, with host
and device outputs, and for the clear error past its size limit.

This file is collected last on purpose; it must pass alone in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest

from paper_2309_08068_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

TOL = 1e-5  # the parity tests' relative tolerance


def _noalloc(lib):
    fn = lib.lbm_reduce_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    return fn


def _close(a, b):
    return all(abs(x - y) <= TOL * max(abs(y), 1e-300) for x, y in zip(a, b))


@pytest.mark.parametrize("model", ["mm", "hv"])
def test_noalloc_matches_reduce_on_consecutive_calls(model):
    from paper_2309_08068_gb300 import build
    from paper_2309_08068_gb300.lbm import lattice_from_workload
    build.build()
    w = wl.hertz_dipole(model, n=40, period=10.0)
    rng = np.random.default_rng(3)
    w.E = rng.standard_normal((3, w.n)) * 1e-4
    w.B = rng.standard_normal((3, w.n)) * 1e-4
    L = lattice_from_workload(w, track_rho=model == "mm")
    fn = _noalloc(L.lib)
    dev_out = torch.zeros(3, dtype=torch.float64, device="cuda")
    for _ in range(2):
        L.step(3)
        ref = L.reduce()
        host = (ctypes.c_double * 3)()
        assert fn(L.h, host, 0) == 0, L.lib.lbm_last_error(L.h)
        assert _close(list(host), ref), (list(host), ref)
        assert fn(L.h, dev_out.data_ptr(), 1) == 0, L.lib.lbm_last_error(L.h)
        L.sync()
        assert _close(dev_out.cpu().tolist(), ref), (dev_out.cpu().tolist(), ref)


def test_noalloc_rejects_more_source_cells_than_its_scratch_holds():
    from paper_2309_08068_gb300 import build
    from paper_2309_08068_gb300.lbm import Lattice
    build.build()
    n = 100
    L = Lattice("hv", (n, n, n))
    L.init_fields(np.zeros((3, n ** 3), np.float32), np.zeros((3, n ** 3), np.float32))
    cells = np.arange(0, 900_000, dtype=np.int64)
    L.add_source(wl.Source("current", cells, wl.TimeFunction("const", 1.0), w=np.zeros((cells.size, 3))))
    fn = _noalloc(L.lib)
    host = (ctypes.c_double * 3)()
    assert fn(L.h, host, 0) == -1
    msg = L.lib.lbm_last_error(L.h).decode()
    assert "static scratch holds 4096" in msg
    assert np.isfinite(L.reduce()[0])  # lbm_reduce, which allocates, still works there
