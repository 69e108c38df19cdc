"""lbm_reduce_noalloc: the reduction entry point for callers that cannot allocate device memory
(their memory belongs to a pool of their own, or their loop cannot take cudaMalloc's implicit
synchronisation). It keeps its partial sums in a static device array instead of a buffer that
lbm_reduce allocates. Checked through the C ABI against lbm_reduce, on two calls in a row, with host
and device outputs; for the clear error past its size limit (MM only); for free device memory left
unchanged; and for the report of a stopped two-step pass.

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


def _with_current_cells(model, n, n_cells):
    from paper_2309_08068_gb300.lbm import Lattice
    L = Lattice(model, (n, n, n))
    L.init_fields(np.zeros((3, n ** 3), np.float32), np.zeros((3, n ** 3), np.float32))
    cells = np.arange(0, n_cells, dtype=np.int64)
    L.add_source(wl.Source("current", cells, wl.TimeFunction("const", 1.0), w=np.full((cells.size, 3), 1e-6)))
    return L


def test_noalloc_rejects_more_mm_source_cells_than_its_scratch_holds():
    """MM keeps one partial sum per 256 source cells (its energy correction at source cells): 900,000
    source cells on a 100^3 lattice need more slots than the static array has, and the call says
    so instead of writing past it. lbm_reduce, which allocates, still works there."""
    from paper_2309_08068_gb300 import build
    build.build()
    L = _with_current_cells("mm", 100, 900_000)
    fn = _noalloc(L.lib)
    host = (ctypes.c_double * 3)()
    assert fn(L.h, host, 0) == -1
    msg = L.lib.lbm_last_error(L.h).decode()
    assert "static scratch holds 4096" in msg
    assert np.isfinite(L.reduce()[0])


def test_noalloc_takes_hv_lattices_with_many_source_cells():
    """HV's reduction has no per-source-cell partial sums, so the same 900,000 source cells fit and
    the result equals lbm_reduce's."""
    from paper_2309_08068_gb300 import build
    build.build()
    L = _with_current_cells("hv", 100, 900_000)
    L.step(2)
    fn = _noalloc(L.lib)
    host = (ctypes.c_double * 3)()
    assert fn(L.h, host, 0) == 0, L.lib.lbm_last_error(L.h)
    ref = L.reduce()
    assert ref[0] > 0
    assert _close(list(host), ref), (list(host), ref)


def test_noalloc_leaves_free_device_memory_unchanged_on_a_fresh_context():
    """The call allocates nothing: on a context that has never reduced (no partial-sum buffer yet),
    the device's free memory is the same before and after it. The library's module is loaded first
    by a call on another context, so its static array already exists."""
    from paper_2309_08068_gb300 import build
    from paper_2309_08068_gb300.lbm import Lattice
    build.build()
    n = 64
    warm = Lattice("mm", (n, n, n))
    warm.init_fields(np.zeros((3, n ** 3), np.float32), np.zeros((3, n ** 3), np.float32))
    fn = _noalloc(warm.lib)
    host = (ctypes.c_double * 3)()
    assert fn(warm.h, host, 0) == 0
    L = Lattice("hv", (n, n, n))
    rng = np.random.default_rng(5)
    L.init_fields(rng.standard_normal((3, n ** 3)).astype(np.float32), np.zeros((3, n ** 3), np.float32))
    L.sync()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert fn(L.h, host, 0) == 0, L.lib.lbm_last_error(L.h)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert host[0] > 0


def test_noalloc_reports_a_stopped_two_step_pass():
    """With host output the call first reports a two-step pass whose dependency wait ran out
    (LBM_ETIMEDOUT, as lbm_reduce does), rather than sums over undefined populations."""
    from paper_2309_08068_gb300 import build
    from paper_2309_08068_gb300.lbm import lattice_from_workload
    build.build()
    w, f = wl.slab_case("hv", (256, 160, 6), seed=142)
    L = lattice_from_workload(w, init=False)
    L.set_step_fusion(2)
    assert L.step_fusion_active
    L.set_populations(np.asarray(f, np.float32), 0)
    L.set_wait_limit(-1)
    L.step(2)
    fn = _noalloc(L.lib)
    host = (ctypes.c_double * 3)()
    assert fn(L.h, host, 0) == -5
    assert "two-step pass" in L.lib.lbm_last_error(L.h).decode()
    L.set_wait_limit(0)
    L.set_populations(np.asarray(f, np.float32), 0)
    L.step(2)
    assert fn(L.h, host, 0) == 0
    ref = L.reduce()
    assert _close(list(host), ref), (list(host), ref)
