"""24-bit population storage (LBM_F24: an FP16 value plus a signed correction byte; FP32 arithmetic).

The encoding is integer and rounding work, so the round trip through the library must equal, bit
for bit, the encoding as the tests write it out from its definition (helpers.f24_value: h = x cut
toward zero to FP16, the remainder in 256ths of ulp(h) rounded to nearest, a count of 256 carried into
h).

Against the FP64 oracle the tolerance follows the arithmetic as for 16-bit storage: each step rounds
every stored population once with relative error at most u = 2^-19 (normal h), the errors are
independent and not amplified, so after T steps the relative L2 error is about u sqrt((T + 1) / 3);
the element-wise tests allow 3 u sqrt(T + 1) plus FP32's own 1e-6.
"""
import numpy as np
import pytest

from helpers import f24_value, rel_l2
from paper_2309_08068_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

U24 = 2.0 ** -19


@pytest.mark.parametrize("model", ["mm", "hv"])
@pytest.mark.parametrize("scale", [1.0, 2.0 ** 10])
def test_f24_round_trip_is_the_definition(model, scale):
    """set_populations then get_populations stores and decodes every value exactly as defined:
    values across FP16's range at both scales, FP16 subnormals and below, zeros, ties, carries into
    the half (across a binade too) and a value beyond FP16's range."""
    from paper_2309_08068_gb300.lbm import Lattice
    rng = np.random.default_rng(11)
    shape = (13, 7, 5)
    n = int(np.prod(shape))
    q = 48 if model == "mm" else 36
    mag = np.exp2(rng.uniform(-30, 14, (q, n)))
    f = np.float32(mag * rng.choice([-1.0, 1.0], (q, n)))
    f[0, :8] = 0.0
    f[1, :8] = np.float32([1 + 3 * 2.0 ** -19, 1 + 2.0 ** -11, 2 - 2.0 ** -22, 1 + 2.0 ** -20,
                           -(1 + 3 * 2.0 ** -19), 6.1e-5, 2.0 ** -24, 65500.0])
    f[2, :6] = np.float32([1 + 2.0 ** -10 - 2.0 ** -20, -(2 - 2.0 ** -22), 5 * 2.0 ** -32, -5 * 2.0 ** -32,
                           -0.0, 1e6])
    f /= np.float32(scale)
    full = np.zeros((50 if model == "mm" else 36, n), np.float32)
    full[:q] = f
    L = Lattice(model, shape, storage="f24", storage_scale=scale)
    L.set_populations(full, 0)
    got = L.populations_host()[:q]
    L.close()
    want = f24_value(f, scale)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


@pytest.mark.parametrize("model", ["mm", "hv"])
@pytest.mark.parametrize("media", ["vacuum", "few", "random"])
def test_random_state_f24(model, media):
    from test_storage16_gpu import pair16
    w, f = wl.random_state(model, (9, 7, 5), seed=31, media=media)
    G, O = pair16(w, "f24", 1.0, pops=f, t0=2)
    q = 48 if model == "mm" else 36
    for steps, total in ((1, 1), (4, 5)):
        G.step(steps)
        O.step(steps)
        tol = 3 * U24 * np.sqrt(total + 1) + 1e-6
        assert rel_l2(G.populations_host()[:q], O.populations()[:q]) <= tol
        g, o = G.fields_host("EB"), O.fields()
        for c in "EB":
            assert rel_l2(g[c], o[c]) <= tol, (c, rel_l2(g[c], o[c]), tol)


@pytest.mark.parametrize("model", ["mm", "hv"])
def test_dielectric_pulse_1500_steps_f24(model):
    """Section IV-A pulse, 1500 steps, scale 2^20 as the bench uses: the stated 24-bit error."""
    from test_storage16_gpu import pair16
    w = wl.dielectric_pulse_1d(model)
    G, O = pair16(w, "f24", 2.0 ** 20)
    G.step(w.steps)
    O.step(w.steps)
    g, o = G.fields_host("EB"), O.fields()
    errs = {c: rel_l2(g[c], o[c]) for c in "EB"}
    print(f"dielectric pulse {model} f24: rel L2 {errs}")
    assert max(errs.values()) <= 1e-3


@pytest.mark.parametrize("model", ["mm", "hv"])
def test_f24_steps_singly_and_batches_bit_for_bit(model):
    """No two-step pass takes 24-bit storage, in any mode; a batch of 24-bit lattices (sources,
    uneven step counts, graph replay) equals each lattice's own lbm_step bit for bit."""
    from paper_2309_08068_gb300.lbm import Batch, Lattice, LbmError, lattice_from_workload
    for mode in (1, 2, 3):
        L = Lattice(model, (256, 256, 16), storage="f24")
        L.set_step_fusion(mode)
        assert L.pass_kind is None
        L.close()
    with pytest.raises(LbmError):
        Lattice(model, (16, 16, 8), storage="f24", z_ghost=True)
    stream = torch.cuda.Stream()
    steps = [5, 2, 4]

    def lattices():
        out = []
        for shape, seed in (((40, 24, 12), 180), ((7, 5, 3), 181), ((33, 9, 4), 182)):
            w, f = wl.slab_case(model, shape, seed=seed, media="few")
            L = lattice_from_workload(w, init=False, stream=stream, storage="f24", storage_scale=2.0 ** 4)
            L.set_populations(np.asarray(f, np.float32), 1)
            out.append(L)
        return out

    solo, grouped = lattices(), lattices()
    batch = Batch(grouped)
    for rep in range(2):
        for L, k in zip(solo, steps):
            L.step(k)
        batch.step(steps)
        for A, B in zip(solo, grouped):
            assert A.time == B.time
            assert np.array_equal(A.populations_host(), B.populations_host()), rep


@pytest.mark.parametrize("model", ["mm", "hv"])
def test_f24_fields_and_reductions_equal_fp32_on_representable_values(model):
    """A 24-bit lattice and an FP32 lattice holding the same values (values the 24-bit storage keeps
    exactly) decode to the same populations, so every field, lbm_reduce and lbm_reduce_noalloc must
    agree bit for bit; sources and per-cell media included."""
    import ctypes
    from paper_2309_08068_gb300.lbm import lattice_from_workload
    w, f = wl.slab_case(model, (20, 12, 9), seed=190, media="random")
    q = 48 if model == "mm" else 36
    scale = 2.0 ** 6
    f = np.asarray(f, np.float32)
    f[:q] = f24_value(f[:q], scale)
    lat = {}
    for storage in ("f32", "f24"):
        L = lattice_from_workload(w, init=False, storage=storage, storage_scale=scale if storage == "f24" else 0.0)
        L.set_populations(f, 4)
        lat[storage] = L
    assert np.array_equal(lat["f32"].populations_host()[:q], lat["f24"].populations_host()[:q])
    a, b = lat["f32"].fields_host("EBDHJ"), lat["f24"].fields_host("EBDHJ")
    for c in "EBDHJ":
        assert np.array_equal(a[c], b[c]), c
    assert lat["f32"].reduce() == lat["f24"].reduce()
    fn = lat["f32"].lib.lbm_reduce_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    outs = []
    for storage in ("f32", "f24"):
        host = (ctypes.c_double * 3)()
        assert fn(lat[storage].h, host, 0) == 0
        outs.append(tuple(host))
    assert outs[0] == outs[1]
    for L in lat.values():
        L.close()
