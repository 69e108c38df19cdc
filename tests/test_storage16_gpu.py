"""16-bit population storage (BF16 / FP16 with a power-of-two scale; FP32 arithmetic) against the
FP64 oracle.

Tolerance derived from the arithmetic. Each step rounds every stored population once to the format's
precision: unit roundoff u = 2^-8 for BF16 and 2^-11 for FP16. The rounding errors are independent
and the step does not amplify them. After T steps, plus the rounding of the initial state, the
relative L2 error is therefore about u * sqrt((T + 1) / 3). The element-wise tests allow 3 * u *
sqrt(T + 1). The long 1500-step pulse records its error and guards it with a loose bound (measured
on GB300: 2-3 % for FP16, 10-21 % for BF16).
"""
import numpy as np
import pytest

from helpers import rel_l2
from paper_2309_08068_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

UNIT_ROUNDOFF = {"bf16": 2.0 ** -8, "f16": 2.0 ** -11}


def pair16(w, storage, scale, pops=None, t0=0, threads=4):
    from paper_2309_08068_gb300.lbm import lattice_from_workload
    from test_parity_gpu import rounded
    from helpers import oracle_from_workload
    w = rounded(w)
    G = lattice_from_workload(w, init=pops is None, storage=storage, storage_scale=scale)
    O = oracle_from_workload(w, threads=threads, init=pops is None)
    if pops is not None:
        p32 = np.asarray(pops, np.float32)
        G.set_populations(p32, t0)
        O.set_populations(p32.astype(np.float64), t0)
    return G, O


@pytest.mark.parametrize("model", ["mm", "hv"])
@pytest.mark.parametrize("storage", ["bf16", "f16"])
@pytest.mark.parametrize("media", ["vacuum", "few", "random"])
def test_random_state_16bit(model, storage, media):
    w, f = wl.random_state(model, (9, 7, 5), seed=31, media=media)
    G, O = pair16(w, storage, 1.0, pops=f, t0=2)
    u = UNIT_ROUNDOFF[storage]
    for steps, total in ((1, 1), (4, 5)):
        G.step(steps)
        O.step(steps)
        tol = 3 * u * np.sqrt(total + 1)
        gp, op = G.populations_host(), O.populations()
        q = 48 if model == "mm" else 36  # MM rest populations are not stored without track_rho
        assert rel_l2(gp[:q], op[:q]) <= tol
        g, o = G.fields_host("EB"), O.fields()
        for c in "EB":
            assert rel_l2(g[c], o[c]) <= tol, (c, rel_l2(g[c], o[c]), tol)


def test_f16_scale_is_exact_and_keeps_small_values_normal():
    """The same state stored with scales 1 and 2^20: with amplitude 1e-5 populations sit below FP16's
    smallest normal at scale 1, so 2^20 must be far more accurate; with O(1) data both agree."""
    w, f = wl.random_state("hv", (6, 5, 4), seed=32, media="vacuum", n_sources=0)
    errs = {}
    for scale in (1.0, 2.0 ** 20):
        G, O = pair16(w, "f16", scale, pops=1e-5 * f, t0=0)
        G.step(3)
        O.step(3)
        errs[scale] = rel_l2(G.populations_host(), O.populations())
    assert errs[2.0 ** 20] <= 3 * UNIT_ROUNDOFF["f16"] * 2
    assert errs[1.0] > 5 * errs[2.0 ** 20]


@pytest.mark.parametrize("model", ["mm", "hv"])
@pytest.mark.parametrize("storage,scale,bound", [("bf16", 1.0, 0.5), ("f16", 2.0 ** 20, 0.05)])
def test_dielectric_pulse_1500_steps_16bit(model, storage, scale, bound):
    """Section IV-A pulse, 1500 steps: the stated 16-bit storage error against the FP64 oracle."""
    w = wl.dielectric_pulse_1d(model)
    G, O = pair16(w, storage, scale)
    G.step(w.steps)
    O.step(w.steps)
    g, o = G.fields_host("EB"), O.fields()
    errs = {c: rel_l2(g[c], o[c]) for c in "EB"}
    print(f"dielectric pulse {model} {storage}: rel L2 {errs}")
    assert max(errs.values()) <= bound
