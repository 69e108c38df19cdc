"""GPU adjoint (lbm_adjoint): loss and dL/d eps_r, dL/d sigma against the FP64 oracle's adjoint and
its central finite differences.

Tolerance from the arithmetic. The loss is the FP32 forward path, so relative error is at most 1e-5.
The gradients add one FP32 rounding per backward step and per term to that path's error. Over T <= 100
steps they stay well inside 1e-4 relative L2, and the tests require that.
"""
import numpy as np
import pytest

from helpers import oracle_from_workload, rel_l2
from paper_2309_08068_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

GRAD_TOL = 1e-4
LOSS_TOL = 1e-5


def f32(a):
    return None if a is None else np.asarray(a, np.float32).astype(np.float64)


def small_case(model, seed=81, shape=(8, 7, 6), plane=(0, 5)):
    """Per-cell eps_r and sigma, a current source and an imposed source away from the plane."""
    rng = np.random.default_rng(seed)
    n = int(np.prod(shape))
    nx, ny, nz = shape
    eps = f32(rng.uniform(1.0, 3.0, n))
    sig = f32(rng.uniform(0.0, 0.3, n) * (rng.random(n) < 0.5))
    cur = np.array([2 + nx * (3 + ny * 2), 1 + nx * (4 + ny * 3)], dtype=np.int64)
    imp = np.array([3 + nx * (1 + ny * 4)], dtype=np.int64)
    sources = [wl.Source("current", cur, wl.TimeFunction("sin", 1.0, 9.0, 0.4), w=f32(rng.standard_normal((2, 3)))),
               wl.Source("impose", imp, wl.TimeFunction("sin", 0.5, 11.0, 0.1),
                         E0=tuple(f32(rng.standard_normal(3))), B0=tuple(f32(rng.standard_normal(3))))]
    f0 = f32(0.1 * rng.standard_normal((wl.POPULATIONS[model], n)))
    w = wl.Workload("adj", model, shape, 0, eps_r=eps, sigma=sig, sources=sources)
    return w, f0, plane


def gpu_adjoint(w, f0, steps, plane, interval=0, t0=3):
    from paper_2309_08068_gb300.lbm import lattice_from_workload
    L = lattice_from_workload(w, init=False)
    L.set_populations(np.asarray(f0, np.float32), t0)
    loss, ge, gs = L.adjoint(steps, plane[0], plane[1], interval)
    return L, loss, ge.cpu().numpy(), gs.cpu().numpy()


@pytest.mark.parametrize("model", ["mm", "hv"])
def test_adjoint_matches_oracle_adjoint(model):
    w, f0, plane = small_case(model)
    steps = 20
    L, loss, ge, gs = gpu_adjoint(w, f0, steps, plane, interval=6)  # segments 2, 6, 6 and the final 6
    O = oracle_from_workload(w, init=False, threads=8)
    O.set_populations(f0, 3)
    loss_ref, ge_ref, gs_ref = O.loss_and_gradient(steps, *plane)
    assert abs(loss - loss_ref) <= LOSS_TOL * loss_ref
    assert rel_l2(ge, ge_ref) <= GRAD_TOL, rel_l2(ge, ge_ref)
    assert rel_l2(gs, gs_ref) <= GRAD_TOL, rel_l2(gs, gs_ref)
    # the context advanced exactly like lbm_step
    assert L.time == 3 + steps
    assert rel_l2(L.populations_host()[:48 if model == "mm" else 36], O.populations()[:48 if model == "mm" else 36]) <= 1e-5
    print(f"adjoint {model}: loss rel {abs(loss - loss_ref) / loss_ref:.2e}, grad eps rel L2 "
          f"{rel_l2(ge, ge_ref):.2e}, grad sigma rel L2 {rel_l2(gs, gs_ref):.2e}")


@pytest.mark.parametrize("model", ["mm", "hv"])
def test_checkpoint_interval_does_not_change_the_result(model):
    """Recomputation replays the same kernels on the same states: every checkpoint interval, and
    keeping every step's record resident (interval -1), gives the same loss and gradients bit for bit."""
    w, f0, plane = small_case(model, seed=82)
    results = [gpu_adjoint(w, f0, 17, plane, interval=k)[1:] for k in (1, 3, 5, 8, 16, 0, 17, 40, -1)]
    for loss, ge, gs in results[1:]:
        assert loss == results[0][0]
        assert np.array_equal(ge, results[0][1])
        assert np.array_equal(gs, results[0][2])


@pytest.mark.parametrize("model", ["mm", "hv"])
def test_autograd_plane_loss(model):
    from paper_2309_08068_gb300.lbm import plane_loss
    w, f0, plane = small_case(model, seed=83)
    eps = torch.tensor(w.eps_r, dtype=torch.float32, device="cuda", requires_grad=True)
    sig = torch.tensor(w.sigma, dtype=torch.float32, device="cuda", requires_grad=True)
    pops = torch.tensor(np.asarray(f0, np.float32), device="cuda")
    loss = plane_loss(model, w.shape, eps, sig, populations=pops, sources=w.sources, steps=12,
                      plane_axis=plane[0], plane_index=plane[1], t0=3)
    (3.0 * loss).backward()
    _, loss2, ge, gs = gpu_adjoint(w, f0, 12, plane)
    assert loss.item() == loss2
    assert np.allclose(eps.grad.cpu().numpy(), 3.0 * ge, rtol=1e-6, atol=0)
    assert np.allclose(sig.grad.cpu().numpy(), 3.0 * gs, rtol=1e-6, atol=0)


@pytest.mark.parametrize("model", ["mm", "hv"])
def test_random_medium_dipole_gradient_16cube(model):
    """The inverse-design check at its stated size: 16^3, per-cell eps_r in [1, 4), dipole at
    (8, 8, 8) with period 24, T = 100 steps, plane x = 12. GPU adjoint against the FP64 oracle adjoint
    over the whole lattice, and against oracle central differences at a few cells. The dipole is
    truncated at radius 3 so that no source cell lies in the plane."""
    w = wl.random_medium_dipole(model, n=16, seed=5, period=24.0, steps=100, r2_max=9.0)
    w.eps_r = f32(w.eps_r)
    for s in w.sources:
        s.w = f32(s.w)
    plane = (0, 12)
    q = wl.POPULATIONS[model]
    f0 = np.zeros((q, w.n))
    _, loss, ge, _ = gpu_adjoint(w, f0, w.steps, plane, t0=0)
    O = oracle_from_workload(w, init=False, threads=8)
    O.set_populations(f0, 0)
    loss_ref, ge_ref, _ = O.loss_and_gradient(w.steps, *plane)
    assert abs(loss - loss_ref) <= LOSS_TOL * loss_ref
    assert rel_l2(ge, ge_ref) <= GRAD_TOL, rel_l2(ge, ge_ref)
    for c in (8 + 16 * (8 + 16 * 8) + 2, 11 + 16 * (3 + 16 * 9), 12 + 16 * (8 + 16 * 8)):
        vals = []
        for sgn in (1, -1):
            eps = w.eps_r.copy()
            h = 1e-5 * eps[c]
            eps[c] += sgn * h
            w2 = wl.Workload(w.name, model, w.shape, 0, eps_r=eps, sources=w.sources)
            O2 = oracle_from_workload(w2, init=False, threads=8)
            O2.set_populations(f0, 0)
            total = 0.0
            for t in range(1, w.steps + 1):
                O2.step(1)
                total += O2.plane_loss(t, O2.populations(), *plane)
            vals.append(total)
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(ge[c] - fd) <= GRAD_TOL * np.abs(ge_ref).max(), (c, ge[c], fd)
    print(f"16^3 dipole {model}: loss {loss:.6e} (oracle {loss_ref:.6e}), grad rel L2 {rel_l2(ge, ge_ref):.2e}")


@pytest.mark.parametrize("model", ["mm", "hv"])
@pytest.mark.parametrize("plane", [(1, 2), (2, 1)])
def test_loss_planes_on_other_axes(model, plane):
    """Planes of constant y and constant z (the loss slots of each orientation), against the oracle."""
    w, f0, _ = small_case(model, seed=85)
    steps = 9
    _, loss, ge, gs = gpu_adjoint(w, f0, steps, plane)
    O = oracle_from_workload(w, init=False, threads=8)
    O.set_populations(f0, 3)
    loss_ref, ge_ref, gs_ref = O.loss_and_gradient(steps, *plane)
    assert abs(loss - loss_ref) <= LOSS_TOL * loss_ref
    assert rel_l2(ge, ge_ref) <= GRAD_TOL, rel_l2(ge, ge_ref)
    assert rel_l2(gs, gs_ref) <= GRAD_TOL, rel_l2(gs, gs_ref)


@pytest.mark.parametrize("model", ["mm", "hv"])
def test_workspace_is_kept_grown_and_released(model):
    from paper_2309_08068_gb300.lbm import lattice_from_workload
    w, f0, plane = small_case(model, seed=86)
    L = lattice_from_workload(w, init=False)

    def run(steps, interval=0):
        L.set_populations(np.asarray(f0, np.float32), 3)
        loss, ge, gs = L.adjoint(steps, *plane, interval)
        return loss, ge.cpu().numpy(), gs.cpu().numpy()

    assert L.adjoint_workspace_bytes == 0
    first = run(10)
    held = L.adjoint_workspace_bytes
    assert held > 0
    again = run(10)
    assert L.adjoint_workspace_bytes == held
    run(30)
    assert L.adjoint_workspace_bytes > held
    L.adjoint_release()
    assert L.adjoint_workspace_bytes == 0
    last = run(10)
    for r in (again, last):
        assert r[0] == first[0]
        assert np.array_equal(r[1], first[1]) and np.array_equal(r[2], first[2])


@pytest.mark.parametrize("model", ["mm", "hv"])
def test_adjoint_refuses_what_it_does_not_support(model):
    """16- and 24-bit storage, a source cell inside the loss plane, a plane index outside the lattice
    and a z-slab context are refused with an error, and the context stays usable."""
    from paper_2309_08068_gb300.lbm import Lattice, LbmError
    shape = (6, 5, 4)
    n = 6 * 5 * 4
    for storage in ("bf16", "f24"):
        L16 = Lattice(model, shape, storage=storage)
        with pytest.raises(LbmError):
            L16.adjoint(3, 0, 2)
        L16.close()
    L = Lattice(model, shape)
    src = wl.Source("current", np.array([2 + 6 * (1 + 5 * 1)]), wl.TimeFunction("const", 1.0), w=np.ones((1, 3)))
    L.add_source(src)  # cell (2, 1, 1): in the plane x = 2
    with pytest.raises(LbmError):
        L.adjoint(3, 0, 2)
    for axis, index in ((0, 6), (1, -1), (3, 0)):
        with pytest.raises(LbmError):
            L.adjoint(3, axis, index)
    loss, ge, gs = L.adjoint(3, 0, 4)  # a plane without sources still works
    assert np.isfinite(loss) and ge.shape == (n,) and bool(torch.isfinite(ge).all())
    L.close()
    S = Lattice(model, (6, 5, 5), z_ghost=True)
    with pytest.raises(LbmError):
        S.adjoint(3, 0, 2)
    S.close()


@pytest.mark.parametrize("model", ["mm", "hv"])
def test_sqrt_interval_stays_within_the_classic_sqrt_layout(model):
    """The checkpointed mode's segment length is the longest whose work space does not exceed that
    of segments of ceil(sqrt(T)) steps (the classic sqrt(T) layout): at least ceil(sqrt(T)), a work
    space no larger than the classic layout's, one step longer already over it, and the same result
    bit for bit."""
    from paper_2309_08068_gb300.lbm import lattice_from_workload
    w, f0, plane = small_case(model, seed=88)
    steps = 400  # long enough that keeping every record costs more than the classic layout
    k0 = 20
    L = lattice_from_workload(w, init=False)
    K = L.sqrt_interval(steps)
    assert k0 <= K < steps
    held = {}
    results = {}
    for k in (k0, K, K + 1):
        L.adjoint_release()
        L.set_populations(np.asarray(f0, np.float32), 3)
        loss, ge, gs = L.adjoint(steps, *plane, k)
        held[k] = L.adjoint_workspace_bytes
        results[k] = (loss, ge.cpu().numpy(), gs.cpu().numpy())
    assert held[K] <= held[k0] < held[K + 1]
    for k in (K, K + 1):
        assert results[k][0] == results[k0][0]
        assert np.array_equal(results[k][1], results[k0][1]) and np.array_equal(results[k][2], results[k0][2])
    L.close()


@pytest.mark.parametrize("interval", [-1, 5])
def test_tiled_recording_equals_single_steps_bitwise(interval):
    """Where lbm_step takes the MM tiled pass (the default mode on a lattice that fills the GPU),
    the adjoint records pairs of forward steps as tiled passes, in the final segment and in every
    recomputed one, and steps back one step per launch. Loss and gradients must equal those of
    single steps (lbm_set_step_fusion(0)) bit for bit: odd step counts and segment lengths leave
    single recording steps, and the sources lie in the tiles."""
    from paper_2309_08068_gb300.lbm import lattice_from_workload
    w, f0, plane = small_case("mm", seed=91, shape=(96, 96, 96), plane=(0, 13))
    steps = 13
    out = {}
    for mode in (0, 1):
        L = lattice_from_workload(w, init=False)
        L.set_step_fusion(mode)
        assert L.pass_kind == (None if mode == 0 else "tiled")
        L.set_populations(np.asarray(f0, np.float32), 3)
        loss, ge, gs = L.adjoint(steps, plane[0], plane[1], interval)
        out[mode] = (loss, ge.cpu().numpy(), gs.cpu().numpy(), L.populations_host())
        L.close()
    assert out[1][0] == out[0][0]
    for k in (1, 2, 3):
        assert np.array_equal(out[1][k], out[0][k]), k
    assert np.isfinite(out[0][0]) and np.abs(out[0][1]).max() > 0


@pytest.mark.parametrize("interval", [-1, 5])
def test_tiled_backward_equals_single_steps_bitwise(interval):
    """With fusion mode 3 (planes of at least 16 x 16), pairs of MM forward steps record and pairs of
    backward steps run as tiled passes. The loss and both gradients must equal those of single steps
    (lbm_set_step_fusion(0)) bit for bit: odd step counts (a single step is left over), a
    current and an imposed source in the tiles, per-cell eps_r and sigma, every record resident or
    segments of 5 steps. The oracle adjoint checks the result as in the other tests."""
    from paper_2309_08068_gb300.lbm import lattice_from_workload
    w, f0, plane = small_case("mm", seed=90, shape=(20, 18, 9), plane=(0, 13))
    steps = 13
    out = {}
    for mode in (0, 3):
        L = lattice_from_workload(w, init=False)
        L.set_step_fusion(mode)
        assert L.pass_kind == (None if mode == 0 else "tiled")
        L.set_populations(np.asarray(f0, np.float32), 3)
        loss, ge, gs = L.adjoint(steps, plane[0], plane[1], interval)
        out[mode] = (loss, ge.cpu().numpy(), gs.cpu().numpy())
        L.close()
    assert out[3][0] == out[0][0]
    assert np.array_equal(out[3][1], out[0][1])
    assert np.array_equal(out[3][2], out[0][2])
    O = oracle_from_workload(w, init=False, threads=8)
    O.set_populations(f0, 3)
    loss_ref, ge_ref, gs_ref = O.loss_and_gradient(steps, *plane)
    assert abs(out[3][0] - loss_ref) <= LOSS_TOL * loss_ref
    assert rel_l2(out[3][1], ge_ref) <= GRAD_TOL
    assert rel_l2(out[3][2], gs_ref) <= GRAD_TOL


@pytest.mark.parametrize("model", ["mm", "hv"])
def test_sigma_gradient_can_be_skipped(model):
    """Without an output for dL/d sigma the adjoint skips its sums; the loss and dL/d eps_r are the
    same bits as with it."""
    from paper_2309_08068_gb300.lbm import lattice_from_workload
    w, f0, plane = small_case(model, seed=91, shape=(20, 18, 9), plane=(0, 13))
    out = []
    for sigma in (True, False):
        L = lattice_from_workload(w, init=False)
        L.set_populations(np.asarray(f0, np.float32), 3)
        loss, ge, gs = L.adjoint(11, plane[0], plane[1], 4, sigma=sigma)
        assert (gs is None) == (not sigma)
        out.append((loss, ge.cpu().numpy()))
        L.close()
    assert out[0][0] == out[1][0]
    assert np.array_equal(out[0][1], out[1][1])
