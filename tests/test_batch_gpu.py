"""Batched stepping of lattices of uneven sizes (lbm_batch_*): one launch per step over every
active lattice, replayed as a captured CUDA graph. It must give the same populations, bit for bit,
as stepping each lattice on its own. The refinement sweep of the skin-effect test runs batched at
full size against the FP64 oracle."""
import numpy as np
import pytest

from helpers import oracle_from_workload, rel_l2
from paper_2309_08068_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

SHAPES = [(7, 5, 3), (16, 16, 16), (33, 9, 4), (1, 1, 40), (1, 1, 1)]
MEDIA = ["random", "few", "vacuum", "few", "vacuum"]
STEPS = [5, 0, 12, 7, 3]


def make_lattices(model, storage, stream, seed=51):
    from paper_2309_08068_gb300.lbm import lattice_from_workload
    out = []
    for k, (shape, media) in enumerate(zip(SHAPES, MEDIA)):
        w, f = wl.random_state(model, shape, seed=seed + k, media=media, n_sources=2 if k % 2 == 0 else 0)
        L = lattice_from_workload(w, init=False, storage=storage, stream=stream, track_rho=model == "mm",
                                  storage_scale=0.0)
        L.set_populations(np.asarray(f, np.float32) * 1e-2, 4)
        out.append(L)
    return out


@pytest.mark.parametrize("model", ["mm", "hv"])
@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_batch_equals_individual_steps_bitwise(model, storage):
    from paper_2309_08068_gb300.lbm import Batch
    stream = torch.cuda.Stream()
    solo = make_lattices(model, storage, stream)
    grouped = make_lattices(model, storage, stream)
    batch = Batch(grouped)
    for rep in range(2):  # the second call replays the captured graph
        for L, n in zip(solo, STEPS):
            L.step(n)
        batch.step(STEPS)
        for k, (A, B) in enumerate(zip(solo, grouped)):
            assert A.time == B.time
            assert np.array_equal(A.populations_host(), B.populations_host()), (rep, k)
    assert batch.launch_count > 0


@pytest.mark.parametrize("model", ["mm", "hv"])
def test_every_launch_configuration_agrees_and_autotune_keeps_state(model):
    from paper_2309_08068_gb300.lbm import Batch
    stream = torch.cuda.Stream()
    ref = make_lattices(model, "f32", stream, seed=61)
    for L, n in zip(ref, STEPS):
        L.step(n)
    want = [L.populations_host() for L in ref]
    for block in (128, 256):
        for persistent in (False, True):
            lats = make_lattices(model, "f32", stream, seed=61)
            batch = Batch(lats)
            before = [L.populations_host() for L in lats]
            chosen = batch.autotune(2)
            assert chosen[0] in (128, 256)
            for L, b in zip(lats, before):
                assert np.array_equal(L.populations_host(), b)  # tuning leaves the state alone
            batch.set_config(block, persistent)
            batch.step(STEPS)
            for L, w in zip(lats, want):
                assert np.array_equal(L.populations_host(), w), (block, persistent)


def test_batch_rejects_mixed_contexts():
    from paper_2309_08068_gb300.lbm import Batch, Lattice, LbmError
    with pytest.raises(LbmError, match="share model"):
        Batch([Lattice("mm", (4, 4, 4)), Lattice("hv", (4, 4, 4))])
    with pytest.raises(LbmError, match="repeated"):
        L = Lattice("hv", (4, 4, 4))
        Batch([L, L])


@pytest.mark.parametrize("model", ["mm", "hv"])
def test_refinement_sweep_full_size_batched_against_oracle(model):
    """The skin-effect refinement sweep (16 lattices N = 32 ... 272, 95.9 M cells, sigma = 0.1), each
    lattice run 10 N steps in one batched call. Every lattice's (x, y) columns must equal each other
    and the FP64 oracle on 1 x 1 x N (the plane-wave problem is uniform in x and y)."""
    from paper_2309_08068_gb300.lbm import Batch, lattice_from_workload
    sigma = 0.1
    stream = torch.cuda.Stream()
    works = wl.refinement_batch(model, sigma)
    lats = [lattice_from_workload(w, stream=stream) for w in works]
    batch = Batch(lats)
    batch.autotune(2)
    batch.step([w.steps for w in works])
    worst = 0.0
    for w, L in zip(works, lats):
        n = w.shape[0]
        ex = L.fields("E")["E"][0].reshape(n, n, n)  # (z, y, x)
        assert torch.equal(ex, ex[:, :1, :1].expand_as(ex))
        w1 = wl.skin_effect_1d(model, n, sigma, periods=8)
        w1.sources[0].E0 = tuple(np.asarray(w1.sources[0].E0, np.float32).astype(np.float64))
        w1.sources[0].B0 = tuple(np.asarray(w1.sources[0].B0, np.float32).astype(np.float64))
        w1.sigma = np.asarray(w1.sigma, np.float32).astype(np.float64)
        O = oracle_from_workload(w1)
        O.step(w.steps)
        err = rel_l2(ex[:, 0, 0].cpu().numpy(), O.fields()["E"][0])
        worst = max(worst, err)
        assert err <= 1e-5, (n, err)
        L.close()
    print(f"refinement sweep {model}: worst rel L2 {worst:.3e}")


@pytest.mark.parametrize("model", ["mm", "hv"])
def test_batch_runs_wide_lattices_as_two_step_passes(model):
    """Lattices large enough for a two-step pass run their pairs of steps as such passes inside the
    batch (here one tiled and one ring pass), the others in the batched launches; with odd and even
    step counts, sources on full planes and on columns, the result equals each lattice's own
    lbm_step bit for bit, twice in a row (the second call replays the captured graph of the small
    lattices)."""
    from paper_2309_08068_gb300.lbm import Batch, lattice_from_workload
    stream = torch.cuda.Stream()
    steps = [5, 6, 3, 7]

    def lattices():
        wide, f0 = wl.slab_case(model, (128, 128, 64), seed=160)  # random media: tiled for both models
        sweep = wl.skin_effect_3d(model, 208, 0.1)  # imposed plane wave on plane 0, 8 planes of it
        sweep.shape = (208, 208, 8)
        sweep.sigma = sweep.sigma[: 208 * 208 * 8].copy()
        sweep.sigma[208 * 208 * 4:] = 0.1
        small1, f2 = wl.random_state(model, (7, 5, 3), seed=161, media="few")
        small2, f3 = wl.random_state(model, (33, 9, 4), seed=162, media="random")
        out = []
        for w, f in ((wide, f0), (sweep, None), (small1, f2), (small2, f3)):
            L = lattice_from_workload(w, init=f is None, stream=stream)
            if f is not None:
                L.set_populations(np.asarray(f, np.float32) * 1e-2, 2)
            out.append(L)
        return out

    solo, grouped = lattices(), lattices()
    assert [L.pass_kind for L in grouped] == ["tiled", "ring", None, None]
    batch = Batch(grouped)
    for rep in range(2):
        for L, n in zip(solo, steps):
            L.step(n)
        batch.step(steps)
        for k, (A, B) in enumerate(zip(solo, grouped)):
            assert A.time == B.time
            assert np.array_equal(A.populations_host(), B.populations_host()), (rep, k)
