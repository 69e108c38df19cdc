"""Two steps per pass (lbm_set_step_fusion): the wavefront kernel must give the populations and
fields of single steps bit for bit (same arithmetic, intermediate planes in the storage format),
for both models, every storage and media mode, sources in the wrap-around planes, shallow
lattices and odd step counts; and it must only switch on where it is allowed."""
import numpy as np
import pytest

from helpers import oracle_from_workload, rel_l2
from paper_2309_08068_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

PLANE = (256, 160)  # 160 tiles of 256 cells per plane: enough to fill the GPU's SMs


def run(w, f, steps, mode, tile=0, **kw):
    from paper_2309_08068_gb300.lbm import lattice_from_workload
    L = lattice_from_workload(w, init=False, **kw)
    L.set_step_fusion(mode, tile)
    active = L.step_fusion_active
    L.set_populations(np.asarray(f, np.float32), 0)
    L.step(steps)
    out = L.populations_host(), L.fields_host("EBJ"), L.time
    L.close()
    return active, out


def assert_same(a, b, q):
    assert np.array_equal(a[0][:q], b[0][:q])
    for k in a[1]:
        assert np.array_equal(a[1][k], b[1][k]), k
    assert a[2] == b[2]


@pytest.mark.parametrize("model", ["mm", "hv"])
@pytest.mark.parametrize("media", ["random", "few", "vacuum"])
@pytest.mark.parametrize("nz", [5, 6, 11])
def test_fused_pairs_equal_single_steps(model, media, nz):
    w, f = wl.slab_case(model, PLANE + (nz,), seed=110 + nz, media=media)
    q = 48 if model == "mm" else 36
    active, fused = run(w, f, 7, 2)  # three passes and one single step
    assert active
    _, single = run(w, f, 7, 0)
    assert_same(fused, single, q)


@pytest.mark.parametrize("model", ["mm", "hv"])
@pytest.mark.parametrize("tile", [256, 768, 4096])
def test_fused_pairs_equal_single_steps_for_every_item_size(model, tile):
    """Items of 1, 3 and 16 blocks of cells (768 leaves a ragged last item in each plane)."""
    w, f = wl.slab_case(model, PLANE + (7,), seed=115)
    q = 48 if model == "mm" else 36
    active, fused = run(w, f, 4, 2, tile)
    assert active
    _, single = run(w, f, 4, 0)
    assert_same(fused, single, q)


@pytest.mark.parametrize("model", ["mm", "hv"])
@pytest.mark.parametrize("plane", [(300, 140), (97, 409)])
def test_fused_pairs_equal_single_steps_when_items_split_rows(model, plane):
    """Planes whose rows are not a whole number of items: 256- and 512-cell items start mid-row, so a
    tile's neighbourhood window covers partial rows and wraps around the plane."""
    w, f = wl.slab_case(model, plane + (7,), seed=125)
    q = 48 if model == "mm" else 36
    active, fused = run(w, f, 5, 2)
    assert active
    _, single = run(w, f, 5, 0)
    assert_same(fused, single, q)


@pytest.mark.parametrize("model", ["mm", "hv"])
@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_fused_pairs_equal_single_steps_in_16_bit_storage(model, storage):
    w, f = wl.slab_case(model, PLANE + (6,), seed=120, amplitude=1e-3)
    kw = dict(storage=storage, storage_scale=2.0 ** 12 if storage == "f16" else 0.0)
    q = 48 if model == "mm" else 36
    active, fused = run(w, f, 6, 2, **kw)
    assert active
    _, single = run(w, f, 6, 0, **kw)
    assert_same(fused, single, q)


@pytest.mark.parametrize("model", ["mm", "hv"])
def test_fused_pairs_match_the_oracle(model):
    w, f = wl.slab_case(model, PLANE + (5,), seed=130)
    f = np.asarray(f, np.float32).astype(np.float64)
    for attr in ("eps_r", "mu_r", "sigma"):
        setattr(w, attr, np.asarray(getattr(w, attr), np.float32).astype(np.float64))
    for s in w.sources:
        if s.w is not None:
            s.w = np.asarray(s.w, np.float32).astype(np.float64)
        s.E0 = tuple(float(np.float32(v)) for v in s.E0)
        s.B0 = tuple(float(np.float32(v)) for v in s.B0)
    _, (pops, _, _) = run(w, f, 4, 2)
    O = oracle_from_workload(w, init=False, threads=16)
    O.set_populations(f, 0)
    O.step(4)
    q = 48 if model == "mm" else 36
    assert rel_l2(pops[:q], O.populations()[:q]) <= 1e-5


def test_fusion_switches_on_only_where_allowed():
    from paper_2309_08068_gb300.lbm import Lattice
    def kind(shape, mode=1, model="mm", eps_r=None, **kw):
        L = Lattice(model, shape, eps_r, **kw)
        L.set_step_fusion(mode)
        k = L.pass_kind
        L.close()
        return k
    # Mode 1, FP32: the tiled pass where its blocks at 8-plane chunks exceed 1.5 waves
    assert kind((96, 96, 96)) == "tiled"                  # MM: 49 tiles x 12 chunks
    assert kind((256, 256, 64)) == "tiled"
    assert kind((64, 64, 64)) is None                     # 200 blocks: single steps
    assert kind(PLANE + (11,)) == "ring"                  # 456 blocks: the ring pass instead
    assert kind((128, 128, 128), model="hv") == "tiled"   # HV, uniform medium: no ring on 128^2 planes
    assert kind((256, 256, 64), model="hv") == "ring"     # HV, uniform medium: the ring pass first
    eps = np.random.default_rng(3).uniform(1.0, 4.0, 256 * 256 * 64).astype(np.float32)
    assert kind((256, 256, 64), model="hv", eps_r=eps) == "tiled"  # HV, other media: the tiled pass first
    assert kind(PLANE + (11,), model="hv") == "ring"
    assert kind((64, 64, 11), model="hv") is None         # neither applies
    # Mode 3: the tiled pass wherever a 16 x 16 extended tile and 3 planes fit
    assert kind((16, 16, 3), mode=3) == "tiled"
    assert kind((64, 64, 11), mode=3, model="hv") == "tiled"
    assert kind((15, 64, 11), mode=3) is None
    assert kind((64, 64, 2), mode=3) is None
    assert kind((256, 256, 64), mode=0) is None
    assert kind((256, 256, 64), track_rho=True) is None  # rest populations are not carried
    assert kind((256, 256, 64), z_ghost=True) is None    # slabs step one plane range at a time
    assert kind((256, 256, 64), mode=3, z_ghost=True) is None
    # Mode 2: the ring pass
    assert kind(PLANE + (11,), mode=2) == "ring"          # 7 planes of 7.9 MB fit in L2
    assert kind((64, 64, 11), mode=2) is None             # 4,096 cells per plane cannot fill the GPU
    assert kind(PLANE + (3,), mode=2) is None             # MM runs A 3 planes ahead: nz >= 4
    assert kind(PLANE + (4,), mode=2) == "ring"
    assert kind((512, 512, 6), mode=2) == "ring"          # forced: 7 x 50 MB exceed L2
    # 16-bit storage: single steps by default, either pass when asked for
    assert kind((256, 256, 64), storage="f16", storage_scale=2.0 ** 12) is None
    assert kind(PLANE + (11,), mode=3, storage="f16", storage_scale=2.0 ** 12) == "tiled"
    assert kind(PLANE + (11,), mode=2, storage="bf16") == "ring"


def test_hv_needs_five_planes():
    from paper_2309_08068_gb300.lbm import Lattice
    for nz, expect in ((4, False), (5, True)):
        L = Lattice("hv", PLANE + (nz,))
        L.set_step_fusion(2)
        assert L.step_fusion_active == expect
        L.close()


def test_fusion_mode_is_checked():
    from paper_2309_08068_gb300.lbm import Lattice, LbmError
    L = Lattice("hv", (8, 8, 8))
    for mode, tile in ((4, 0), (-1, 0), (1, 100), (1, 8192), (1, -256)):
        with pytest.raises(LbmError):
            L.set_step_fusion(mode, tile)
    L.close()


@pytest.mark.parametrize("model", ["mm", "hv"])
def test_expired_wait_stops_the_pass_and_reports_etimedout(model):
    """A dependency wait that runs out stops every block of the pass, and the next waiting call
    returns LBM_ETIMEDOUT once, naming the pass. A negative wait limit makes the first check of every
    dependent item give up, so the path is taken on every run, without a fault or a hang. The
    context then steps as before: restored populations give single steps' results bit for bit."""
    from paper_2309_08068_gb300.lbm import LbmError, lattice_from_workload
    w, f = wl.slab_case(model, PLANE + (7,), seed=140)
    f = np.asarray(f, np.float32)
    q = 48 if model == "mm" else 36
    L = lattice_from_workload(w, init=False)
    L.set_step_fusion(2)
    assert L.step_fusion_active
    L.set_populations(f, 0)
    L.set_wait_limit(-1)
    L.step(2)
    with pytest.raises(LbmError) as err:
        L.sync()
    assert err.value.code == -5  # LBM_ETIMEDOUT
    assert "two-step pass" in str(err.value)
    L.sync()  # reported once
    L.set_wait_limit(0)
    L.set_populations(f, 0)
    L.step(4)
    fused = L.populations_host(), L.fields_host("EBJ"), L.time
    L.close()
    _, single = run(w, f, 4, 0)
    assert_same(fused, single, q)


def test_expired_wait_is_reported_by_host_reductions_and_reads():
    """Every host-side read after a stopped pass reports it: lbm_reduce, lbm_get_populations and
    lbm_fields return LBM_ETIMEDOUT instead of values of undefined populations."""
    from paper_2309_08068_gb300.lbm import LbmError, lattice_from_workload
    w, f = wl.slab_case("mm", PLANE + (6,), seed=141)
    L = lattice_from_workload(w, init=False)
    L.set_step_fusion(2)
    L.set_populations(np.asarray(f, np.float32), 0)
    for read in (L.reduce, L.populations_host, lambda: L.fields_host("E")):
        L.set_wait_limit(-1)
        L.step(2)
        with pytest.raises(LbmError) as err:
            read()
        assert err.value.code == -5
    L.set_wait_limit(0)
    L.close()


@pytest.mark.parametrize("model", ["mm", "hv"])
@pytest.mark.parametrize("tile", [256, 768])
def test_fused_pairs_equal_single_steps_with_full_source_planes(model, tile):
    """Every cell of a plane a source cell: an imposed plane wave on plane 0 (a wrap plane) and a
    current over the whole of plane 3 and half of plane 4. Each tile recomputes its own source cells
    after its ordinary update, so a plane of 40,960 source cells adds work to every tile of it
    rather than to one item; the results must still equal single steps bit for bit."""
    w, f = wl.random_state(model, PLANE + (7,), seed=150, media="few", n_sources=0)
    nxy = PLANE[0] * PLANE[1]
    rng = np.random.default_rng(151)
    c = wl.LIGHT_SPEED[model]
    w.sources = [
        wl.Source("impose", np.arange(nxy, dtype=np.int64), wl.TimeFunction("sin", 1.0, 40.0, 0.3),
                  E0=(1e-3, 0.0, 0.0), B0=(0.0, 1e-3 / c, 0.0)),
        wl.Source("current", np.arange(3 * nxy, 4 * nxy + nxy // 2, dtype=np.int64),
                  wl.TimeFunction("sin", 1e-3, 17.0, 0.1), w=rng.standard_normal((nxy + nxy // 2, 3))),
    ]
    q = 48 if model == "mm" else 36
    active, fused = run(w, f, 5, 2, tile)
    assert active
    _, single = run(w, f, 5, 0)
    assert_same(fused, single, q)



# ---------------------------------------------------------------------------------------------
# The tiled pass (mode 3; mode 1's choice where it fills the GPU): shared-memory tiles with a one-cell ring
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("model", ["mm", "hv"])
@pytest.mark.parametrize("media", ["random", "few", "vacuum"])
@pytest.mark.parametrize("shape", [(256, 160, 11), (29, 17, 9), (16, 16, 3), (45, 31, 40), (64, 48, 5)],
                         ids=lambda s: "x".join(map(str, s)))
def test_tiled_pairs_equal_single_steps(model, media, shape):
    """Ragged last tiles in x and y (29 = 14 + 15, 45 = 3 x 14 + 3), the smallest plane and depth the
    pass takes (16 x 16 x 3: the ring of a tile wraps onto its neighbour on both sides), several
    chunks of planes per tile column (nz = 40), odd step counts, sources in every plane."""
    w, f = wl.slab_case(model, shape, seed=170 + shape[2], media=media)
    q = 48 if model == "mm" else 36
    active, tiled = run(w, f, 7, 3)
    assert active
    _, single = run(w, f, 7, 0)
    assert_same(tiled, single, q)


@pytest.mark.parametrize("model", ["mm", "hv"])
@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_tiled_pairs_equal_single_steps_in_16_bit_storage(model, storage):
    w, f = wl.slab_case(model, (64, 40, 9), seed=175, amplitude=1e-3)
    kw = dict(storage=storage, storage_scale=2.0 ** 12 if storage == "f16" else 0.0)
    q = 48 if model == "mm" else 36
    active, tiled = run(w, f, 6, 3, **kw)
    assert active
    _, single = run(w, f, 6, 0, **kw)
    assert_same(tiled, single, q)


@pytest.mark.parametrize("model", ["mm", "hv"])
def test_tiled_pairs_with_full_source_planes(model):
    """Whole planes of source cells: every extended cell of those planes is recomputed after the
    ordinary update, in both phases, including the wrap plane 0."""
    w, f = wl.random_state(model, (64, 48, 7), seed=176, media="few", n_sources=0)
    nxy = 64 * 48
    rng = np.random.default_rng(177)
    c = wl.LIGHT_SPEED[model]
    w.sources = [
        wl.Source("impose", np.arange(nxy, dtype=np.int64), wl.TimeFunction("sin", 1.0, 40.0, 0.3),
                  E0=(1e-3, 0.0, 0.0), B0=(0.0, 1e-3 / c, 0.0)),
        wl.Source("current", np.arange(3 * nxy, 4 * nxy + nxy // 2, dtype=np.int64),
                  wl.TimeFunction("sin", 1e-3, 17.0, 0.1), w=rng.standard_normal((nxy + nxy // 2, 3))),
    ]
    q = 48 if model == "mm" else 36
    active, tiled = run(w, f, 5, 3)
    assert active
    _, single = run(w, f, 5, 0)
    assert_same(tiled, single, q)


@pytest.mark.parametrize("model", ["mm", "hv"])
def test_tiled_pairs_match_the_oracle(model):
    w, f = wl.slab_case(model, (40, 33, 6), seed=178)
    f = np.asarray(f, np.float32).astype(np.float64)
    for attr in ("eps_r", "mu_r", "sigma"):
        setattr(w, attr, np.asarray(getattr(w, attr), np.float32).astype(np.float64))
    for s in w.sources:
        if s.w is not None:
            s.w = np.asarray(s.w, np.float32).astype(np.float64)
        s.E0 = tuple(float(np.float32(v)) for v in s.E0)
        s.B0 = tuple(float(np.float32(v)) for v in s.B0)
    _, (pops, _, _) = run(w, f, 4, 3)
    O = oracle_from_workload(w, init=False, threads=16)
    O.set_populations(f, 0)
    O.step(4)
    q = 48 if model == "mm" else 36
    assert rel_l2(pops[:q], O.populations()[:q]) <= 1e-5
