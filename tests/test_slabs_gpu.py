"""z-slab decomposition on one GPU: a lattice split into slabs with ghost planes, exchanging their
halos before every step, must give the populations of the unsplit lattice bit for bit (each cell
runs the same arithmetic on the same inputs), and so match the FP64 oracle like the unsplit run."""
import numpy as np
import pytest

from helpers import oracle_from_workload, rel_l2
from paper_2309_08068_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

SHAPE = (12, 10, 14)


def unsplit(w, f, steps, **kw):
    from paper_2309_08068_gb300.lbm import lattice_from_workload
    L = lattice_from_workload(w, init=False, **kw)
    L.set_populations(np.asarray(f, np.float32), 0)
    L.step(steps)
    out = L.populations_host()
    fields = L.fields_host("EBJ")
    red = L.reduce()
    L.close()
    return out, fields, red


def split(w, f, steps, parts, **kw):
    from paper_2309_08068_gb300.slabs import Slabs
    S = Slabs(w, parts, init=False, **kw)
    S.set_populations(f, 0)
    S.step(steps)
    out = S.populations_host()
    fields = S.fields_host("EBJ")
    red = S.reduce()
    assert S.time == steps
    S.close()
    return out, fields, red


@pytest.mark.parametrize("model", ["mm", "hv"])
@pytest.mark.parametrize("parts", [1, 2, 3, 5])
def test_slabs_equal_the_unsplit_lattice_bitwise(model, parts):
    w, f = wl.slab_case(model, SHAPE, seed=90 + parts)
    steps = 24
    ref, ref_fields, ref_red = unsplit(w, f, steps)
    got, got_fields, got_red = split(w, f, steps, parts)
    q = 48 if model == "mm" else 36
    assert np.array_equal(got[:q], ref[:q])
    for k in ref_fields:
        assert np.array_equal(got_fields[k], ref_fields[k]), k
    assert got_red[0] == pytest.approx(ref_red[0], rel=1e-12)
    assert got_red[1] == pytest.approx(ref_red[1], rel=1e-12)


@pytest.mark.parametrize("model", ["mm", "hv"])
def test_slabs_match_the_oracle(model):
    w, f = wl.slab_case(model, SHAPE, seed=97)
    f = np.asarray(f, np.float32).astype(np.float64)
    for attr in ("eps_r", "mu_r", "sigma"):
        setattr(w, attr, np.asarray(getattr(w, attr), np.float32).astype(np.float64))
    for s in w.sources:
        if s.w is not None:
            s.w = np.asarray(s.w, np.float32).astype(np.float64)
        s.E0 = tuple(float(np.float32(v)) for v in s.E0)
        s.B0 = tuple(float(np.float32(v)) for v in s.B0)
    steps = 20
    got, _, _ = split(w, f, steps, 3)
    O = oracle_from_workload(w, init=False, threads=8)
    O.set_populations(f, 0)
    O.step(steps)
    q = 48 if model == "mm" else 36
    assert rel_l2(got[:q], O.populations()[:q]) <= 1e-5


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_slabs_bitwise_in_16_bit_storage(storage):
    w, f = wl.slab_case("mm", SHAPE, seed=98, amplitude=1e-3)
    kw = dict(storage=storage, storage_scale=2.0 ** 12 if storage == "f16" else 0.0)
    ref, _, _ = unsplit(w, f, 16, **kw)
    got, _, _ = split(w, f, 16, 2, **kw)
    assert np.array_equal(got[:48], ref[:48])


def test_slabs_keep_the_charge_with_track_rho():
    w, f = wl.slab_case("mm", SHAPE, seed=99)
    ref, _, ref_red = unsplit(w, f, 12, track_rho=True)
    got, _, got_red = split(w, f, 12, 3, track_rho=True)
    assert np.array_equal(got, ref)
    assert got_red[2] == pytest.approx(ref_red[2], rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("model", ["mm", "hv"])
def test_host_pack_and_unpack_equal_the_device_exchange(model):
    """Exchanging through host buffers (the path a host-staged transport would take) gives what
    lbm_halo_exchange gives; packed faces have the documented size."""
    from paper_2309_08068_gb300.slabs import Slabs
    w, f = wl.slab_case(model, SHAPE, seed=100)
    A = Slabs(w, 2, init=False)
    B = Slabs(w, 2, init=False)
    for S in (A, B):
        S.set_populations(f, 0)
    nxy = SHAPE[0] * SHAPE[1]
    per_cell = 4 * 16 if model == "mm" else 16 + 8
    for L in A.lattices:
        assert L.halo_bytes == per_cell * nxy
    lib = A.lattices[0].lib
    for step in range(6):
        A.exchange()
        lo, hi = B.lattices
        for lower, upper in ((lo, hi), (hi, lo)):
            up = np.empty(lower.halo_bytes, np.uint8)
            down = np.empty(upper.halo_bytes, np.uint8)
            assert lib.lbm_halo_pack(lower.h, 1, up.ctypes.data, 0) == 0
            assert lib.lbm_halo_pack(upper.h, 0, down.ctypes.data, 0) == 0
            assert lib.lbm_halo_unpack(upper.h, 0, up.ctypes.data, 0) == 0
            assert lib.lbm_halo_unpack(lower.h, 1, down.ctypes.data, 0) == 0
        for S in (A, B):
            for L in S.lattices:
                L.step(1)
    assert np.array_equal(A.populations_host(), B.populations_host())
    A.close()
    B.close()


def test_slab_rank_with_one_rank_is_the_periodic_lattice():
    from paper_2309_08068_gb300.slabs import SlabRank, interior
    w, f = wl.slab_case("hv", SHAPE, seed=101)
    ref, _, _ = unsplit(w, f, 10)
    R = SlabRank(w, 0, 1, init=False)
    nxy = SHAPE[0] * SHAPE[1]
    planes = np.concatenate([[SHAPE[2] - 1], np.arange(SHAPE[2]), [0]])
    cells = (planes[:, None] * nxy + np.arange(nxy)[None, :]).reshape(-1)
    R.lattice.set_populations(np.asarray(f, np.float32)[:, cells], 0)
    R.step(10)
    R.exchange()  # the boundary planes' populations are read from the ghost planes
    assert np.array_equal(interior(R.lattice.populations_host(), R.lattice.shape), ref)
    R.close()


def test_slab_arguments_are_checked():
    from paper_2309_08068_gb300.lbm import Lattice, LbmError, lattice_from_workload
    w, _ = wl.slab_case("mm", (6, 5, 4), seed=102)
    L = lattice_from_workload(w, init=False)
    with pytest.raises(LbmError):
        L.halo_bytes
    assert L.lib.lbm_halo_pack(L.h, 0, None, 0) != 0
    with pytest.raises(LbmError):
        Lattice("mm", (6, 5, 2), z_ghost=True)
    G = Lattice("mm", (6, 5, 4), z_ghost=True)
    with pytest.raises(LbmError):  # a source in ghost plane 0
        G.add_source(wl.Source("current", np.array([3]), wl.TimeFunction("const"), w=np.ones((1, 3))))
    with pytest.raises(LbmError):
        G.adjoint(2, 0, 1)
    assert G.lib.lbm_halo_pack(G.h, 2, G.halo_pack(0).data_ptr(), 1) != 0
    L.close()
    G.close()


def test_bench_slab_split_runs_on_one_rank():
    """The benchmark's z-slab mode (bench.time_slab_split) on one rank: the single slab closes the
    periodic ring on itself, so every step packs and unpacks both faces through the same exchange
    schedule the multi-rank run uses, and the fields stay finite."""
    import bench
    stream = torch.cuda.Stream()
    res = bench.time_slab_split(64, 16, 4, 3, 0, 1, stream)
    assert res["finite"]
    assert res["slab_planes"] == (0, 16)
    assert res["launches"] > 0 and res["elapsed_ms"] > 0 and res["e2e_s"] > 0
    assert res["halo_bytes_sent_per_step"]["mm"] == 2 * 4 * 16 * 64 * 64
    assert res["halo_bytes_sent_per_step"]["hv"] == 2 * (16 + 8) * 64 * 64
