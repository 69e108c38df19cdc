"""The z-slab decomposition's host logic on CPU, without a GPU.

* slab_bounds / slab_workload: plane ranges, ghost planes, media and source mapping.
* The exchange schedule (slabs.exchange) over gloo ranks. Each rank steps one z-slab of the FP64
  oracle plus two ghost planes, and swaps whole boundary planes with its neighbours before every
  step. The oracle advects by pushing, so its ghost planes are stepped too: they carry the
  neighbours' media and sources. The gathered slabs must equal the unsplit oracle bit for bit.
"""
import os
import socket

import numpy as np
import pytest

from helpers import oracle_from_workload
from paper_2309_08068_gb300 import workloads as wl
from paper_2309_08068_gb300.slabs import slab_bounds, slab_planes, slab_workload, interior

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

SHAPE = (6, 5, 9)
STEPS = 8


def test_slab_bounds_cover_the_lattice_evenly():
    for nz in (1, 2, 7, 9, 64):
        for parts in range(1, min(nz, 6) + 1):
            b = slab_bounds(nz, parts)
            assert b[0][0] == 0 and b[-1][1] == nz
            assert all(b[k][1] == b[k + 1][0] for k in range(parts - 1))
            sizes = [z1 - z0 for z0, z1 in b]
            assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        slab_bounds(4, 5)
    assert list(slab_planes(0, 3, 9)) == [8, 0, 1, 2, 3]
    assert list(slab_planes(6, 9, 9)) == [5, 6, 7, 8, 0]


def test_slab_workload_maps_media_fields_and_sources():
    w, _ = wl.slab_case("mm", SHAPE, seed=7)
    nx, ny, nz = SHAPE
    nxy = nx * ny
    w.E = np.random.default_rng(1).standard_normal((3, w.n))
    z0, z1 = 3, 6
    p = slab_workload(w, z0, z1)
    assert p.shape == (nx, ny, z1 - z0 + 2)
    for local, g in enumerate(slab_planes(z0, z1, nz)):
        assert np.array_equal(p.eps_r[local * nxy:(local + 1) * nxy], w.eps_r[g * nxy:(g + 1) * nxy])
        assert np.array_equal(p.E[:, local * nxy:(local + 1) * nxy], w.E[:, g * nxy:(g + 1) * nxy])
    # every source cell of planes z0..z1-1 appears once, shifted by one plane, with its weight
    for s, ps in zip([s for s in w.sources if ((np.asarray(s.cells) // nxy >= z0) & (np.asarray(s.cells) // nxy < z1)).any()],
                     p.sources):
        cells = np.asarray(s.cells)
        keep = (cells // nxy >= z0) & (cells // nxy < z1)
        assert np.array_equal(ps.cells, cells[keep] - (z0 - 1) * nxy)
        if s.w is not None:
            assert np.array_equal(ps.w, np.asarray(s.w)[keep])
    local_planes = np.concatenate([np.asarray(s.cells) // nxy for s in p.sources])
    assert local_planes.min() >= 1 and local_planes.max() <= z1 - z0


def _oracle_slab(w, z0, z1):
    """Oracle lattice of slab [z0, z1) with ghost planes that carry the neighbours' sources."""
    nx, ny, nz = w.shape
    nxy = nx * ny
    part = slab_workload(w, z0, z1)
    planes = slab_planes(z0, z1, nz)
    sources = []
    for s in w.sources:
        cells = np.asarray(s.cells, dtype=np.int64)
        local, rows = [], []
        for l, g in enumerate(planes):
            hit = np.nonzero(cells // nxy == g)[0]
            local.append(l * nxy + cells[hit] % nxy)
            rows.append(hit)
        local, rows = np.concatenate(local), np.concatenate(rows)
        if local.size:
            weights = None if s.w is None else np.asarray(s.w).reshape(-1, 3)[rows]
            sources.append(wl.Source(s.kind, local, s.fn, w=weights, E0=s.E0, B0=s.B0))
    part.sources = sources
    return oracle_from_workload(part, init=False), planes


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, model, seed, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    from paper_2309_08068_gb300.slabs import exchange
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, f = wl.slab_case(model, SHAPE, seed)
        nx, ny, nz = SHAPE
        nxy = nx * ny
        z0, z1 = slab_bounds(nz, world)[rank]
        O, planes = _oracle_slab(w, z0, z1)
        cells = (planes[:, None] * nxy + np.arange(nxy)[None, :]).reshape(-1)
        O.set_populations(f[:, cells], 0)
        top = z1 - z0  # local index of the last own plane

        def pack(face):
            p = 1 if face == 0 else top
            return torch.from_numpy(np.ascontiguousarray(O.populations()[:, p * nxy:(p + 1) * nxy]))

        def unpack(face, t):
            p = 0 if face == 0 else top + 1
            g = O.populations()
            g[:, p * nxy:(p + 1) * nxy] = t.numpy()
            O.set_populations(g, O.time)

        for _ in range(STEPS):
            exchange(pack, unpack, rank, world)
            O.step(1)
        q.put((rank, interior(O.populations(), O.shape)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("model", ["mm", "hv"])
def test_oracle_slabs_on_gloo_ranks_equal_the_unsplit_oracle(world, model):
    seed = 40 + world
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, model, seed, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = dict(q.get(timeout=180) for _ in range(world))
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    got = np.concatenate([results[r] for r in range(world)], axis=1)
    w, f = wl.slab_case(model, SHAPE, seed)
    O = oracle_from_workload(w, init=False)
    O.set_populations(f, 0)
    O.step(STEPS)
    assert np.array_equal(got, O.populations())
