"""z-slab decomposition of one periodic lattice.

Within a step a cell reads only its 3 x 3 x 3 neighbourhood (the advection of Sections II and III),
so the lattice splits into slabs along z that share one plane of populations per face and step.
Each slab is a ``z_ghost`` lattice: its planes 1 .. nz_k are slab planes z0 .. z1 - 1 of the whole
lattice, and planes 0 and nz_k + 1 are ghost copies of planes z0 - 1 and z1 (periodic). Before every
step, each face's crossing populations go to the neighbour's ghost plane (``lbm_halo_*``). That is
all the coupling there is, so the slabs reproduce the unsplit lattice bit for bit.

``Slabs`` keeps every slab on this device and exchanges with ``lbm_halo_exchange``. ``SlabRank``
keeps slab ``rank`` of ``world`` on this rank's device. ``exchange`` moves the packed faces between
ranks with ``torch.distributed`` point-to-point operations (NCCL between GPUs). It takes the pack
and unpack steps as arguments, so the same exchange schedule serves any slab storage.
"""
from __future__ import annotations

import numpy as np

from . import workloads as wl


def slab_bounds(nz: int, parts: int) -> list:
    """[(z0, z1)] of `parts` slabs covering 0 .. nz - 1, sizes differing by at most one plane."""
    if parts < 1 or parts > nz:
        raise ValueError(f"cannot split {nz} planes into {parts} slabs")
    base, extra = divmod(nz, parts)
    out, z = [], 0
    for k in range(parts):
        size = base + (1 if k < extra else 0)
        out.append((z, z + size))
        z += size
    return out


def slab_planes(z0: int, z1: int, nz: int) -> np.ndarray:
    """Global z of the slab's local planes: ghost z0 - 1, z0 .. z1 - 1, ghost z1 (periodic)."""
    return np.concatenate([[(z0 - 1) % nz], np.arange(z0, z1), [z1 % nz]]).astype(np.int64)


def _plane_cells(shape, planes: np.ndarray) -> np.ndarray:
    nx, ny, _ = shape
    nxy = nx * ny
    return (planes[:, None] * nxy + np.arange(nxy)[None, :]).reshape(-1)


def slab_workload(w: wl.Workload, z0: int, z1: int) -> wl.Workload:
    """The part of workload `w` that slab [z0, z1) steps, as a workload of z1 - z0 + 2 planes.

    Media and initial fields cover the ghost planes too (copied from the neighbouring planes).
    Sources keep their order and only their cells in the slab's own planes: a ghost cell is stepped
    by the slab that owns it.
    """
    nx, ny, nz = w.shape
    nxy = nx * ny
    planes = slab_planes(z0, z1, nz)
    take = _plane_cells(w.shape, planes)

    def part(a, rows=False):
        if a is None:
            return None
        a = np.asarray(a)
        return a[:, take].copy() if rows else a[take].copy()

    sources = []
    for s in w.sources:
        cells = np.asarray(s.cells, dtype=np.int64).reshape(-1)
        z = cells // nxy
        keep = (z >= z0) & (z < z1)
        if not keep.any():
            continue
        local = cells[keep] - z0 * nxy + nxy
        weights = None if s.w is None else np.asarray(s.w).reshape(-1, 3)[keep]
        sources.append(wl.Source(s.kind, local, s.fn, w=weights, E0=s.E0, B0=s.B0))
    return wl.Workload(f"{w.name}[z {z0}:{z1}]", w.model, (nx, ny, z1 - z0 + 2), w.steps, eps_r=part(w.eps_r),
                       mu_r=part(w.mu_r), sigma=part(w.sigma), E=part(w.E, rows=True), B=part(w.B, rows=True),
                       sources=sources)


def interior(a, shape, rows: bool = True):
    """Drop the two ghost planes of a slab array ((k, n) when rows, else (n,))."""
    nx, ny, _ = shape
    nxy = nx * ny
    return a[:, nxy:-nxy] if rows else a[nxy:-nxy]


def exchange(pack, unpack, rank: int, world: int, group=None) -> None:
    """One halo exchange of a periodic ring of `world` slabs, slab k on rank k.

    pack(face) returns the outgoing values of face 0 (down) or 1 (up) as a tensor. unpack(face,
    tensor) stores what arrived from below (face 0) or above (face 1). Each direction carries its
    own tag, so that with two ranks, where both neighbours are the same rank, the up and down
    messages still pair correctly. The four operations are posted as one batch, which NCCL needs
    to run the sends and receives of a pair together.
    """
    import torch
    import torch.distributed as dist
    send_up, send_down = pack(1), pack(0)
    if world == 1:
        unpack(0, send_up)
        unpack(1, send_down)
        return
    up, down = (rank + 1) % world, (rank - 1) % world
    from_below, from_above = torch.empty_like(send_up), torch.empty_like(send_down)
    ops = [dist.P2POp(dist.isend, send_up, up, group, tag=0), dist.P2POp(dist.isend, send_down, down, group, tag=1),
           dist.P2POp(dist.irecv, from_below, down, group, tag=0), dist.P2POp(dist.irecv, from_above, up, group, tag=1)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    unpack(0, from_below)
    unpack(1, from_above)


def _slab_lattice(w: wl.Workload, storage: str, storage_scale: float, track_rho: bool, stream, init: bool):
    from .lbm import Lattice
    L = Lattice(w.model, w.shape, w.eps_r, w.mu_r, w.sigma, track_rho=track_rho, stream=stream, storage=storage,
                storage_scale=storage_scale, z_ghost=True)
    for s in w.sources:
        L.add_source(s)
    if init:
        zeros = np.zeros((3, w.n), np.float32)
        L.init_fields(zeros if w.E is None else w.E, zeros if w.B is None else w.B)
    return L


class Slabs:
    """All `parts` z-slabs of workload `w` on this device: one lattice per slab, stepped in turn,
    with one ``lbm_halo_exchange`` per interface before every step."""

    def __init__(self, w: wl.Workload, parts: int, *, storage: str = "f32", storage_scale: float = 0.0,
                 track_rho: bool = False, stream=None, init: bool = True):
        self.workload = w
        self.bounds = slab_bounds(w.shape[2], parts)
        self.parts = [slab_workload(w, z0, z1) for z0, z1 in self.bounds]
        self.lattices = [_slab_lattice(p, storage, storage_scale, track_rho, stream, init) for p in self.parts]

    def exchange(self) -> None:
        k = len(self.lattices)
        for i in range(k):
            self.lattices[i].halo_exchange(self.lattices[(i + 1) % k])

    def step(self, n: int = 1) -> None:
        for _ in range(int(n)):
            self.exchange()
            for L in self.lattices:
                L.step(1)

    def set_populations(self, f, t: int = 0) -> None:
        """Load whole-lattice populations (q, n) in the canonical layout, ghost planes included."""
        f = np.asarray(f, dtype=np.float32)
        for (z0, z1), L in zip(self.bounds, self.lattices):
            L.set_populations(f[:, _plane_cells(self.workload.shape, slab_planes(z0, z1, self.workload.shape[2]))], t)

    # Reading a cell pulls its populations from the neighbours, so the boundary planes read the ghost
    # planes: every read below first brings the halo up to date (an exchange is idempotent).
    def populations_host(self) -> np.ndarray:
        """Whole-lattice populations (q, n) from the slabs' own planes."""
        self.exchange()
        return np.concatenate([interior(L.populations_host(), L.shape) for L in self.lattices], axis=1)

    def fields_host(self, names: str = "EB") -> dict:
        self.exchange()
        parts = [L.fields_host(names) for L in self.lattices]
        return {k: np.concatenate([interior(p[k], L.shape) for p, L in zip(parts, self.lattices)], axis=1)
                for k in parts[0]}

    def reduce(self):
        self.exchange()
        totals = [L.reduce() for L in self.lattices]
        return tuple(sum(t[i] for t in totals) for i in range(3))

    @property
    def time(self) -> int:
        return self.lattices[0].time

    def close(self) -> None:
        for L in self.lattices:
            L.close()


class SlabRank:
    """Slab `rank` of `world` on this rank's device (multi-GPU: one slab per rank, ``torch.distributed``
    initialised by the caller). Every step exchanges the halo with the neighbouring ranks, then steps."""

    def __init__(self, w: wl.Workload, rank: int, world: int, *, storage: str = "f32", storage_scale: float = 0.0,
                 track_rho: bool = False, stream=None, init: bool = True, group=None):
        self.rank, self.world, self.group = rank, world, group
        self.bounds = slab_bounds(w.shape[2], world)[rank]
        self.part = slab_workload(w, *self.bounds)
        self.lattice = _slab_lattice(self.part, storage, storage_scale, track_rho, stream, init)
        self._bufs = {}

    def _pack(self, face: int):
        buf = self._bufs.get(face)
        out = self.lattice.halo_pack(face, buf)
        self._bufs[face] = out
        return out

    def exchange(self) -> None:
        """Bring the ghost planes up to date (before a step, and before reading the slab)."""
        exchange(self._pack, self.lattice.halo_unpack, self.rank, self.world, self.group)

    def step(self, n: int = 1) -> None:
        for _ in range(int(n)):
            self.exchange()
            self.lattice.step(1)

    def close(self) -> None:
        self.lattice.close()
