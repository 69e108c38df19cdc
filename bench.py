"""Benchmark: lattice updates per second of the MM and HV time steps on the Hertz-dipole workload.

Workload (one GPU): a 256^3 vacuum lattice per model with the Section IV-C Gaussian dipole current
(J0 = 1e-4, alpha = 0.5, period 32 steps), FP32 populations. One benchmark step = one MM time step
on its lattice plus one HV time step on its lattice (the whole fused update of every cell, source
cells included). Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--n 256]

Under torchrun (N > 1) every rank runs its own pair of lattices (independent problems, weak
scaling, no data-path collective) by default. With ``--decomposition slabs`` the ranks instead split
one lattice per model into N z-slabs, one per rank, and exchange one plane of populations per face
and step with their neighbours (NCCL send/recv of packed faces; strong scaling). Timing is the
maximum over ranks. ``--impl reference`` times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2309_08068_gb300 import workloads as wl  # noqa: E402

METRIC = "MLUPS"
BYTES_PER_CELL = {"mm": 384, "hv": 288}  # FP32 populations read + written; vacuum needs no media bytes
POPULATION_BYTES = {"f32": 4, "bf16": 2, "f16": 2, "f24": 3}
F16_SCALE = 2.0 ** 20  # keeps populations of 1e-4-amplitude fields in FP16's normal range


def storage_scale(storage: str) -> float:
    """Power-of-two scale of the storages whose range is FP16's (FP16 and the 24-bit split)."""
    return F16_SCALE if storage in ("f16", "f24") else 0.0
FALLBACK_HBM_GBS = 6800.0
PROFILE_FILE = os.path.join(ROOT, "profiles", "traffic.json")


def kernel_source_hash(files) -> str:
    """Hash of the source files that define a kernel (so a stale ncu record is detected)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2309_08068_gb300", "csrc")
    for name in sorted(files):
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(name.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def l2_resident_bandwidth(stream, mb: int = 32, reps: int = 200):
    """Copy and write rates on a buffer that stays in L2, timed outside the timed region with
    torch's own copy and fill kernels, replayed from a CUDA graph (a 32 MB copy takes a few
    microseconds, about what a launch from Python costs). This is the on-chip ceiling that the
    two-step pass runs against, since its intermediate planes live in L2."""
    import torch
    n = mb * (1 << 20) // 4
    with torch.cuda.stream(stream):
        a = torch.ones(n, device="cuda")
        b = torch.empty_like(a)
        b.copy_(a)
        b.fill_(2.0)
    stream.synchronize()
    graphs = {}
    for name, op in (("copy", lambda: b.copy_(a)), ("write", lambda: b.fill_(2.0))):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            for _ in range(reps):
                op()
        graphs[name] = g
    out = {"buffer_MB": mb, "kernels": "torch copy_ and fill_ in a CUDA graph"}
    for name, g in graphs.items():
        with torch.cuda.stream(stream):  # a graph replays on the current stream
            g.replay()
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(3):
                g.replay()
            e1.record(stream)
        e1.synchronize()
        per_op_s = e0.elapsed_time(e1) * 1e-3 / (3 * reps)
        moved = (2 if name == "copy" else 1) * n * 4  # a copy reads and writes the buffer
        out[f"{name}_GBps"] = round(moved / per_op_s / 1e9, 1)
    del graphs, a, b
    return out


def ncu_traffic(kernel: str, n_cells: int):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, scaled to n_cells, or None
    when the summary is missing or was taken on a different kernel source."""
    try:
        with open(PROFILE_FILE) as fh:
            prof = json.load(fh)
    except Exception:
        return None
    entry = prof.get(kernel)
    if not entry or entry.get("source_hash") != kernel_source_hash(entry["sources"]):
        return None
    return entry["dram_bytes_per_launch"] * n_cells / entry["cells"]


class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[3 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_info():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float, world: int) -> float:
    """Largest value of x over all ranks (the job's time is its slowest rank's)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    device = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(cells_per_rank_step: int, steps: int, world: int, seconds: float) -> float:
    """Whole-job MLUPS: every rank updates its own lattices (weak scaling), divided by the slowest
    rank's time."""
    return cells_per_rank_step * steps * world / seconds / 1e6


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on the host cores, bounded sample
# ------------------------------------------------------------------------------------------------

def oracle_mlups(n_side: int, budget_s: float, threads: int, steps: int | None = None, warmup: int = 1):
    """Time the oracle on an n_side^3 dipole lattice per model; returns (MLUPS, steps, seconds)."""
    from oracle import OracleLattice, TimeFn
    total_updates = 0
    total_s = 0.0
    done = {}
    for model in ("mm", "hv"):
        w = wl.hertz_dipole(model, n=n_side)
        L = OracleLattice(model, w.shape, threads=threads)
        s = w.sources[0]
        L.add_current(s.cells, s.w, TimeFn("sin", s.fn.amplitude, s.fn.period, s.fn.phase))
        L.init_fields(np.zeros((3, w.n)), np.zeros((3, w.n)))
        L.step(warmup)
        k = 0
        t0 = time.perf_counter()
        while True:
            L.step(1)
            k += 1
            el = time.perf_counter() - t0
            if (steps is not None and k >= steps) or (steps is None and el >= budget_s / 2):
                break
        total_updates += w.n * k
        total_s += el
        done[model] = k
    return total_updates / total_s / 1e6, done, total_s


def storage_accuracy(storages=("f32", "bf16", "f16", "f24")):
    """Relative L2 error of E and B against the FP64 oracle after the 1500-step dielectric pulse
    (1 x 1 x 1024, eps_r = 2.5 slab) for each storage, both models."""
    from oracle import OracleLattice
    from paper_2309_08068_gb300.lbm import lattice_from_workload
    out = {st: {} for st in storages}
    for model in ("mm", "hv"):
        w = wl.dielectric_pulse_1d(model)
        w.eps_r = np.asarray(w.eps_r, np.float32).astype(np.float64)
        w.E = np.asarray(w.E, np.float32).astype(np.float64)
        w.B = np.asarray(w.B, np.float32).astype(np.float64)
        O = OracleLattice(model, w.shape, w.eps_r)
        O.init_fields(w.E, w.B)
        O.step(w.steps)
        o = O.fields()
        for st in storages:
            L = lattice_from_workload(w, storage=st, storage_scale=storage_scale(st))
            L.step(w.steps)
            g = L.fields_host("EB")
            out[st][model] = {c: float(np.linalg.norm(g[c] - o[c]) / np.linalg.norm(o[c])) for c in "EB"}
            L.close()
    return out


def slab_storage_accuracy(storages=("f32", "bf16", "f16", "f24")):
    """Storage precision on the 512 x 64 x 64 slab lattice (64 dielectric slabs, eps_r in [1, 8), plane
    pulse of amplitude 1e-4): relative L2 error of E and B of one (y, z) column against the FP64 oracle
    on the exact 1-D reduction (512 x 1 x 1), after 3000 steps for MM and 1000 for HV (HV grows
    exponentially on this medium, in FP64 too)."""
    from oracle import OracleLattice
    from paper_2309_08068_gb300.lbm import lattice_from_workload
    out = {st: {} for st in storages}
    for model, steps in (("mm", 3000), ("hv", 1000)):
        w3 = wl.slab_pulse(model)
        w1 = wl.slab_pulse(model, shape=(512, 1, 1))
        f64 = lambda a: np.asarray(a, np.float32).astype(np.float64)
        O = OracleLattice(model, w1.shape, f64(w1.eps_r), threads=8)
        O.init_fields(f64(w1.E), f64(w1.B))
        O.step(steps)
        o = O.fields()
        for st in storages:
            L = lattice_from_workload(w3, storage=st, storage_scale=storage_scale(st))
            L.step(steps)
            g = L.fields("EB")
            out[st][model] = {}
            for c in "EB":
                col = g[c].reshape(3, 64, 64, 512)[:, 17, 41, :].cpu().numpy().astype(np.float64)
                out[st][model][c] = float(np.linalg.norm(col - o[c]) / np.linalg.norm(o[c]))
            L.close()
    out["steps"] = {"mm": 3000, "hv": 1000}
    return out


def refinement_sweep(stream, steps: int):
    """The skin-effect mesh-refinement sweep (16 lattices N = 32 ... 272, 95.9 M cells, sigma = 0.1):
    `steps` steps of every lattice, batched (lattices whose planes fill the GPU as two-step passes,
    the others one launch per step, captured graph, autotuned launch configuration) against each
    lattice stepped on its own, one launch per step (lbm_step(ctx, 1)) and in one call
    (lbm_step(ctx, steps), two-step passes where they apply), same stream, same data."""
    import torch
    from paper_2309_08068_gb300.lbm import Batch, lattice_from_workload
    out = {}
    for model in ("mm", "hv"):
        works = wl.refinement_batch(model, 0.1)
        cells = sum(w.n for w in works)
        with torch.cuda.stream(stream):
            lats = [lattice_from_workload(w, stream=stream) for w in works]
        batch = Batch(lats)
        block, persistent = batch.autotune(3)
        batch.step(2)  # capture the graph of a 2-step call, then time fresh calls
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        batch.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_capture = e0.elapsed_time(e1)
        e0.record(stream)
        batch.step(steps)  # same call again: graph replay
        e1.record(stream)
        torch.cuda.synchronize()
        ms_batched = e0.elapsed_time(e1)
        e0.record(stream)
        for _ in range(steps):
            for L in lats:
                L.step(1)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_single = e0.elapsed_time(e1)
        e0.record(stream)
        for L in lats:
            L.step(steps)  # lbm_step(ctx, steps): two-step passes where they apply
        e1.record(stream)
        torch.cuda.synchronize()
        ms_own = e0.elapsed_time(e1)
        passes = [L.pass_kind for L in lats]
        out[model] = {"lattices": len(works), "cells": cells, "steps": steps,
                      "two_step_pass_by_size": {str(w.shape[0]): a for w, a in zip(works, passes) if a},
                      "batched_graph_MLUPS": round(cells * steps / (ms_batched * 1e-3) / 1e6, 1),
                      "per_lattice_launches_MLUPS": round(cells * steps / (ms_single * 1e-3) / 1e6, 1),
                      "per_lattice_lbm_step_MLUPS": round(cells * steps / (ms_own * 1e-3) / 1e6, 1),
                      "first_call_with_capture_ms": round(ms_capture, 2),
                      "autotuned": {"block": block, "persistent": persistent}}
        batch.close()
        for L in lats:
            L.close()
        torch.cuda.empty_cache()
    return out


def slab_decomposition(stream, n: int, steps: int):
    """The n^3 dipole lattice split into 2 and 4 z-slabs on this one GPU, each slab with two ghost
    planes and one halo exchange per interface before every step, against the unsplit lattice:
    `steps` steps each, CUDA events on the lattices' stream. What a multi-GPU slab run adds per GPU,
    apart from moving the packed faces between devices. Slabs step one step per launch (their ghost
    planes are refreshed between steps), so `over_unsplit` compares them with the unsplit lattice
    stepped the same way; the unsplit lattice's two-step pass is reported beside it."""
    import torch
    from paper_2309_08068_gb300.lbm import lattice_from_workload
    from paper_2309_08068_gb300.slabs import Slabs
    out = {}
    for model in ("mm", "hv"):
        w = wl.hertz_dipole(model, n=n, steps=steps)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            L = lattice_from_workload(w, stream=stream)
        unsplit = {}
        for mode in (0, 1):
            L.set_step_fusion(mode)
            L.step(4)
            torch.cuda.synchronize()
            e0.record(stream)
            L.step(steps)
            e1.record(stream)
            torch.cuda.synchronize()
            unsplit[mode] = e0.elapsed_time(e1) / steps
        ms_one = unsplit[0]
        halo = None
        L.close()
        res = {"unsplit_ms_per_step": round(ms_one, 4), "unsplit_two_step_pass_ms_per_step": round(unsplit[1], 4)}
        for parts in (2, 4):
            with torch.cuda.stream(stream):
                S = Slabs(w, parts, stream=stream)
            S.step(3)
            torch.cuda.synchronize()
            e0.record(stream)
            S.step(steps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            halo = S.lattices[0].halo_bytes
            res[f"slabs_{parts}"] = {"ms_per_step": round(ms, 4), "over_unsplit": round(ms / ms_one, 4),
                                     "MLUPS": round(w.n / (ms * 1e-3) / 1e6, 1)}
            S.close()
            torch.cuda.empty_cache()
        res["halo_bytes_per_face"] = halo
        out[model] = res
    return out


def adjoint_cost(stream, steps: int):
    """Inverse-design workload: 128^3 lattice, per-cell eps_r uniform in [1, 4), dipole with period
    24, loss plane x = 100. Time `steps` forward steps, then lbm_adjoint over `steps` steps from the
    same start: every step's record resident in HBM (interval -1); segments of ceil(sqrt(steps))
    steps (the classic sqrt(T) layout: that many checkpoints and records); and the segment length the
    library's checkpointed mode uses (lbm_adjoint_sqrt_interval), the longest within the classic
    layout's work space. Wall time of the whole call per step, against the forward step: the first
    call allocates the work space, the second (reported) reuses it."""
    import torch
    from paper_2309_08068_gb300.lbm import lattice_from_workload
    out = {}
    k_sqrt = int(math.ceil(math.sqrt(steps)))
    for model in ("mm", "hv"):
        w = wl.random_medium_dipole(model, n=128, steps=steps)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            L = lattice_from_workload(w, stream=stream)
        L.step(3)
        torch.cuda.synchronize()
        e0.record(stream)
        L.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        fwd_ms = e0.elapsed_time(e1) / steps
        L.close()
        res = {"cells": w.n, "steps": steps, "forward_ms_per_step": round(fwd_ms, 4)}
        losses = []
        with torch.cuda.stream(stream):
            L = lattice_from_workload(w, stream=stream)
        k_win = L.sqrt_interval(steps)
        L.close()
        res["sqrt_interval"] = k_win
        for mode, interval in (("resident", -1), (f"checkpoint_{k_sqrt}", k_sqrt), ("checkpoint_sqrt", k_win)):
            with torch.cuda.stream(stream):
                L = lattice_from_workload(w, stream=stream)
            torch.cuda.synchronize()
            # first call: allocates the work space; second: reuses it, as an optimisation loop does
            calls = []
            for call in range(2):
                t0 = time.perf_counter()
                loss, ge, _ = L.adjoint(steps, 0, 100, interval, sigma=False)  # C5 asks for dL/d eps_r
                calls.append((time.perf_counter() - t0) * 1e3 / steps)
                if call == 0:
                    losses.append(loss)  # both modes start from the same state here
            first_ms, adj_ms = calls
            layout = {"resident": "every step's record on the device, nothing recomputed",
                      f"checkpoint_{k_sqrt}": f"classic sqrt(T) layout: segments of {k_sqrt} steps, as many states and records",
                      "checkpoint_sqrt": f"segments of {k_win} steps: the longest within the classic layout's work space"}[mode]
            res[mode] = {"layout": layout, "adjoint_ms_per_step": round(adj_ms, 4),
                         "adjoint_over_forward": round(adj_ms / fwd_ms, 3),
                         "first_call_ms_per_step": round(first_ms, 4),
                         "workspace_gb": round(L.adjoint_workspace_bytes / 1e9, 3),
                         "gradient_finite": bool(torch.isfinite(ge).all().item())}
            L.close()
            del ge
            torch.cuda.empty_cache()
        res["loss"] = losses[0]
        res["modes_agree"] = all(x == losses[0] for x in losses)
        # Field energy every steps/4 steps: both schemes grow exponentially on this random medium,
        # which bounds how far the gradient is meaningful.
        with torch.cuda.stream(stream):
            L = lattice_from_workload(w, stream=stream)
        energy = {}
        for k in range(1, 5):
            L.step(steps // 4)
            energy[str(k * (steps // 4))] = L.reduce()[0]
        L.close()
        res["field_energy"] = energy
        e_half, e_end = energy[str(2 * (steps // 4))], energy[str(4 * (steps // 4))]
        res["energy_growth_per_step"] = (math.log(e_end / e_half) / (steps - 2 * (steps // 4))
                                         if e_half > 0 and e_end > 0 else None)
        out[model] = res
    return out


def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args):
    world, rank, _ = dist_info()
    if rank != 0:
        return
    import oracle
    oracle.build()
    cores = cpu_cores()
    side = 48
    # W untimed warm-up steps, then exactly K timed steps per model
    mlups, per_model, secs = oracle_mlups(side, 0.0, cores, steps=args.steps, warmup=args.warmup)
    # each benchmark step is one MM and one HV step on a 48^3 sample of the dipole workload
    line = {
        "impl": "reference", "metric": METRIC, "value": round(mlups, 4), "unit": "Mcell-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * secs / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"hertz_dipole_{args.n}^3_mm+hv", "sample": f"{side}^3 lattice per model",
                   "parallelism": "cpu threads"},
        "cpu_baseline": {"value": round(mlups, 4), "unit": "Mcell-updates/s", "cores": cores, "kind": "oracle",
                         "sample": f"{side}^3 dipole lattice per model, {args.steps} timed steps each after "
                                   f"{args.warmup} warm-up steps"},
        "e2e": {"value": round(mlups, 4), "unit": "Mcell-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------------

def run_ours(args):
    import torch
    world, rank, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2309_08068_gb300.lbm import lattice_from_workload

    n_side = args.n
    nz = args.nz or n_side
    ncell = n_side * n_side * nz
    stream = torch.cuda.Stream()
    lats = {}
    scale = storage_scale(args.storage)
    with torch.cuda.stream(stream):
        for model in ("mm", "hv"):
            w = wl.hertz_dipole(model, n=n_side, period=32.0, nz=nz)
            lats[model] = lattice_from_workload(w, stream=stream, storage=args.storage, storage_scale=scale)
            lats[model].set_step_fusion(args.fusion)
    torch.cuda.synchronize()
    kinds = {m: L.pass_kind for m, L in lats.items()}  # "tiled", "ring" or None (single steps)
    fused = {m: k is not None for m, k in kinds.items()}

    def chunks(k):
        """Steps per call: pairs when lbm_step runs two steps per pass, singles otherwise."""
        if args.fusion == 0:
            return [1] * k
        return [2] * (k // 2) + [1] * (k % 2)

    def advance(c, ev=None):
        if ev is not None:
            ev[0].record(stream)
        lats["mm"].step(c)
        if ev is not None:
            ev[1].record(stream)
        lats["hv"].step(c)
        if ev is not None:
            ev[2].record(stream)

    for c in chunks(args.warmup):
        advance(c)
    torch.cuda.synchronize()
    plan = chunks(args.steps)
    events = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in plan]
    launches0 = sum(L.launch_count for L in lats.values())
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        start.record(stream)
        for c, ev in zip(plan, events):
            advance(c, ev)
        stop.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    launches = sum(L.launch_count for L in lats.values()) - launches0
    elapsed_ms = start.elapsed_time(stop)
    mm_ms = sum(e[0].elapsed_time(e[1]) for e in events) / args.steps
    hv_ms = sum(e[1].elapsed_time(e[2]) for e in events) / args.steps
    for L in lats.values():
        L.sync()  # also reports a pass whose dependency wait timed out

    # the same lattices one step per launch (the single-step kernels), and as ring passes (the
    # wavefront with its intermediate planes in L2), for reference
    single, ring = {}, {}
    for model, L in lats.items():
        k1 = max(10, min(args.steps, 50))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for mode, out, per_call in ((0, single, 1), (2, ring, 2)):
            L.set_step_fusion(mode)
            if mode == 2 and L.pass_kind != "ring":
                continue
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(k1 // per_call):
                L.step(per_call)
            e1.record(stream)
            torch.cuda.synchronize()
            out[model] = e0.elapsed_time(e1) / (k1 // per_call * per_call)
        L.set_step_fusion(args.fusion)
    elapsed_ms = max_over_ranks(elapsed_ms, world)
    finite = all(L.check_finite() for L in lats.values())

    # 16- and 24-bit storage variants on the same workload (shorter timed run each)
    variants = {}
    for st in ("bf16", "f16", "f24"):
        variants[st] = {}
        for model in ("mm", "hv"):
            with torch.cuda.stream(stream):
                w = wl.hertz_dipole(model, n=n_side, period=32.0, nz=nz)
                Lv = lattice_from_workload(w, stream=stream, storage=st,
                                           storage_scale=storage_scale(st))
            Lv.set_step_fusion(args.fusion)
            for c in chunks(args.warmup):
                Lv.step(c)
            kv = max(10, min(args.steps, 200))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for c in chunks(kv):
                Lv.step(c)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / kv
            fv = Lv.pass_kind
            nbytes = BYTES_PER_CELL[model] * POPULATION_BYTES[st] // 4 // (2 if fv is not None else 1)  # per cell and step
            variants[st][model] = {"MLUPS": round(ncell / (ms * 1e-3) / 1e6, 2), "ms_per_step": round(ms, 4),
                                   "two_steps_per_pass": fv, "bytes_per_cell_step": nbytes,
                                   "algorithmic_GBps": round(nbytes * ncell / (ms * 1e-3) / 1e9, 1),
                                   "steps_timed": kv}
            Lv.close()
    accuracy = storage_accuracy() if rank == 0 else None
    slab_accuracy = slab_storage_accuracy() if rank == 0 and args.slab_accuracy else None
    refinement = refinement_sweep(stream, args.refine_steps) if args.refine_steps > 0 else None
    adjoint = adjoint_cost(stream, args.adjoint_steps) if args.adjoint_steps > 0 else None
    slabs = slab_decomposition(stream, args.n, args.slab_steps) if args.slab_steps > 0 else None

    # end to end through the C ABI with host buffers: upload fields, K steps, read E and B back
    pinned_E = torch.zeros((3, ncell), dtype=torch.float32).pin_memory()
    pinned_B = torch.zeros((3, ncell), dtype=torch.float32).pin_memory()
    out = {m: torch.empty((2, 3, ncell), dtype=torch.float32).pin_memory() for m in lats}
    e2e_steps = args.steps
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for m, L in lats.items():
        L.lib.lbm_init_fields(L.h, pinned_E.data_ptr(), pinned_B.data_ptr(), 0)
    for c in chunks(e2e_steps):
        lats["mm"].step(c)
        lats["hv"].step(c)
    for m, L in lats.items():
        L._check(L.lib.lbm_fields(L.h, 3, out[m].data_ptr(), 0))
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    h2d = 2 * 2 * 3 * ncell * 4
    d2h = 2 * 2 * 3 * ncell * 4

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    value = job_value(2 * ncell, args.steps, world, elapsed_ms * 1e-3)
    peak, peak_kind = hbm_peak()
    # Algorithmic HBM bytes per cell and step: one read and one write of the populations per step,
    # or per pair of steps when a pass runs two (the intermediate step stays on chip).
    bpc1 = {m: BYTES_PER_CELL[m] * POPULATION_BYTES[args.storage] // 4 for m in BYTES_PER_CELL}
    bpc = {m: bpc1[m] // (2 if fused[m] else 1) for m in bpc1}
    mm_gbs = bpc["mm"] * ncell / (mm_ms * 1e-3) / 1e9
    hv_gbs = bpc["hv"] * ncell / (hv_ms * 1e-3) / 1e9
    kname = {m: {"tiled": f"{m}_tile2_kernel", "ring": f"{m}_fused2_kernel", None: f"{m}_step_kernel"}[kinds[m]]
             for m in kinds}
    # ncu traffic is per launch: a fused launch covers two steps
    traffic = ncu_traffic(kname["mm"], ncell) if args.storage == "f32" else None
    hv_traffic = ncu_traffic(kname["hv"], ncell) if args.storage == "f32" else None
    single_gbs = {m: bpc1[m] * ncell / (single[m] * 1e-3) / 1e9 for m in single}
    l2 = l2_resident_bandwidth(stream)
    # Second roofline, against L2 writes (stores from the SMs plus fills from HBM). Per cell, a
    # single step writes its populations into L2 twice (the output, and the fill of its inputs from
    # HBM); a ring pass three times per two steps (the ring slot, the output and the fill), 1.5 times
    # per step; a tiled pass twice per two steps (the fill and the output), once per step.
    pop = {m: bpc1[m] // 2 for m in bpc1}
    l2w = {m: {"tiled": pop[m], "ring": 3 * pop[m] // 2, None: 2 * pop[m]}[kinds[m]] for m in pop}
    step_ms = {"mm": mm_ms, "hv": hv_ms}
    l2_roof = {m: {"kernel": kname[m], "bytes_per_cell_step": l2w[m],
                   "achieved": round(l2w[m] * ncell / (step_ms[m] * 1e-3) / 1e9, 1), "peak": l2["write_GBps"],
                   "unit": "GB/s"} for m in l2w}
    for m in l2_roof:
        l2_roof[m]["frac"] = round(l2_roof[m]["achieved"] / l2["write_GBps"], 4)
    cores = cpu_cores()
    cpu_mlups, cpu_steps, cpu_s = oracle_mlups(64, args.cpu_seconds, cores)
    # the same oracle on one thread, on a smaller sample (a fifth of the all-core budget)
    st_mlups, st_steps, st_s = oracle_mlups(32, args.cpu_seconds / 5, 1)
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "Mcell-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(elapsed_ms / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "storage": args.storage,
        "data": "synthetic",
        "config": {"workload": (f"hertz_dipole_{n_side}^3_mm+hv" if nz == n_side
                                else f"hertz_dipole_{n_side}x{n_side}x{nz}_mm+hv"), "cells_per_model": ncell,
                   "step": "one MM step + one HV step, each on its own lattice", "period": 32, "J0": 1e-4,
                   "calls": ("lbm_step(ctx, 2): two steps per pass where it applies" if args.fusion
                             else "lbm_step(ctx, 1)"),
                   "l2": "inputs larger than L2 (MM 3.2 GB, HV 2.4 GB per population buffer)",
                   "parallelism": f"independent lattices per rank x{world}"},
        "per_model": {
            "mm": {"MLUPS": round(ncell / (mm_ms * 1e-3) / 1e6, 2), "ms_per_step": round(mm_ms, 4),
                   "two_steps_per_pass": kinds["mm"], "kernel": kname["mm"],
                   "algorithmic_GBps": round(mm_gbs, 1), "bytes_per_cell_step": bpc["mm"]},
            "hv": {"MLUPS": round(ncell / (hv_ms * 1e-3) / 1e6, 2), "ms_per_step": round(hv_ms, 4),
                   "two_steps_per_pass": kinds["hv"], "kernel": kname["hv"],
                   "algorithmic_GBps": round(hv_gbs, 1), "bytes_per_cell_step": bpc["hv"]},
        },
        "ring_pass": {
            m: {"kernel": f"{m}_fused2_kernel", "ms_per_step": round(ring[m], 4),
                "MLUPS": round(ncell / (ring[m] * 1e-3) / 1e6, 2)} for m in ring},
        "single_step_kernels": {
            m: {"ms_per_step": round(single[m], 4), "MLUPS": round(ncell / (single[m] * 1e-3) / 1e6, 2),
                "bytes_per_cell_step": bpc1[m], "algorithmic_GBps": round(single_gbs[m], 1),
                "frac": round(single_gbs[m] / peak, 4)} for m in single},
        "roofline": roofline_entry("mm", kname["mm"], fused["mm"], bpc1["mm"], bpc["mm"], ncell, mm_ms, peak,
                                   peak_kind, traffic),
        "roofline_hv": roofline_entry("hv", kname["hv"], fused["hv"], bpc1["hv"], bpc["hv"], ncell, hv_ms, peak,
                                      peak_kind, hv_traffic),
        "l2_resident": l2,
        "l2_write_roofline": dict(l2_roof, note="L2 writes = stores from the SMs + fills from HBM; "
                                  "peak = l2_resident.write_GBps"),
        "cpu_baseline": {"value": round(cpu_mlups, 4), "unit": "Mcell-updates/s", "cores": cores, "kind": "oracle",
                         "sample": f"64^3 dipole lattice per model, FP64, {cpu_steps} steps, {cpu_s:.1f} s",
                         "single_thread": {"value": round(st_mlups, 4), "cores": 1,
                                           "sample": f"32^3 dipole lattice per model, {st_steps} steps, {st_s:.1f} s"}},
        "e2e": {"value": round(job_value(2 * ncell, e2e_steps, world, e2e_s), 2), "unit": "Mcell-updates/s",
                "h2d_bytes_per_step": h2d // e2e_steps, "d2h_bytes_per_step": d2h // e2e_steps,
                "job": f"lbm_init_fields from pinned host E, B + {e2e_steps} steps + lbm_fields E, B to pinned host memory"},
        "storage_variants": {
            st: {m: dict(v, frac=round(v["algorithmic_GBps"] / peak, 4)) for m, v in variants[st].items()}
            for st in variants},
        "rel_l2_vs_fp64_dielectric_pulse_1500": accuracy,
        "rel_l2_vs_fp64_slab_pulse_512x64x64": slab_accuracy,
        "refinement_batch": refinement,
        "adjoint": adjoint,
        "slab_decomposition_one_gpu": slabs,
        "gpu_launches": int(launches),
        "finite": finite,
        "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def time_slab_split(n_side: int, nz: int, steps: int, warmup: int, rank: int, world: int, stream):
    """One n_side^2 x nz dipole lattice per model split into `world` z-slabs, slab `rank` on this
    device: every step exchanges the halo with the neighbouring ranks (slabs.exchange: NCCL send and
    receive of packed faces; a single slab closes the ring on itself), then steps the slab once.
    Returns per-model step and exchange times (CUDA events on the slabs' stream, this rank) and the
    bytes each rank sends per step."""
    import torch
    from paper_2309_08068_gb300.slabs import SlabRank
    models = ("mm", "hv")
    with torch.cuda.stream(stream):
        parts = {m: SlabRank(wl.hertz_dipole(m, n=n_side, period=32.0, nz=nz), rank, world, stream=stream)
                 for m in models}
        for _ in range(warmup):
            for m in models:
                parts[m].step(1)
        torch.cuda.synchronize()
        events = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
        launches0 = sum(P.lattice.launch_count for P in parts.values())
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for ev in events:
            ev[0].record(stream)
            parts["mm"].step(1)
            ev[1].record(stream)
            parts["hv"].step(1)
            ev[2].record(stream)
        torch.cuda.synchronize()
        wall_s = time.perf_counter() - t0
        launches = sum(P.lattice.launch_count for P in parts.values()) - launches0
        per_model = {m: sum(e[k].elapsed_time(e[k + 1]) for e in events) / steps for k, m in enumerate(models)}
        elapsed_ms = events[0][0].elapsed_time(events[-1][2])
        # the exchange alone, for the record
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k = max(5, min(steps, 50))
        exch = {}
        for m in models:
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(k):
                parts[m].exchange()
            e1.record(stream)
            torch.cuda.synchronize()
            exch[m] = e0.elapsed_time(e1) / k
        # end to end through the C ABI: the slab's fields from pinned host memory, the steps, E and B
        # of the slab back to host memory
        slab_n = parts["mm"].lattice.n
        pinned = torch.zeros((3, slab_n), dtype=torch.float32).pin_memory()
        host_out = np.empty((2, 3, slab_n), np.float32)
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for P in parts.values():
            P.lattice._check(P.lattice.lib.lbm_init_fields(P.lattice.h, pinned.data_ptr(), pinned.data_ptr(), 0))
        for _ in range(steps):
            for m in models:
                parts[m].step(1)
        for P in parts.values():
            P.lattice._check(P.lattice.lib.lbm_fields(P.lattice.h, 3, host_out.ctypes.data, 0))
        e2e_s = time.perf_counter() - t0
    out = {"elapsed_ms": elapsed_ms, "wall_s": wall_s, "launches": launches, "per_model_ms": per_model,
           "e2e_s": e2e_s, "e2e_bytes": 2 * 2 * 3 * slab_n * 4,
           "exchange_ms": exch, "slab_planes": parts["mm"].bounds,
           "halo_bytes_sent_per_step": {m: 2 * P.lattice.halo_bytes for m, P in parts.items()},
           "finite": all(P.lattice.check_finite() for P in parts.values())}
    for P in parts.values():
        P.close()
    return out


def run_slabs(args):
    """--decomposition slabs under torchrun with N > 1: one lattice per model split across the ranks
    (strong scaling); rank 0 prints the line."""
    import torch
    import torch.distributed as dist
    world, rank, local = dist_info()
    torch.cuda.set_device(local)
    dist.init_process_group("nccl")
    n_side = args.n
    nz = args.nz or n_side
    ncell = n_side * n_side * nz
    stream = torch.cuda.Stream()
    with ClockSampler(local) as clocks:
        res = time_slab_split(n_side, nz, args.steps, args.warmup, rank, world, stream)
    elapsed_ms = max_over_ranks(res["elapsed_ms"], world)
    mm_ms = max_over_ranks(res["per_model_ms"]["mm"], world)
    hv_ms = max_over_ranks(res["per_model_ms"]["hv"], world)
    e2e_s = max_over_ranks(res["e2e_s"], world)
    if rank != 0:
        dist.destroy_process_group()
        return
    peak, peak_kind = hbm_peak()
    cells_rank = ncell // world
    bpc = {m: BYTES_PER_CELL[m] for m in BYTES_PER_CELL}
    cores = cpu_cores()
    cpu_mlups, cpu_steps, cpu_s = oracle_mlups(64, args.cpu_seconds, cores)
    line = {
        "metric": METRIC, "value": round(2 * ncell * args.steps / (elapsed_ms * 1e-3) / 1e6, 2),
        "unit": "Mcell-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(elapsed_ms / args.steps, 4), "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f32", "storage": "f32", "data": "synthetic",
        "config": {"workload": f"hertz_dipole_{n_side}x{n_side}x{nz}_mm+hv", "cells_per_model": ncell,
                   "step": "per model: halo exchange with both neighbours, then one step of the rank's slab",
                   "parallelism": f"z-slabs x{world} (one per rank), NCCL send/recv of packed faces",
                   "slab_planes_rank0": res["slab_planes"],
                   "l2": "inputs larger than L2 when the slab is"},
        "per_model": {m: {"ms_per_step": round(t, 4), "MLUPS": round(ncell / (t * 1e-3) / 1e6, 2),
                          "exchange_ms": round(res["exchange_ms"][m], 4),
                          "halo_bytes_sent_per_rank_step": res["halo_bytes_sent_per_step"][m]}
                      for m, t in (("mm", mm_ms), ("hv", hv_ms))},
        "roofline": {"bound": "hbm", "kernel": "mm_step_kernel (one step per launch on each slab)",
                     "achieved": round(bpc["mm"] * cells_rank / (mm_ms * 1e-3) / 1e9, 1), "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": round(bpc["mm"] * cells_rank / (mm_ms * 1e-3) / 1e9 / peak, 4),
                     "traffic": None, "note": "per rank, exchange included in the step time"},
        "cpu_baseline": {"value": round(cpu_mlups, 4), "unit": "Mcell-updates/s", "cores": cores, "kind": "oracle",
                         "sample": f"64^3 dipole lattice per model, FP64, {cpu_steps} steps, {cpu_s:.1f} s"},
        "e2e": {"value": round(2 * ncell * args.steps / e2e_s / 1e6, 2), "unit": "Mcell-updates/s",
                "h2d_bytes_per_step": res["e2e_bytes"] * world // args.steps,
                "d2h_bytes_per_step": res["e2e_bytes"] * world // args.steps,
                "job": f"per rank: lbm_init_fields of its slab from pinned host E, B + {args.steps} steps with "
                       "halo exchanges + lbm_fields E, B to host"},
        "gpu_launches": int(res["launches"]),
        "finite": res["finite"],
        "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)
    dist.destroy_process_group()


def roofline_entry(model, kernel, fused, bytes_update, bytes_own, ncell, ms_per_step, peak, peak_kind, traffic):
    """Roofline of one model's step kernel. `achieved` and `frac` count the method's algorithmic
    bytes per cell update (populations read and written once per step: 384 B MM, 288 B HV in FP32)
    over the measured time per step, so a two-step pass that keeps the intermediate step on chip can
    exceed 1. Beside it: the pass against its own minimum (the populations cross HBM once per pair
    of steps) and the ncu-measured DRAM traffic per launch over the same launch time."""
    steps_per_launch = 2 if fused else 1
    launch_s = steps_per_launch * ms_per_step * 1e-3
    achieved = bytes_update * ncell / (ms_per_step * 1e-3) / 1e9
    own = bytes_own * ncell / (ms_per_step * 1e-3) / 1e9
    entry = {"bound": "hbm",
             "kernel": kernel + (" (two steps per launch, sources included)" if fused else " (+ source-cell launch)"),
             "achieved": round(achieved, 1), "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
             "frac": round(achieved / peak, 4),
             "bytes_per_cell_update": bytes_update, "updates_per_launch": steps_per_launch * ncell,
             "launch_ms": round(launch_s * 1e3, 4),
             "traffic": None if traffic is None else round(traffic)}
    if fused:
        entry["own_minimum"] = {"bytes_per_cell_step": bytes_own, "achieved": round(own, 1),
                                "frac": round(own / peak, 4),
                                "note": "populations read and written once per two-step launch"}
    if traffic is not None:
        dram = traffic / launch_s / 1e9
        entry["dram_traffic"] = {"bytes_per_cell_launch": round(traffic / ncell, 1), "achieved": round(dram, 1),
                                 "frac": round(dram / peak, 4),
                                 "note": "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch (profiles/)"}
    return entry


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--nz", type=int, default=0, help="z extent of the timed lattices (default n: a cube)")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--fusion", type=int, choices=[0, 1, 2, 3], default=1,
                    help="lbm_set_step_fusion mode of the timed lattices: 0 one launch per step, 1 the two-step "
                         "pass measured fastest per model (default), 2 the ring pass, 3 the tiled pass")
    ap.add_argument("--slab-steps", type=int, default=50,
                    help="steps of the z-slab decomposition measurement on the dipole lattice (0 skips it)")
    ap.add_argument("--adjoint-steps", type=int, default=1000,
                    help="steps of the adjoint-cost measurement on the 128^3 random medium (0 skips it)")
    ap.add_argument("--refine-steps", type=int, default=100,
                    help="steps of the batched refinement-sweep measurement (0 skips it)")
    ap.add_argument("--slab-accuracy", type=int, default=1,
                    help="1: storage accuracy on the 512 x 64 x 64 slab pulse against the FP64 oracle (0 skips it)")
    ap.add_argument("--storage", choices=["f32", "bf16", "f16", "f24"], default="f32",
                    help="population storage of the main timed run (arithmetic is FP32 in every case)")
    ap.add_argument("--decomposition", choices=["replicas", "slabs"], default="replicas",
                    help="with N > 1 ranks: independent lattices per rank (replicas, weak scaling) or one "
                         "lattice per model split into N z-slabs with a halo exchange every step (slabs, "
                         "strong scaling). With one rank both are the unsplit lattice.")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        from paper_2309_08068_gb300 import build
        build.build()
        import oracle
        oracle.build()
        if args.decomposition == "slabs" and dist_info()[0] > 1:
            run_slabs(args)
        else:
            run_ours(args)


if __name__ == "__main__":
    main()
