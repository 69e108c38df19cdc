"""Python binding of liblbm.so (declared in include/lbm.h): argument marshalling only.

Every step of the MM / HV update runs in the library's CUDA kernels; this module converts arrays to
pointers and checks return codes. Device buffers are torch CUDA tensors (float32, contiguous); host
buffers are numpy arrays. There is no CPU fallback: creating a ``Lattice`` without the built
library or without a CUDA device raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from . import build as _build

LBM_MM, LBM_HV = 0, 1
MODELS = {"mm": LBM_MM, "hv": LBM_HV}
ERRORS = {0: "LBM_OK", -1: "LBM_EINVAL", -2: "LBM_ENOMEM", -3: "LBM_ECUDA", -4: "LBM_ENONFINITE",
          -5: "LBM_ETIMEDOUT", -6: "LBM_EUNSUPPORTED"}
FIELD_BITS = {"E": 1, "B": 2, "D": 4, "H": 8, "J": 16}
FIELD_ORDER = "EBDHJ"
FN_KINDS = {"sin": 0, "table": 1, "const": 2}
SRC_KINDS = {"current": 0, "impose": 1}
HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "lbm.h")


class LbmError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"{ERRORS.get(code, code)}: {message}")
        self.code = code


class _Media(ctypes.Structure):
    _fields_ = [("eps_r", ctypes.c_void_p), ("mu_r", ctypes.c_void_p), ("sigma", ctypes.c_void_p),
                ("on_device", ctypes.c_int)]


class _Options(ctypes.Structure):
    _fields_ = [("storage", ctypes.c_int), ("cuda_stream", ctypes.c_void_p), ("track_rho", ctypes.c_int),
                ("eps0", ctypes.c_double), ("mu0", ctypes.c_double), ("storage_scale", ctypes.c_double),
                ("z_ghost", ctypes.c_int)]


STORAGE = {"f32": 0, "bf16": 1, "f16": 2, "f24": 3}


class _TimeFn(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("amplitude", ctypes.c_double), ("period", ctypes.c_double),
                ("phase", ctypes.c_double), ("table", ctypes.c_void_p), ("table_len", ctypes.c_int64)]


class _Source(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n_cells", ctypes.c_int64), ("cells", ctypes.c_void_p),
                ("w", ctypes.c_void_p), ("E0", ctypes.c_float * 3), ("B0", ctypes.c_float * 3), ("fn", _TimeFn)]


_lib = None


def header_functions() -> list:
    """Names of the functions include/lbm.h declares."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(lbm_\w+)\s*\(", text, re.M)))


def load_library(path: str | None = None):
    """Load liblbm.so and declare its signatures. Raises if the library has not been built."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"liblbm.so is not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    sig = {
        "lbm_create": (I, [I, I, I, I, ctypes.POINTER(_Media), ctypes.POINTER(_Options), ctypes.POINTER(P)]),
        "lbm_init_fields": (I, [P, P, P, I]),
        "lbm_set_source": (I, [P, ctypes.POINTER(_Source)]),
        "lbm_clear_sources": (I, [P]),
        "lbm_step": (I, [P, I]),
        "lbm_fields": (I, [P, ctypes.c_uint, P, I]),
        "lbm_num_populations": (I, [I]),
        "lbm_get_populations": (I, [P, P, I]),
        "lbm_set_populations": (I, [P, P, I, I64]),
        "lbm_reduce": (I, [P, ctypes.POINTER(D)]),
        "lbm_check_finite": (I, [P]),
        "lbm_time": (I64, [P]),
        "lbm_launch_count": (I64, [P]),
        "lbm_last_error": (ctypes.c_char_p, [P]),
        "lbm_sync": (I, [P]),
        "lbm_destroy": (I, [P]),
        "lbm_adjoint": (I, [P, I, I, I, I, ctypes.POINTER(D), P, P, I]),
        "lbm_adjoint_release": (I, [P]),
        "lbm_set_step_fusion": (I, [P, I, I]),
        "lbm_step_fusion_active": (I, [P]),
        "lbm_set_wait_limit": (I, [P, ctypes.c_longlong]),
        "lbm_fused_schedule_check": (I, [I, I, I, I, I, I]),
        "lbm_tiled_layout_check": (I, [I, I]),
        "lbm_halo_bytes": (I64, [P]),
        "lbm_halo_pack": (I, [P, I, P, I]),
        "lbm_halo_unpack": (I, [P, I, P, I]),
        "lbm_halo_exchange": (I, [P, P]),
        "lbm_adjoint_workspace_bytes": (I64, [P]),
        "lbm_adjoint_sqrt_interval": (I, [P, I]),
        "lbm_batch_create": (I, [ctypes.POINTER(P), I, ctypes.POINTER(P)]),
        "lbm_batch_step": (I, [P, ctypes.POINTER(I)]),
        "lbm_batch_autotune": (I, [P, I, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "lbm_batch_set_config": (I, [P, I, I]),
        "lbm_batch_launch_count": (I64, [P]),
        "lbm_batch_last_error": (ctypes.c_char_p, [P]),
        "lbm_batch_destroy": (I, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path == _build.LIB:
        _lib = lib
    return lib


def _is_torch_cuda(x) -> bool:
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


def _as_f32(x, count: int, name: str):
    """Return (pointer, on_device, keepalive) for a float32 array of `count` values."""
    if _is_torch_cuda(x):
        import torch
        t = x.detach().to(torch.float32).contiguous()
        if t.numel() != count:
            raise ValueError(f"{name}: expected {count} values, got {t.numel()}")
        return t.data_ptr(), 1, t
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    if a.size != count:
        raise ValueError(f"{name}: expected {count} values, got {a.size}")
    return a.ctypes.data, 0, a


class Lattice:
    """A periodic nx x ny x nz lattice of the MM or HV model on the current CUDA device.

    ``stream``: a ``torch.cuda.Stream`` (default: torch's current stream). Media are per-cell
    arrays (numpy or torch CUDA), None for eps_r = mu_r = 1, sigma = 0.

    Device tensors passed in or returned are ordered against torch's current stream: the library's
    stream waits for what the current stream has queued before it reads or writes them, and the
    current stream waits for the library's work before the tensors are used there.
    """

    def __init__(self, model: str, shape, eps_r=None, mu_r=None, sigma=None, *, track_rho: bool = False,
                 eps0: float = 0.0, mu0: float = 0.0, stream=None, storage: str = "f32", storage_scale: float = 0.0,
                 z_ghost: bool = False):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Lattice needs a CUDA device; there is no CPU fallback")
        self.lib = load_library()
        self.model = model
        self.shape = tuple(int(s) for s in shape)
        nx, ny, nz = self.shape
        self.n = nx * ny * nz
        self.q = 50 if model == "mm" else 36
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        keep = []
        media = _Media(None, None, None, 0)
        on_dev = set()
        for field, arr in (("eps_r", eps_r), ("mu_r", mu_r), ("sigma", sigma)):
            if arr is None:
                continue
            ptr, dev, k = _as_f32(arr, self.n, field)
            keep.append(k)
            on_dev.add(dev)
            setattr(media, field, ptr)
        if len(on_dev) > 1:
            raise ValueError("media arrays must all be host or all device arrays")
        media.on_device = on_dev.pop() if on_dev else 0
        opts = _Options(STORAGE[storage], ctypes.c_void_p(self.stream.cuda_stream), int(track_rho), float(eps0),
                        float(mu0), float(storage_scale), int(z_ghost))
        self.storage = storage
        self.z_ghost = bool(z_ghost)
        h = ctypes.c_void_p()
        if media.on_device:
            self._inputs_ready()
        rc = self.lib.lbm_create(MODELS[model], nx, ny, nz, ctypes.byref(media), ctypes.byref(opts), ctypes.byref(h))
        if rc != 0:
            raise LbmError(rc, self.lib.lbm_last_error(None).decode())
        self.h = h
        if media.on_device:
            self._outputs_ready(*keep)

    # -- plumbing --------------------------------------------------------------------------
    def _inputs_ready(self):
        """The context stream waits for the work torch's current stream has queued (device inputs
        written there, output tensors allocated there)."""
        import torch
        cur = torch.cuda.current_stream(self.device)
        if cur != self.stream:
            self.stream.wait_stream(cur)

    def _outputs_ready(self, *tensors):
        """torch's current stream waits for the context stream, and each torch tensor's memory stays
        reserved until the context stream has finished with it."""
        import torch
        cur = torch.cuda.current_stream(self.device)
        if cur != self.stream:
            cur.wait_stream(self.stream)
            for t in tensors:
                if isinstance(t, torch.Tensor) and t.is_cuda:
                    t.record_stream(self.stream)

    def _check(self, rc: int):
        if rc != 0:
            raise LbmError(rc, self.lib.lbm_last_error(self.h).decode())

    def close(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            self.lib.lbm_destroy(h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def time(self) -> int:
        return int(self.lib.lbm_time(self.h))

    @property
    def launch_count(self) -> int:
        return int(self.lib.lbm_launch_count(self.h))

    def sync(self):
        self._check(self.lib.lbm_sync(self.h))

    # -- API -------------------------------------------------------------------------------
    def init_fields(self, E, B):
        pe, de, ke = _as_f32(E, 3 * self.n, "E")
        pb, db, kb = _as_f32(B, 3 * self.n, "B")
        if de != db:
            raise ValueError("E and B must both be host or both be device arrays")
        if de:
            self._inputs_ready()
        self._check(self.lib.lbm_init_fields(self.h, pe, pb, de))
        if de:
            self._outputs_ready(ke, kb)

    def add_source(self, src):
        """``src``: a ``workloads.Source``."""
        cells = np.ascontiguousarray(np.asarray(src.cells, dtype=np.int64).reshape(-1))
        w = None
        if src.kind == "current":
            w = np.ascontiguousarray(np.asarray(src.w, dtype=np.float32).reshape(-1))
            if w.size != 3 * cells.size:
                raise ValueError("current source needs 3 weights per cell")
        table = None
        if src.fn.kind == "table":
            table = np.ascontiguousarray(np.asarray(src.fn.table, dtype=np.float64).reshape(-1))
        fn = _TimeFn(FN_KINDS[src.fn.kind], float(src.fn.amplitude), float(src.fn.period), float(src.fn.phase),
                     None if table is None else table.ctypes.data, 0 if table is None else table.size)
        s = _Source(SRC_KINDS[src.kind], cells.size, cells.ctypes.data if cells.size else None,
                    None if w is None else w.ctypes.data, (ctypes.c_float * 3)(*[float(v) for v in src.E0]),
                    (ctypes.c_float * 3)(*[float(v) for v in src.B0]), fn)
        self._check(self.lib.lbm_set_source(self.h, ctypes.byref(s)))

    def clear_sources(self):
        self._check(self.lib.lbm_clear_sources(self.h))

    def step(self, n: int = 1):
        self._check(self.lib.lbm_step(self.h, int(n)))

    def fields(self, names: str = "EB", out=None) -> dict:
        """Fields at the current time as torch CUDA tensors (3, n), stream-ordered."""
        import torch
        names = "".join(c for c in FIELD_ORDER if c in names)
        mask = sum(FIELD_BITS[c] for c in names)
        if out is None:
            out = torch.empty((len(names), 3, self.n), dtype=torch.float32, device=self.device)
        self._inputs_ready()
        self._check(self.lib.lbm_fields(self.h, mask, out.data_ptr(), 1))
        self._outputs_ready(out)
        return {c: out[k] for k, c in enumerate(names)}

    def fields_host(self, names: str = "EB") -> dict:
        """Fields copied to host numpy arrays (3, n); waits for the stream."""
        names = "".join(c for c in FIELD_ORDER if c in names)
        mask = sum(FIELD_BITS[c] for c in names)
        out = np.empty((len(names), 3, self.n), dtype=np.float32)
        self._check(self.lib.lbm_fields(self.h, mask, out.ctypes.data, 0))
        return {c: out[k] for k, c in enumerate(names)}

    def populations(self):
        """Populations in the canonical layout, torch CUDA tensor (q, n)."""
        import torch
        out = torch.empty((self.q, self.n), dtype=torch.float32, device=self.device)
        self._inputs_ready()
        self._check(self.lib.lbm_get_populations(self.h, out.data_ptr(), 1))
        self._outputs_ready(out)
        return out

    def populations_host(self) -> np.ndarray:
        out = np.empty((self.q, self.n), dtype=np.float32)
        self._check(self.lib.lbm_get_populations(self.h, out.ctypes.data, 0))
        return out

    def set_populations(self, f, t: int = 0):
        p, dev, k = _as_f32(f, self.q * self.n, "populations")
        if dev:
            self._inputs_ready()
        self._check(self.lib.lbm_set_populations(self.h, p, dev, int(t)))
        if dev:
            self._outputs_ready(k)

    def reduce(self):
        """(field energy, sum of squared populations, MM total charge), double precision."""
        out = (ctypes.c_double * 3)()
        self._check(self.lib.lbm_reduce(self.h, out))
        return float(out[0]), float(out[1]), float(out[2])

    def adjoint(self, steps: int, plane_axis: int, plane_index: int, checkpoint_interval: int = 0,
                sigma: bool = True):
        """Advance `steps` steps and return (L, dL/d eps_r, dL/d sigma) for the plane loss
        L = sum_t sum_plane |E(t)|^2 (lbm_adjoint); gradients are torch CUDA tensors (n,).
        checkpoint_interval: the segment length K. < 0 keeps every step's record on the device; > 0
        records the final K steps in the forward pass and recomputes each earlier K-step segment
        once from a checkpoint; 0 picks the first when it fits in half the free memory, else
        K = sqrt_interval(steps). sigma=False skips dL/d sigma (returned as None)."""
        import torch
        ge = torch.empty(self.n, dtype=torch.float32, device=self.device)
        gs = torch.empty(self.n, dtype=torch.float32, device=self.device) if sigma else None
        loss = ctypes.c_double()
        self._inputs_ready()
        self._check(self.lib.lbm_adjoint(self.h, int(steps), int(plane_axis), int(plane_index), int(checkpoint_interval),
                                         ctypes.byref(loss), ge.data_ptr(), gs.data_ptr() if sigma else None, 1))
        self._outputs_ready(*(t for t in (ge, gs) if t is not None))
        return loss.value, ge, gs

    # -- two steps per pass ----------------------------------------------------------------------
    def set_step_fusion(self, mode: int, tile_cells: int = 0) -> None:
        """0: one launch per step; 1 (default, FP32 storage): pairs of steps as one pass, the tiled
        pass where it fills the GPU (HV with a uniform medium takes the ring pass first), else the
        L2-ring pass where it fits; 2: the ring pass wherever it applies; 3: the tiled pass wherever
        it applies. tile_cells: cells per work item of the ring pass (multiple of 256; 0 keeps the
        current value) (lbm_set_step_fusion)."""
        self._check(self.lib.lbm_set_step_fusion(self.h, int(mode), int(tile_cells)))

    def set_wait_limit(self, ns: int) -> None:
        """Limit of each dependency wait of a two-step pass in nanoseconds; 0 restores the default
        (2 s); negative: every dependent item gives up at once, for tests (lbm_set_wait_limit)."""
        self._check(self.lib.lbm_set_wait_limit(self.h, int(ns)))

    @property
    def step_fusion_active(self) -> bool:
        return self.pass_kind is not None

    @property
    def pass_kind(self):
        """The pass lbm_step would run pairs of steps as: "tiled", "ring", or None for single steps."""
        rc = int(self.lib.lbm_step_fusion_active(self.h))
        if rc < 0:
            self._check(rc)
        return {0: None, 1: "ring", 2: "tiled"}[rc]

    # -- z-slab halo (z_ghost lattices) ---------------------------------------------------------
    @property
    def halo_bytes(self) -> int:
        b = int(self.lib.lbm_halo_bytes(self.h))
        if b < 0:
            raise LbmError(b, "halo_bytes: not a z_ghost lattice")
        return b

    def halo_pack(self, face: int, out=None):
        """Outgoing populations of face 0 (down) or 1 (up) as a uint8 CUDA tensor (lbm_halo_pack)."""
        import torch
        if out is None:
            out = torch.empty(self.halo_bytes, dtype=torch.uint8, device=self.device)
        self._inputs_ready()
        self._check(self.lib.lbm_halo_pack(self.h, int(face), out.data_ptr(), 1))
        self._outputs_ready(out)
        return out

    def halo_unpack(self, face: int, data) -> None:
        """Write a neighbour's packed face into ghost plane 0 (face 0) or nz - 1 (face 1)."""
        if data.numel() * data.element_size() != self.halo_bytes or not data.is_cuda:
            raise ValueError("halo_unpack: need a CUDA buffer of halo_bytes bytes")
        self._inputs_ready()
        self._check(self.lib.lbm_halo_unpack(self.h, int(face), data.data_ptr(), 1))
        self._outputs_ready(data)

    def halo_exchange(self, upper: "Lattice") -> None:
        """Exchange across the interface between this slab (below) and `upper` (lbm_halo_exchange)."""
        self._check(self.lib.lbm_halo_exchange(self.h, upper.h))

    def adjoint_release(self) -> None:
        """Free the work space that adjoint() keeps between calls (lbm_adjoint_release)."""
        self._check(self.lib.lbm_adjoint_release(self.h))

    @property
    def adjoint_workspace_bytes(self) -> int:
        return int(self.lib.lbm_adjoint_workspace_bytes(self.h))

    def sqrt_interval(self, steps: int) -> int:
        """Segment length of the checkpointed adjoint for `steps` steps: the longest within the work
        space of the classic sqrt(T) layout (lbm_adjoint_sqrt_interval)."""
        k = int(self.lib.lbm_adjoint_sqrt_interval(self.h, int(steps)))
        if k < 0:
            self._check(k)
        return k

    def check_finite(self) -> bool:
        rc = self.lib.lbm_check_finite(self.h)
        if rc == -4:
            return False
        self._check(rc)
        return True


def lattice_from_workload(w, *, track_rho: bool = False, stream=None, init: bool = True, storage: str = "f32",
                          storage_scale: float = 0.0) -> Lattice:
    """Build a Lattice from a ``workloads.Workload``: media, sources and initial fields."""
    L = Lattice(w.model, w.shape, w.eps_r, w.mu_r, w.sigma, track_rho=track_rho, stream=stream, storage=storage,
                storage_scale=storage_scale)
    for s in w.sources:
        L.add_source(s)
    if init:
        E = np.zeros((3, w.n), np.float32) if w.E is None else w.E
        B = np.zeros((3, w.n), np.float32) if w.B is None else w.B
        L.init_fields(E, B)
    return L


class Batch:
    """Several lattices of one model and storage on one stream, stepped together (lbm_batch_*)."""

    def __init__(self, lattices):
        self.lattices = list(lattices)
        self.lib = load_library()
        arr = (ctypes.c_void_p * len(self.lattices))(*[L.h.value for L in self.lattices])
        h = ctypes.c_void_p()
        rc = self.lib.lbm_batch_create(arr, len(self.lattices), ctypes.byref(h))
        if rc != 0:
            raise LbmError(rc, self.lib.lbm_batch_last_error(None).decode())
        self.h = h

    def _check(self, rc):
        if rc != 0:
            raise LbmError(rc, self.lib.lbm_batch_last_error(self.h).decode())

    def step(self, steps):
        """Advance lattice k by steps[k] (an int applies to every lattice)."""
        if isinstance(steps, int):
            steps = [steps] * len(self.lattices)
        arr = (ctypes.c_int * len(self.lattices))(*[int(s) for s in steps])
        self._check(self.lib.lbm_batch_step(self.h, arr))

    def autotune(self, trial_steps: int = 5):
        block, persistent = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.lbm_batch_autotune(self.h, int(trial_steps), ctypes.byref(block), ctypes.byref(persistent)))
        return block.value, bool(persistent.value)

    def set_config(self, block: int, persistent: bool):
        self._check(self.lib.lbm_batch_set_config(self.h, int(block), int(persistent)))

    @property
    def launch_count(self) -> int:
        return int(self.lib.lbm_batch_launch_count(self.h))

    def close(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            self.lib.lbm_batch_destroy(h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plane_loss(model: str, shape, eps_r, sigma=None, *, populations=None, sources=(), steps: int, plane_axis: int,
               plane_index: int, t0: int = 0, checkpoint_interval: int = 0):
    """L = sum_{t=1..steps} sum over plane (plane_axis, plane_index) of |E(t)|^2, differentiable in
    eps_r (and sigma) with torch autograd. The gradient comes from the library's adjoint
    (lbm_adjoint), computed when the loss is evaluated. eps_r and sigma are per-cell CUDA tensors;
    the run starts from `populations` (canonical layout, default zero) at time t0."""
    import torch

    class _PlaneLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, eps, sig):
            L = Lattice(model, shape, eps_r=eps.detach(), sigma=None if sig is None else sig.detach())
            for s in sources:
                L.add_source(s)
            q = 50 if model == "mm" else 36
            f0 = populations if populations is not None else torch.zeros((q, L.n), device=eps.device)
            L.set_populations(f0, t0)
            loss, ge, gs = L.adjoint(steps, plane_axis, plane_index, checkpoint_interval)
            ctx.save_for_backward(ge, gs)
            ctx.has_sigma = sig is not None
            L.close()
            return torch.tensor(loss, dtype=torch.float64, device=eps.device)

        @staticmethod
        def backward(ctx, grad_out):
            ge, gs = ctx.saved_tensors
            g = grad_out.to(torch.float32)
            return g * ge, (g * gs if ctx.has_sigma else None)

    return _PlaneLoss.apply(eps_r, sigma)
