"""Thin Python binding of libicmpt.so (argument marshalling only).

Every step of the simulation runs in the library's CUDA kernels; this module
only converts numpy arrays / CUDA torch tensors into pointers and sizes.  If
the library has not been built, importing works but creating a Context raises
``RuntimeError``: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import sys
import os
import threading
import weakref
from dataclasses import dataclass

import numpy as np

from .inputs import CHIMERA, CUBIC3D, GAUSS, HYPERCUBIC4D, PM_J, SQUARE2D  # noqa: F401  (re-exported constants)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libicmpt.so")
DEVICE_PTR = 1
PENDING = 1          # icm_query / server results: work still running
CANCELLED = 2        # server results: the request was cancelled

_lock = threading.Lock()
_lib = None

_ERRORS = {-1: "ICM_ERR_ARG", -2: "ICM_ERR_OOM", -3: "ICM_ERR_BUDGET", -4: "ICM_ERR_CUDA",
           -5: "ICM_ERR_TIMEOUT", -6: "ICM_ERR_STATE", -7: "ICM_ERR_UNSUPPORTED"}


class IcmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRORS.get(code, code)}: {msg}")
        self.code = code


class Schedule(ctypes.Structure):
    _fields_ = [("icm_every", ctypes.c_int32), ("swap_every", ctypes.c_int32), ("enable_2a", ctypes.c_int32),
                ("enable_metropolis", ctypes.c_int32), ("t_meas", ctypes.c_int64), ("trace", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


EXPORTS = [
    "icm_ctx_create", "icm_ctx_create_ex", "icm_ctx_memory", "icm_ctx_destroy", "icm_last_error", "icm_sync", "icm_query", "icm_lattice_size",
    "icm_batch_create",
    "icm_batch_destroy", "icm_batch_load", "icm_set_schedule", "icm_get_schedule", "icm_run_sweeps",
    "icm_read_couplings", "icm_read_overlaps", "icm_read_icm_stats", "icm_read_cluster_masks", "icm_read_spins", "icm_read_energies", "icm_read_sweeps", "icm_read_observables",
    "icm_clear_observables",
    "icm_read_bond_counts", "icm_server_create", "icm_server_destroy", "icm_server_last_error",
    "icm_server_submit", "icm_server_step", "icm_server_poll", "icm_server_status", "icm_server_class_info",
    "icm_server_clock", "icm_server_cancel", "icm_batch_set_cluster", "icm_batch_cluster",
    "icm_batch_set_cluster_growth", "icm_batch_cluster_growth",
    "icm_read_trace", "icm_batch_info", "icm_energies_static", "icm_batch_set_slot", "icm_batch_set_active",
    "icm_batch_start_window", "icm_therm_update", "icm_batch_delta", "icm_batch_set_threads",
    "icm_batch_autotune", "icm_group_create", "icm_group_create_shared", "icm_group_info", "icm_group_run",
    "icm_group_destroy", "icm_percolation",
    "icm_percolation_random", "icm_set_temperatures", "icm_save", "icm_load",
]


class ThermState(ctypes.Structure):
    _fields_ = [("blocks", ctypes.c_int32), ("stable", ctypes.c_int32), ("e", ctypes.c_double * 3),
                ("ql", ctypes.c_double * 3), ("delta", ctypes.c_double)]


class ThermCriterion(ctypes.Structure):
    _fields_ = [("eps_e", ctypes.c_double), ("eps_ql", ctypes.c_double), ("need", ctypes.c_int32)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("slots_per_class", ctypes.c_int32), ("quantum", ctypes.c_int32), ("max_sweeps", ctypes.c_uint32),
                ("crit", ThermCriterion), ("hbm_budget", ctypes.c_uint64)]


class _Request(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int32), ("L", ctypes.c_int32), ("disorder", ctypes.c_int32),
                ("n_T", ctypes.c_int32), ("T", ctypes.c_void_p), ("T_icm", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("instance_id", ctypes.c_uint32), ("couplings", ctypes.c_void_p),
                ("spins", ctypes.c_void_p)]


class ServerResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("thermalized", ctypes.c_int32), ("sweeps", ctypes.c_uint32),
                ("slot", ctypes.c_int32), ("e", ctypes.c_double), ("q_l", ctypes.c_double),
                ("delta", ctypes.c_double), ("accE", ctypes.c_double), ("acc_d", ctypes.c_int64),
                ("n_meas", ctypes.c_int64), ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double)]


def load_library(path: str = LIB_PATH):
    """Load libicmpt.so; raises RuntimeError when it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"libicmpt.so not built ({path}); run paper_1501_05630_gb300.build.build()")
        L = ctypes.CDLL(path)
        vp, i32, u32, u64, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64
        L.icm_ctx_create.argtypes = [ctypes.POINTER(vp), i32, vp]
        L.icm_ctx_create_ex.argtypes = [ctypes.POINTER(vp), i32, vp, ctypes.c_size_t, vp]
        L.icm_ctx_memory.argtypes = [vp, vp, vp]
        L.icm_ctx_destroy.argtypes = [vp]
        L.icm_last_error.argtypes = [vp]
        L.icm_last_error.restype = ctypes.c_char_p
        L.icm_sync.argtypes = [vp]
        L.icm_query.argtypes = [vp]
        L.icm_lattice_size.argtypes = [i32, i32, vp, vp]
        L.icm_batch_create.argtypes = [vp, i32, i32, i32, i32, vp, vp, vp, vp, i32, ctypes.c_double, u64, u32,
                                       ctypes.POINTER(vp)]
        L.icm_batch_destroy.argtypes = [vp]
        L.icm_batch_load.argtypes = [vp, vp, vp, u32, u32]
        L.icm_set_schedule.argtypes = [vp, ctypes.POINTER(Schedule)]
        L.icm_get_schedule.argtypes = [vp, ctypes.POINTER(Schedule)]
        L.icm_run_sweeps.argtypes = [vp, u32]
        L.icm_read_spins.argtypes = [vp, vp, u32]
        L.icm_read_couplings.argtypes = [vp, vp, u32]
        L.icm_read_cluster_masks.argtypes = [vp, vp]
        L.icm_read_overlaps.argtypes = [vp, vp, vp, vp, vp]
        L.icm_read_icm_stats.argtypes = [vp, vp, u32]
        L.icm_read_energies.argtypes = [vp, vp, u32]
        L.icm_read_sweeps.argtypes = [vp, vp, u32]
        L.icm_read_observables.argtypes = [vp] + [vp] * 7 + [u32]
        L.icm_read_bond_counts.argtypes = [vp, vp]
        L.icm_server_create.argtypes = [i32, ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]
        L.icm_server_destroy.argtypes = [vp]
        L.icm_server_last_error.argtypes = [vp]
        L.icm_server_last_error.restype = ctypes.c_char_p
        L.icm_server_submit.argtypes = [vp, ctypes.POINTER(_Request), ctypes.POINTER(u64)]
        L.icm_server_step.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
        L.icm_server_poll.argtypes = [vp, u64, ctypes.POINTER(ServerResult)]
        L.icm_server_status.argtypes = [vp] + [ctypes.POINTER(i32)] * 3
        L.icm_server_class_info.argtypes = [vp, i32] + [ctypes.POINTER(i32)] * 6
        L.icm_server_cancel.argtypes = [vp, u64]
        L.icm_server_clock.argtypes = []
        L.icm_server_clock.restype = ctypes.c_double
        L.icm_clear_observables.argtypes = [vp]
        L.icm_read_trace.argtypes = [vp] + [vp] * 7 + [u32]
        L.icm_batch_info.argtypes = [vp] + [vp] * 5
        L.icm_energies_static.argtypes = [vp, i32, i32, i32, i32, i32, vp, vp, vp]
        L.icm_batch_set_slot.argtypes = [vp, i32, vp, vp, u32, u32]
        L.icm_batch_set_active.argtypes = [vp, i32, i32]
        L.icm_batch_start_window.argtypes = [vp, i32, i64]
        L.icm_therm_update.argtypes = [ctypes.POINTER(ThermState), ctypes.POINTER(ThermCriterion),
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.POINTER(i32)]
        L.icm_batch_delta.argtypes = [vp, i32, vp, vp, vp]
        L.icm_batch_set_threads.argtypes = [vp, i32]
        L.icm_batch_autotune.argtypes = [vp, u32, vp, vp]
        L.icm_group_create.argtypes = [vp, vp, i32, u32, ctypes.POINTER(vp)]
        L.icm_group_create_shared.argtypes = [vp, vp, i32, u32, vp, ctypes.POINTER(vp)]
        L.icm_group_info.argtypes = [vp, vp, vp, vp, vp, vp]
        L.icm_group_run.argtypes = [vp, u32]
        L.icm_group_destroy.argtypes = [vp]
        L.icm_percolation.argtypes = [vp, i32, i32, i32, vp, vp, u32]
        L.icm_percolation_random.argtypes = [vp, i32, i32, ctypes.c_double, u64, i32, vp, u32]
        L.icm_set_temperatures.argtypes = [vp, vp, i32, ctypes.c_double]
        L.icm_save.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_size_t)]
        L.icm_load.argtypes = [vp, vp, ctypes.c_size_t]
        for name in EXPORTS:
            if name not in ("icm_last_error", "icm_server_last_error", "icm_server_clock"):
                getattr(L, name).restype = i32
        _ = i64
        _lib = L
        return L


def lattice_size(lattice: int, L: int):
    lib = load_library()
    n, nb = ctypes.c_int32(), ctypes.c_int32()
    rc = lib.icm_lattice_size(lattice, L, ctypes.byref(n), ctypes.byref(nb))
    if rc:
        raise IcmError(rc, "bad lattice")
    return n.value, nb.value


def _ptr(a):
    """(pointer, flags) of a numpy array or a CUDA torch tensor."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr(), (DEVICE_PTR if a.is_cuda else 0)
    raise TypeError(f"unsupported buffer type {type(a)}")


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p)


class _Allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("user", ctypes.c_void_p)]


def _torch_allocator() -> _Allocator:
    """Hooks that hand the library's device memory to PyTorch's caching
    allocator (blocks tied to the context's stream)."""
    import torch

    def alloc(nbytes, device, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), int(device), int(stream or 0))
        except Exception:          # out of memory: the library reports ICM_ERR_OOM
            return None

    def free(ptr, nbytes, device, stream, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    return _Allocator(_ALLOC_FN(alloc), _FREE_FN(free), None)


class Context:
    """A device and a stream (a cudaStream_t handle as int, or None).

    hbm_budget: device bytes the context's batches may hold at once (0 = no
    limit; past it calls fail with ICM_ERR_BUDGET).  allocator: None
    (cudaMalloc) or "torch" (PyTorch's caching allocator owns the memory)."""

    def __init__(self, device: int = 0, stream=None, hbm_budget: int = 0, allocator=None):
        self._lib = load_library()
        h = ctypes.c_void_p()
        st = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        self._alloc = None
        if hbm_budget or allocator is not None:
            if allocator not in (None, "torch"):
                raise ValueError("allocator must be None or 'torch'")
            self._alloc = _torch_allocator() if allocator == "torch" else None
            rc = self._lib.icm_ctx_create_ex(ctypes.byref(h), int(device), st, int(hbm_budget),
                                             None if self._alloc is None else ctypes.byref(self._alloc))
        else:
            rc = self._lib.icm_ctx_create(ctypes.byref(h), int(device), st)
        if rc:
            raise IcmError(rc, "icm_ctx_create failed (no CUDA device?)")
        self.device = int(device)
        self._h = h
        self._batches = weakref.WeakSet()

    def memory(self):
        """(device bytes held by the context's batches, budget or 0)."""
        used, budget = ctypes.c_size_t(), ctypes.c_size_t()
        self.check(self._lib.icm_ctx_memory(self._h, ctypes.byref(used), ctypes.byref(budget)))
        return used.value, budget.value

    def check(self, rc: int):
        if rc:
            raise IcmError(rc, self._lib.icm_last_error(self._h).decode())

    def sync(self):
        self.check(self._lib.icm_sync(self._h))

    def query(self) -> bool:
        """True when all work enqueued on the context's stream has finished."""
        rc = self._lib.icm_query(self._h)
        if rc == PENDING:
            return False
        self.check(rc)
        return True

    def close(self):
        if getattr(self, "_h", None):
            for b in list(self._batches):      # the library frees them with the context
                b._h = None
            self._lib.icm_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        # at interpreter exit PyTorch may already be torn down: a context whose
        # memory it owns is left to the process exit instead of freed through it
        if self._alloc_is_torch() and sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass

    def _alloc_is_torch(self) -> bool:
        return getattr(self, "_alloc", None) is not None


def largest_clusters(ctx: Context, lattice: int, L: int, masks) -> np.ndarray:
    """Largest occupied cluster of each mask [n][N] (site percolation)."""
    N, _ = lattice_size(lattice, L)
    m = masks if hasattr(masks, "data_ptr") else np.ascontiguousarray(masks, dtype=np.uint8).reshape(-1, N)
    n = int(m.shape[0])
    mp, f = _ptr(m)
    if f:
        import torch
        out_t = torch.empty(n, dtype=torch.int32, device=m.device)
        ctx.check(ctx._lib.icm_percolation(ctx._h, int(lattice), int(L), n, mp, out_t.data_ptr(), f))
        return out_t.cpu().numpy()
    out = np.empty(n, dtype=np.int32)
    ctx.check(ctx._lib.icm_percolation(ctx._h, int(lattice), int(L), n, mp, out.ctypes.data, 0))
    return out


def largest_clusters_random(ctx: Context, lattice: int, L: int, p: float, seed: int, n_masks: int) -> np.ndarray:
    """Largest cluster of n_masks random masks (occupation p) drawn on the device."""
    out = np.empty(int(n_masks), dtype=np.int32)
    ctx.check(ctx._lib.icm_percolation_random(ctx._h, int(lattice), int(L), float(p),
                                              int(seed) & 0xFFFFFFFFFFFFFFFF, int(n_masks), out.ctypes.data, 0))
    return out


def therm_update(state: ThermState, crit: ThermCriterion, e: float, q_l: float, T_min: float,
                 bonds_per_site: float) -> bool:
    """One window of the per-instance thermalization test (host only)."""
    lib = load_library()
    out = ctypes.c_int32()
    rc = lib.icm_therm_update(ctypes.byref(state), ctypes.byref(crit), float(e), float(q_l), float(T_min),
                              float(bonds_per_site), ctypes.byref(out))
    if rc:
        raise IcmError(rc, "icm_therm_update")
    return bool(out.value)


def _check_static_args(device: int, N: int, Nb: int, disorder: int, couplings, spins, out):
    """Shapes, dtypes and device of the energies_static tensors: the library
    reads and writes exactly [n_inst][N_b] couplings (int8 for +-J, float32
    for Gaussian), [n_inst][n_rep][N] int8 spins and [n_inst][n_rep] float64
    energies, so any other shape or dtype would be read or written past the
    caller's buffers on the device.  Returns (n_inst, n_rep)."""
    names = ("couplings", "spins", "out")
    for name, a in zip(names, (couplings, spins, out)):
        if not (hasattr(a, "is_cuda") and a.is_cuda and a.is_contiguous()):
            raise ValueError(f"energies_static: {name} must be a contiguous CUDA tensor")
        dev = getattr(a, "device", None)
        if getattr(dev, "index", device) not in (None, device):
            raise ValueError(f"energies_static: {name} is on {dev}, the context is on cuda:{device}")
    if len(spins.shape) != 3 or int(spins.shape[2]) != N:
        raise ValueError(f"energies_static: spins must be [n_inst][n_rep][{N}], got {tuple(spins.shape)}")
    n_inst, n_rep = int(spins.shape[0]), int(spins.shape[1])
    want_j = "torch.float32" if disorder == GAUSS else "torch.int8"
    if str(couplings.dtype) != want_j or tuple(couplings.shape) != (n_inst, Nb):
        raise ValueError(f"energies_static: couplings must be {want_j} [{n_inst}][{Nb}], "
                         f"got {couplings.dtype} {tuple(couplings.shape)}")
    if str(spins.dtype) != "torch.int8":
        raise ValueError(f"energies_static: spins must be torch.int8, got {spins.dtype}")
    if str(out.dtype) != "torch.float64" or tuple(out.shape) != (n_inst, n_rep):
        raise ValueError(f"energies_static: out must be torch.float64 [{n_inst}][{n_rep}], "
                         f"got {out.dtype} {tuple(out.shape)}")
    return n_inst, n_rep


def energies_static(ctx: Context, lattice: int, L: int, disorder: int, couplings, spins, out):
    """Energies [n_inst][n_rep] of device spin arrays, computed on the library's
    fixed device scratch (no device allocation; see icm_energies_static).
    Raises ValueError before any device work when a tensor's shape, dtype or
    device does not match the lattice, the disorder kind and the context."""
    if disorder not in (PM_J, GAUSS):
        raise ValueError("energies_static: disorder must be PM_J or GAUSS")
    N, Nb = lattice_size(lattice, L)
    n_inst, n_rep = _check_static_args(ctx.device, N, Nb, disorder, couplings, spins, out)
    ctx.check(ctx._lib.icm_energies_static(ctx._h, int(lattice), int(L), int(disorder), n_inst, n_rep,
                                           couplings.data_ptr(), spins.data_ptr(), out.data_ptr()))
    return out


@dataclass
class Observables:
    accE: np.ndarray
    acc_n: np.ndarray
    acc_q2: np.ndarray
    acc_pmin: np.ndarray
    acc_d: np.ndarray
    hist: np.ndarray
    n_meas: np.ndarray
    nb: np.ndarray | None = None      # bonds present per instance (the q_l normalisation)


class Batch:
    """n_inst disorder instances sharing one lattice, disorder kind and ladder.

    couplings [n_inst][N_b] (host array or device tensor), or None: the
    library draws them from the seed and the instance ids (then give n_inst
    or instance_ids)."""

    def __init__(self, ctx: Context, lattice: int, L: int, disorder: int, couplings, T, T_icm: float,
                 seed: int, spins=None, instance_ids=None, n_inst=None):
        self.ctx = ctx
        self._lib = ctx._lib
        self.lattice, self.L, self.disorder = int(lattice), int(L), int(disorder)
        self.N, self.Nb = lattice_size(lattice, L)
        self.T = np.ascontiguousarray(T, dtype=np.float64)
        self.nT = len(self.T)
        self.R = 2 * self.nT
        if couplings is not None:
            n_inst = couplings.shape[0]
        elif n_inst is None:
            if instance_ids is None:
                raise ValueError("without couplings, give n_inst or instance_ids")
            n_inst = len(instance_ids)
        self.n_inst = int(n_inst)
        cp, cflags = _ptr(couplings)
        sp, sflags = _ptr(spins)
        if spins is not None and couplings is not None and cflags != sflags:
            raise ValueError("couplings and spins must both be host or both be device buffers")
        ids = None if instance_ids is None else np.ascontiguousarray(instance_ids, dtype=np.uint32)
        h = ctypes.c_void_p()
        ctx.check(self._lib.icm_batch_create(
            ctx._h, self.lattice, self.L, self.disorder, self.n_inst, cp, sp,
            None if ids is None else ids.ctypes.data, self.T.ctypes.data, self.nT, float(T_icm),
            int(seed) & 0xFFFFFFFFFFFFFFFF, cflags | sflags, ctypes.byref(h)))
        self._h = h
        ctx._batches.add(self)

    # -- control
    def schedule(self) -> Schedule:
        s = Schedule()
        self.ctx.check(self._lib.icm_get_schedule(self._h, ctypes.byref(s)))
        return s

    def set_schedule(self, **kw):
        s = self.schedule()
        for k, v in kw.items():
            setattr(s, k, int(v))
        self.ctx.check(self._lib.icm_set_schedule(self._h, ctypes.byref(s)))

    def checkpoint(self) -> bytes:
        """Checkpoint of the batch state (a versioned blob)."""
        n = ctypes.c_size_t()
        self.ctx.check(self._lib.icm_save(self._h, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        self.ctx.check(self._lib.icm_save(self._h, buf, ctypes.byref(n)))
        return buf.raw[: n.value]

    def restore(self, blob: bytes):
        """Restore a checkpoint taken from a batch of the same shape and seed."""
        buf = ctypes.create_string_buffer(blob, len(blob))
        self.ctx.check(self._lib.icm_load(self._h, buf, len(blob)))

    def set_temperatures(self, T, T_icm: float):
        T = np.ascontiguousarray(T, dtype=np.float64)
        self.ctx.check(self._lib.icm_set_temperatures(self._h, T.ctypes.data, len(T), float(T_icm)))
        self.T = T

    def run(self, n_sweeps: int):
        self.ctx.check(self._lib.icm_run_sweeps(self._h, int(n_sweeps)))

    def load(self, couplings=None, spins=None, t0: int = 0):
        cp, cf = _ptr(couplings)
        sp, sf = _ptr(spins)
        self.ctx.check(self._lib.icm_batch_load(self._h, cp, sp, int(t0), cf | sf))

    def clear_observables(self):
        self.ctx.check(self._lib.icm_clear_observables(self._h))

    # -- serving: per-slot control
    def set_slot(self, slot: int, couplings, spins=None, instance_id: int = 0):
        cp, cf = _ptr(couplings)
        sp, sf = _ptr(spins)
        self.ctx.check(self._lib.icm_batch_set_slot(self._h, int(slot), cp, sp, int(instance_id), cf | sf))

    def set_active(self, slot: int, active: bool):
        self.ctx.check(self._lib.icm_batch_set_active(self._h, int(slot), int(bool(active))))

    def start_window(self, slot: int, t_start: int):
        self.ctx.check(self._lib.icm_batch_start_window(self._h, int(slot), int(t_start)))

    def delta(self, k: int = 0):
        """Eq. 2 over the batch at temperature position k: (mean, standard error, instances)."""
        m, se, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
        self.ctx.check(self._lib.icm_batch_delta(self._h, int(k), ctypes.byref(m), ctypes.byref(se),
                                                 ctypes.byref(n)))
        return m.value, se.value, n.value

    # -- reads
    def read_couplings(self, out=None):
        """Couplings [n_inst][N_b] as loaded or drawn (int8 +-J, float32 Gaussian)."""
        if out is None:
            out = np.empty((self.n_inst, self.Nb), dtype=np.float32 if self.disorder == GAUSS else np.int8)
        p, f = _ptr(out)
        self.ctx.check(self._lib.icm_read_couplings(self._h, p, f))
        return out

    def read_overlaps(self, hist: bool = True):
        """(q_mean, q2_mean, ql_mean, q_hist) per instance and temperature (see icm_read_overlaps)."""
        shape = (self.n_inst, self.nT)
        q, q2, ql = (np.empty(shape, dtype=np.float64) for _ in range(3))
        h = np.empty(shape + (self.N + 1,), dtype=np.int64) if hist else None
        self.ctx.check(self._lib.icm_read_overlaps(self._h, q.ctypes.data, q2.ctypes.data, ql.ctypes.data,
                                                   None if h is None else h.ctypes.data))
        return q, q2, ql, h

    def read_icm_stats(self) -> np.ndarray:
        """[n_inst][2] uint64: cluster moves (pairs with n > 0) and growth
        scans since the last clear (see icm_read_icm_stats)."""
        out = np.empty((self.n_inst, 2), dtype=np.uint64)
        self.ctx.check(self._lib.icm_read_icm_stats(self._h, out.ctypes.data, 0))
        return out

    def read_cluster_masks(self) -> np.ndarray:
        """[n_inst][n_T][N] uint8: the clusters moved in the last traced sweep."""
        out = np.zeros((self.n_inst, self.nT, self.N), dtype=np.uint8)
        self.ctx.check(self._lib.icm_read_cluster_masks(self._h, out.ctypes.data))
        return out

    def read_spins(self, out=None):
        if out is None:
            out = np.empty((self.n_inst, self.R, self.N), dtype=np.int8)
        p, f = _ptr(out)
        self.ctx.check(self._lib.icm_read_spins(self._h, p, f))
        return out

    def read_energies(self, out=None):
        if out is None:
            out = np.empty((self.n_inst, self.R), dtype=np.float64)
        p, f = _ptr(out)
        self.ctx.check(self._lib.icm_read_energies(self._h, p, f))
        return out

    def read_sweeps(self):
        out = np.empty(self.n_inst, dtype=np.uint32)
        self.ctx.check(self._lib.icm_read_sweeps(self._h, out.ctypes.data, 0))
        return out

    def read_observables(self, hist: bool = True) -> Observables:
        n, nT = self.n_inst, self.nT
        o = Observables(np.empty((n, nT)), *[np.empty((n, nT), np.int64) for _ in range(4)],
                        np.empty((n, nT, self.N + 1), np.int64) if hist else None, np.empty(n, np.int64))
        self.ctx.check(self._lib.icm_read_observables(
            self._h, o.accE.ctypes.data, o.acc_n.ctypes.data, o.acc_q2.ctypes.data, o.acc_pmin.ctypes.data,
            o.acc_d.ctypes.data, o.hist.ctypes.data if hist else None, o.n_meas.ctypes.data, 0))
        o.nb = self.bond_counts()
        return o

    def bond_counts(self) -> np.ndarray:
        """Bonds present (coupling != 0) per instance; N_b unless diluted."""
        out = np.empty(self.n_inst, dtype=np.int32)
        self.ctx.check(self._lib.icm_read_bond_counts(self._h, out.ctypes.data))
        return out

    def read_trace(self) -> dict:
        n, nT = self.n_inst, self.nT
        tr = dict(n_pre=np.empty((n, nT), np.int32), flip2a=np.empty((n, nT), np.int32),
                  seed_site=np.empty((n, nT), np.int32), csize=np.empty((n, nT), np.int32),
                  esum_before=np.empty((n, nT)), esum_after=np.empty((n, nT)),
                  swap_acc=np.empty((n, 2, nT - 1), np.uint8))
        self.ctx.check(self._lib.icm_read_trace(self._h, *[tr[k].ctypes.data for k in (
            "n_pre", "flip2a", "seed_site", "csize", "esum_before", "esum_after", "swap_acc")], 0))
        return tr

    def set_threads(self, threads: int):
        self.ctx.check(self._lib.icm_batch_set_threads(self._h, int(threads)))

    def set_cluster(self, K: int, threads: int):
        """One instance per thread-block cluster of K CTAs (K = 0: one CTA per instance)."""
        self.ctx.check(self._lib.icm_batch_set_cluster(self._h, int(K), int(threads)))

    def cluster(self) -> int:
        k = ctypes.c_int32()
        self.ctx.check(self._lib.icm_batch_cluster(self._h, ctypes.byref(k)))
        return k.value

    def set_cluster_growth(self, mode: int):
        """Cluster growth of the thread-block-cluster layout: 1 union-find,
        0 label propagation by scans, -1 the library's choice (propagation)."""
        self.ctx.check(self._lib.icm_batch_set_cluster_growth(self._h, int(mode)))

    def cluster_growth(self) -> int:
        """Pairs per union-find group (0: label propagation or not clustered)."""
        g = ctypes.c_int32()
        self.ctx.check(self._lib.icm_batch_cluster_growth(self._h, ctypes.byref(g)))
        return g.value

    def autotune(self, sweeps: int = 16):
        """Pick the fastest CTA width; the batch's state is left unchanged."""
        th, ms = ctypes.c_int32(), ctypes.c_float()
        self.ctx.check(self._lib.icm_batch_autotune(self._h, int(sweeps), ctypes.byref(th), ctypes.byref(ms)))
        return th.value, ms.value

    def info(self) -> dict:
        t, c, g, s = (ctypes.c_int32() for _ in range(4))
        la = ctypes.c_int64()
        self.ctx.check(self._lib.icm_batch_info(self._h, ctypes.byref(t), ctypes.byref(c), ctypes.byref(g),
                                                ctypes.byref(s), ctypes.byref(la)))
        return dict(threads=t.value, ctas_per_sm=c.value, grid=g.value, smem_bytes=s.value, launches=la.value)

    def close(self):
        """Free the batch (refused while a Group holds it: close the group first)."""
        if getattr(self, "_h", None) and getattr(self.ctx, "_h", None):
            self.ctx.check(self._lib.icm_batch_destroy(self._h))
        self._h = None

    def __del__(self):
        if self.ctx._alloc_is_torch() and sys.is_finalizing():
            return                              # see Context.__del__
        try:
            self.close()
        except Exception:
            pass


SHARED_WIDTHS = (32, 64, 128, 224, 448, 896)   # threads per instance of the shared group kernel (divisors of 896)


def tune_shared_widths(ctx: Context, batches, sweeps: int = 16, widths=SHARED_WIDTHS):
    """Threads per instance (and with them the instances per tile) of each
    batch for the shared group kernel, by timing: each batch alone in a
    shared group at every width that fits, one untimed and one timed launch
    of `sweeps` sweeps; the fastest width per spin update wins.  Every
    batch's state is restored from a checkpoint afterwards, so tuning does
    not advance the chains (the cluster-move counters of icm_read_icm_stats
    are not part of a checkpoint: they keep the tuning launches' counts).
    Returns (widths, {batch index: {width: ms}})."""
    import time
    best, table = [], {}
    for c, b in enumerate(batches):
        blob = b.checkpoint()
        times = {}
        for w in widths:
            try:
                g = Group(ctx, [b], sweeps, shared=True, team_threads=[w])
            except IcmError:
                continue
            g.run(1)
            ctx.sync()
            t0 = time.perf_counter()
            g.run(1)
            ctx.sync()
            times[w] = (time.perf_counter() - t0) * 1e3
            g.close()
        b.restore(blob)
        if not times:
            raise IcmError(-7, f"batch {c}: no width fits the shared group kernel")
        table[c] = times
        best.append(min(times, key=times.get))
    return best, table


class Group:
    """Several batches replayed as one CUDA graph.  shared=False: one kernel
    per batch on forked streams (icm_group_create); shared=True: the
    instances of every batch share one persistent kernel launch, each run by
    a team of team_threads[c] threads (icm_group_create_shared; None picks
    the widths)."""

    def __init__(self, ctx: Context, batches, sweeps_per_launch: int, shared: bool = False, team_threads=None):
        self.ctx, self._lib, self.batches = ctx, ctx._lib, list(batches)
        arr = (ctypes.c_void_p * len(self.batches))(*[b._h for b in self.batches])
        h = ctypes.c_void_p()
        if shared:
            tt = None
            if team_threads is not None:
                tt = np.ascontiguousarray(team_threads, dtype=np.int32)
                if tt.shape != (len(self.batches),):
                    raise ValueError("team_threads: one entry per batch")
            ctx.check(self._lib.icm_group_create_shared(ctx._h, arr, len(self.batches), int(sweeps_per_launch),
                                                        None if tt is None else tt.ctypes.data, ctypes.byref(h)))
        else:
            ctx.check(self._lib.icm_group_create(ctx._h, arr, len(self.batches), int(sweeps_per_launch),
                                                 ctypes.byref(h)))
        self._h = h
        self.shared = bool(shared)
        self.sweeps = int(sweeps_per_launch)

    def info(self) -> dict:
        """Threads per instance and instances per tile of each batch; grid,
        shared memory per CTA and tiles of the shared kernel."""
        n = len(self.batches)
        tt, tile = np.zeros(n, np.int32), np.zeros(n, np.int32)
        g, sm, it = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        self.ctx.check(self._lib.icm_group_info(self._h, tt.ctypes.data, tile.ctypes.data, ctypes.byref(g),
                                                ctypes.byref(sm), ctypes.byref(it)))
        return dict(team_threads=tt.tolist(), tile=tile.tolist(), grid=g.value, smem_bytes=sm.value,
                    n_items=it.value)

    def run(self, n_launches: int = 1):
        self.ctx.check(self._lib.icm_group_run(self._h, int(n_launches)))

    def close(self):
        if getattr(self, "_h", None) and getattr(self.ctx, "_h", None):
            self._lib.icm_group_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
