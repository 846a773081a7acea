"""Continuous-batching request server: disorder instances run to thermalization.

The Python face of the library's native request server (``icm_server_*`` in
``include/icmpt.h``).  Requests -- one disorder instance each, any lattice
kind and size the library supports -- are grouped by shape (lattice, size,
disorder kind, temperature ladder, T_icm, seed) into classes; each class is
one slot-table batch on its own CUDA stream.  One ``step`` of the native loop

  1. admits queued requests into free slots of idle classes while the
     device-memory budget allows (a class's batch is created when its first
     request arrives);
  2. collects every class whose last launch has finished (a non-blocking
     query of its stream), advances its slots by ``quantum`` sweeps and, at
     each slot that reached the end of a doubling window [2^(b-1) Q, 2^b Q),
     applies the thermalization test at the lowest temperature
     (icm_therm_update), then finishes the request (freeing the slot) or
     starts the next window;
  3. launches the next ``quantum`` simulation steps of every idle class with
     active slots.  Classes advance independently, so a class of large
     lattices does not hold back the small ones.

The random streams are keyed by (seed, instance id) only, so a request's
trajectory does not depend on its slot or on the other requests in the mix.
This module only converts requests and results; the loop runs in C++.
"""
from __future__ import annotations

import ctypes
import time
from dataclasses import dataclass

import numpy as np

from . import icmpt


@dataclass
class Request:
    lattice: int
    L: int
    disorder: int
    T: np.ndarray
    T_icm: float
    seed: int
    instance_id: int
    couplings: np.ndarray | None   # None: drawn from seed and instance_id by the library
    spins: np.ndarray | None = None
    arrival: float = 0.0          # time.perf_counter() seconds; 0 = the submit time


@dataclass
class Result:
    ticket: int
    status: str                 # "thermalized", "not_thermalized" or "cancelled"
    sweeps: int
    arrival: float
    done: float
    e: float                    # last window's energy per spin at the lowest temperature
    q_l: float                  # last window's link overlap at the lowest temperature
    delta: float                # E(q_l) - e of the last window (Eq. 1 / Eq. 2, one instance)
    accE: float                 # raw accumulators of the last window (k = 0)
    acc_d: int
    n_meas: int
    slot: int = -1
    admitted: float = 0.0       # when the request entered a slot (same clock as done)

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class ClassInfo:
    lattice: int
    L: int
    disorder: int
    n_T: int
    threads: int                # CTA width of the class batch (> 128: global-resident layout)
    active: int                 # slots in use


class Server:
    """Native request server on one device (one host thread at a time).

    Times are seconds of the host's monotonic clock, the clock of
    ``time.perf_counter()`` on Linux."""

    def __init__(self, device: int = 0, slots_per_class: int = 256, quantum: int = 64,
                 eps_e: float = 0.005, eps_ql: float = 0.01, need: int = 2, max_sweeps: int = 1 << 16,
                 hbm_budget: int = 8 << 30):
        if quantum < 1 or quantum & (quantum - 1):
            raise ValueError("quantum must be a power of two")
        self._lib = icmpt.load_library()
        cfg = icmpt.ServerConfig(int(slots_per_class), int(quantum), int(max_sweeps),
                                 icmpt.ThermCriterion(float(eps_e), float(eps_ql), int(need)), int(hbm_budget))
        h = ctypes.c_void_p()
        rc = self._lib.icm_server_create(int(device), ctypes.byref(cfg), ctypes.byref(h))
        if rc:
            raise icmpt.IcmError(rc, "icm_server_create")
        self._h = h
        self.quantum = int(quantum)
        self._arrival: dict[int, float] = {}

    def _check(self, rc: int):
        if rc:
            raise icmpt.IcmError(rc, self._lib.icm_server_last_error(self._h).decode())

    # -- public API
    def submit(self, req: Request) -> int:
        T = np.ascontiguousarray(req.T, dtype=np.float64)
        J = None if req.couplings is None else \
            np.ascontiguousarray(req.couplings, dtype=np.float32 if req.disorder == icmpt.GAUSS else np.int8)
        s = None if req.spins is None else np.ascontiguousarray(req.spins, dtype=np.int8)
        r = icmpt._Request(int(req.lattice), int(req.L), int(req.disorder), len(T), T.ctypes.data,
                           float(req.T_icm), int(req.seed) & 0xFFFFFFFFFFFFFFFF, int(req.instance_id),
                           None if J is None else J.ctypes.data, None if s is None else s.ctypes.data)
        t = ctypes.c_uint64()
        self._check(self._lib.icm_server_submit(self._h, ctypes.byref(r), ctypes.byref(t)))   # arrays copied
        if not req.arrival:
            req.arrival = time.perf_counter()
        self._arrival[t.value] = req.arrival
        return t.value

    def poll(self, ticket: int) -> Result | None:
        out = icmpt.ServerResult()
        self._check(self._lib.icm_server_poll(self._h, int(ticket), ctypes.byref(out)))
        if out.status == icmpt.PENDING:
            return None
        status = ("cancelled" if out.status == icmpt.CANCELLED else
                  "thermalized" if out.thermalized else "not_thermalized")
        return Result(int(ticket), status, int(out.sweeps),
                      self._arrival.get(int(ticket), out.t_submit), out.t_done, out.e, out.q_l, out.delta,
                      out.accE, int(out.acc_d), int(out.n_meas), int(out.slot), out.t_admit)

    def cancel(self, ticket: int):
        """Drop a queued request, or release a running one at its class's next collection."""
        self._check(self._lib.icm_server_cancel(self._h, int(ticket)))

    def status(self) -> tuple[int, int, int]:
        """(requests queued, requests in slots, classes)."""
        q, a, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        self._check(self._lib.icm_server_status(self._h, ctypes.byref(q), ctypes.byref(a), ctypes.byref(c)))
        return q.value, a.value, c.value

    @property
    def active(self) -> int:
        return self.status()[1]

    def idle(self) -> bool:
        q, a, _ = self.status()
        return q == 0 and a == 0

    def step(self) -> int:
        """One admit / collect / launch pass; returns the requests finished."""
        fin, lau = ctypes.c_int32(), ctypes.c_int32()
        self._check(self._lib.icm_server_step(self._h, ctypes.byref(fin), ctypes.byref(lau)))
        if fin.value == 0 and lau.value == 0:
            time.sleep(50e-6)                          # every class is busy on the device
        return fin.value

    def run_until_idle(self, max_steps: int = 1 << 30):
        n = 0
        while not self.idle() and n < max_steps:
            self.step()
            n += 1

    def class_info(self) -> list[ClassInfo]:
        out = []
        for i in range(self.status()[2]):
            v = [ctypes.c_int32() for _ in range(6)]
            self._check(self._lib.icm_server_class_info(self._h, i, *[ctypes.byref(x) for x in v]))
            out.append(ClassInfo(*[x.value for x in v]))
        return out

    def close(self):
        if getattr(self, "_h", None):
            self._lib.icm_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
