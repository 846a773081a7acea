"""Continuous-batching request loop: disorder instances run to thermalization.

Requests (one disorder instance each, any lattice kind and size the library
supports) are grouped by shape -- lattice, size, disorder kind, temperature
ladder and T_icm -- into classes.  Each class is one slot-table batch with its
own CUDA stream.  A step of the loop

  1. admits queued requests into free slots while the memory budget allows
     (a class's batch is created when its first request arrives);
  2. for every class whose last launch has finished (a non-blocking query of
     its stream), advances the sweep counters of the slots in that launch and,
     at each slot that reached the end of a doubling window [2^(b-1) Q, 2^b Q),
     reads the window's block means at the lowest temperature, applies the
     thermalization test (icm_therm_update) and either finishes the request
     (freeing the slot) or starts the next window;
  3. launches the next `quantum` simulation steps of every idle class with
     active slots.  Classes advance independently on their own streams, so a
     class of large lattices does not hold back the small ones.

The random streams are keyed by (seed, instance id) only, so a request's
trajectory does not depend on its slot or on the other requests in the mix.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

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
    couplings: np.ndarray
    spins: np.ndarray | None = None
    arrival: float = 0.0


@dataclass
class Result:
    ticket: int
    status: str                 # "thermalized" or "not_thermalized"
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

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class _Slot:
    ticket: int
    req: Request
    t: int = 0
    boundary: int = 0
    state: icmpt.ThermState = field(default_factory=icmpt.ThermState)


class _Class:
    def __init__(self, ctx_dev: int, req: Request, capacity: int):
        import torch
        self.stream = torch.cuda.Stream()
        self.ctx = icmpt.Context(ctx_dev, self.stream.cuda_stream)
        self.N, self.Nb = icmpt.lattice_size(req.lattice, req.L)
        # placeholder couplings of the free slots: all bonds present (a zero
        # coupling is an absent bond, which would switch the batch to its
        # diluted kernels)
        dummy = np.ones((capacity, self.Nb), dtype=req.couplings.dtype)
        self.batch = icmpt.Batch(self.ctx, req.lattice, req.L, req.disorder, dummy, req.T, req.T_icm, req.seed)
        self.batch.set_active(-1, False)
        self.free = list(range(capacity))[::-1]
        self.slots: dict[int, _Slot] = {}
        self.T_min = float(req.T[0])
        self.bytes = capacity * slot_bytes(req)
        self.in_flight: set[int] = set()       # slots of the launch still running


def shape_key(r: Request):
    return (r.lattice, r.L, r.disorder, tuple(np.round(np.asarray(r.T, dtype=np.float64), 12)), float(r.T_icm),
            int(r.seed))


def slot_bytes(r: Request) -> int:
    """Device bytes one slot of this request's class takes (state, staging, observables)."""
    N, Nb = icmpt.lattice_size(r.lattice, r.L)
    nT = len(r.T)
    R = 2 * nT
    Z = {icmpt.SQUARE2D: 4, icmpt.HYPERCUBIC4D: 8}.get(r.lattice, 6)
    G = (R + 31) // 32
    return (N * Z * 4 + G * N * 4 + R * N + Nb * 4 + nT * (N + 1) * 8 + 8 * nT * 8 + R * 16 + 64)


class Server:
    def __init__(self, device: int = 0, slots_per_class: int = 256, quantum: int = 64,
                 eps_e: float = 0.005, eps_ql: float = 0.01, need: int = 2, max_sweeps: int = 1 << 16,
                 hbm_budget: int = 8 << 30):
        if quantum < 1 or quantum & (quantum - 1):
            raise ValueError("quantum must be a power of two")
        self.device = device
        self.capacity = slots_per_class
        self.quantum = quantum
        self.crit = icmpt.ThermCriterion(eps_e, eps_ql, need)
        self.max_sweeps = max_sweeps
        self.budget = hbm_budget
        self.used = 0
        self.classes: dict[tuple, _Class] = {}
        self.queue: collections.deque[tuple[int, Request]] = collections.deque()
        self.results: dict[int, Result] = {}
        self.next_ticket = 0
        self.clock = time.perf_counter

    # -- public API
    def submit(self, req: Request) -> int:
        t = self.next_ticket
        self.next_ticket += 1
        if not req.arrival:
            req.arrival = self.clock()
        self.queue.append((t, req))
        return t

    def poll(self, ticket: int) -> Result | None:
        return self.results.get(ticket)

    @property
    def active(self) -> int:
        return sum(len(c.slots) for c in self.classes.values())

    def idle(self) -> bool:
        return not self.queue and self.active == 0

    def step(self) -> int:
        """Admit; collect every class whose launch finished and test its
        windows; launch the next quantum of every idle class.  Returns the
        number of requests that finished in this step."""
        self._admit()
        finished = 0
        progressed = False
        for c in self.classes.values():
            if c.in_flight:
                if not c.ctx.query():
                    continue
                progressed = True
                due = []
                for slot in c.in_flight:
                    st = c.slots[slot]
                    st.t += self.quantum
                    if st.t >= st.boundary:
                        due.append(slot)
                c.in_flight = set()
                if due:
                    obs = c.batch.read_observables(hist=False)
                    for slot in due:
                        finished += self._window(c, slot, obs)
            if c.slots and not c.in_flight:
                c.batch.run(self.quantum)
                c.in_flight = set(c.slots)
                progressed = True
        if not progressed:
            time.sleep(50e-6)                          # every class is busy on the device
        return finished

    def run_until_idle(self, max_steps: int = 1 << 30):
        n = 0
        while not self.idle() and n < max_steps:
            self.step()
            n += 1

    # -- internals
    def _admit(self):
        waiting = collections.deque()
        while self.queue:
            ticket, req = self.queue.popleft()
            key = shape_key(req)
            c = self.classes.get(key)
            if c is None:
                need = self.capacity * slot_bytes(req)
                if self.used + need > self.budget:
                    waiting.append((ticket, req))      # admission by memory budget: wait
                    continue
                c = _Class(self.device, req, self.capacity)
                self.classes[key] = c
                self.used += c.bytes
            if not c.free or c.in_flight:
                # no free slot, or the class is running: its slot tables are
                # written between launches (a copy from pageable host memory
                # would wait for the running launch)
                waiting.append((ticket, req))
                continue
            slot = c.free.pop()
            c.batch.set_slot(slot, np.ascontiguousarray(req.couplings), None if req.spins is None
                             else np.ascontiguousarray(req.spins), req.instance_id)
            c.batch.start_window(slot, self.quantum)   # first window [Q, 2Q)
            c.slots[slot] = _Slot(ticket, req, 0, 2 * self.quantum)
        self.queue = waiting

    def _window(self, c: _Class, slot: int, obs) -> int:
        st = c.slots[slot]
        m = int(obs.n_meas[slot])
        e = obs.accE[slot, 0] / (2.0 * c.N * m)
        nb = int(obs.nb[slot]) if obs.nb is not None else c.Nb     # bonds present (dilution)
        ql = 1.0 - 2.0 * obs.acc_d[slot, 0] / (max(nb, 1) * m)
        done = icmpt.therm_update(st.state, self.crit, e, ql, c.T_min, nb / c.N)
        if done or st.t >= self.max_sweeps:
            self.results[st.ticket] = Result(st.ticket, "thermalized" if done else "not_thermalized", st.t,
                                             st.req.arrival, self.clock(), e, ql, st.state.delta,
                                             float(obs.accE[slot, 0]), int(obs.acc_d[slot, 0]), m, slot)
            c.batch.set_active(slot, False)
            del c.slots[slot]
            c.free.append(slot)
            return 1
        c.batch.start_window(slot, st.t)              # next window [t, 2t)
        st.boundary = 2 * st.t
        return 0

    def close(self):
        for c in self.classes.values():
            c.batch.close()
            c.ctx.close()
        self.classes.clear()
