"""Experiments of the paper at reduced scale: the fraction of potential
cluster sites (Fig. 1), thermalization (Fig. 2, Fig. 3) and simulated
annealing with cluster moves.

Fig. 1: p(T) is the fraction of sites with negative overlap q_i = -1 between
the two replicas at temperature T, after step 2a (so p <= 1/2), averaged over
the measured sweeps and then over disorder instances.  Clusters of the
isoenergetic move percolate once p exceeds the site-percolation threshold
p_c of the lattice; `crossing_temperature` locates where p(T) reaches p_c.

Thermalization (and the frequency of the cluster moves judged on it):

For one method -- plain parallel tempering (no cluster moves), PT with the
isoenergetic cluster moves (ICM at T_k <= T_icm, with step 2a), or the
Houdayer algorithm (HCA: cluster moves at every temperature, no step 2a) --
a batch of disorder instances is run in doubling windows [2^(b-1), 2^b) and
Delta(t) of Eq. 2 (disorder average of E(q_l) - <H>/N at the lowest
temperature, with its standard error) is recorded at t = 2^b.  The paper
read thermalization times "by eye"; here the thermalization time is the
first t = 2^b from which |Delta| stays within `nsig` standard errors (and
`floor`) for every later window of the run.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import icmpt

METHODS = ("pt", "icm", "hca")


@dataclass
class DeltaCurve:
    method: str
    t: np.ndarray          # window ends 2^b
    delta: np.ndarray      # Eq. 2 at the lowest temperature
    se: np.ndarray         # standard error over instances


def method_schedule(method: str, T_icm: float):
    """(T_icm, icm_every, enable_2a) of a method."""
    if method == "pt":
        return T_icm, 0, 1
    if method == "icm":
        return T_icm, 1, 1
    if method == "hca":
        return float("inf"), 1, 0
    raise ValueError(method)


def delta_curve(ctx, lattice: int, L: int, disorder: int, couplings, spins, T, T_icm: float, seed: int,
                method: str, log2_min: int, log2_max: int, instance_ids=None, icm_every=None) -> DeltaCurve:
    ticm, every, two_a = method_schedule(method, T_icm)
    if icm_every is not None and every:
        every = int(icm_every)                 # cluster moves every n-th sweep instead of every sweep
    b = icmpt.Batch(ctx, lattice, L, disorder, couplings, T, min(ticm, 1e300), seed, spins=spins,
                    instance_ids=instance_ids)
    b.set_schedule(icm_every=every, enable_2a=two_a, t_meas=1 << 62)
    ts, ds, ses = [], [], []
    t = 0
    start = 1 << (log2_min - 1)
    if start > 0:
        b.run(start)
        t = start
    for k in range(log2_min, log2_max + 1):
        b.clear_observables()
        b.set_schedule(t_meas=t)
        end = 1 << k
        b.run(end - t)
        t = end
        m, se, _ = b.delta(0)
        ts.append(t)
        ds.append(m)
        ses.append(se)
    b.close()
    return DeltaCurve(method, np.array(ts), np.array(ds), np.array(ses))


def thermalization_time(curve: DeltaCurve, nsig: float = 2.0, floor: float = 0.0):
    """First window end from which |Delta| <= max(nsig * se, floor) holds for
    every later window; None if the last window does not satisfy it."""
    ok = np.abs(curve.delta) <= np.maximum(nsig * curve.se, floor)
    if not ok[-1]:
        return None
    i = len(ok) - 1
    while i > 0 and ok[i - 1]:
        i -= 1
    return int(curve.t[i])


@dataclass
class FrequencyRow:
    icm_every: int
    t_therm: int | None      # thermalization time in sweeps (None: not within the run)
    ms_per_sweep: float      # time of one simulation step of the batch at this frequency
    cost_ms: float | None    # t_therm x ms_per_sweep: time to the criterion


def icm_frequency(ctx, lattice: int, L: int, disorder: int, couplings, spins, T, T_icm: float, seed: int,
                  candidates=(1, 2, 4, 8), log2_min: int = 4, log2_max: int = 16, nsig: float = 2.0,
                  timing_sweeps: int = 256, instance_ids=None):
    """The frequency of the cluster moves, judged on time to the
    thermalization criterion -- the figure of merit of the isoenergetic
    cluster algorithm -- and not on spin updates per second: cluster moves
    every n-th sweep cost less per sweep but may need more sweeps.  For each
    candidate n: the thermalization time t_n (sweeps) from Delta(t) of Eq. 2
    at the lowest temperature over doubling windows (delta_curve,
    thermalization_time), and the time per sweep s_n of the batch at that
    frequency (a timed run of `timing_sweeps` steps); the cost is t_n s_n.
    Returns (the n of least cost, or None when no candidate thermalized, and
    the rows)."""
    import time
    rows = []
    for n in candidates:
        c = delta_curve(ctx, lattice, L, disorder, couplings, spins, T, T_icm, seed, "icm", log2_min, log2_max,
                        instance_ids=instance_ids, icm_every=n)
        t_th = thermalization_time(c, nsig=nsig)
        b = icmpt.Batch(ctx, lattice, L, disorder, couplings, T, T_icm, seed, spins=spins,
                        instance_ids=instance_ids)
        b.set_schedule(icm_every=int(n))
        b.run(16)
        ctx.sync()
        t0 = time.perf_counter()
        b.run(timing_sweeps)
        ctx.sync()
        s_n = (time.perf_counter() - t0) * 1e3 / timing_sweeps
        b.close()
        rows.append(FrequencyRow(int(n), t_th, s_n, None if t_th is None else t_th * s_n))
    done = [r for r in rows if r.cost_ms is not None]
    best = min(done, key=lambda r: r.cost_ms).icm_every if done else None
    return best, rows


def anneal(ctx, lattice: int, L: int, disorder: int, couplings, spins, T_hi: float, T_lo: float, steps: int,
           sweeps_per_step: int, icm: bool, seed: int, instance_ids=None):
    """Simulated annealing of two replicas per instance (one temperature,
    geometric from T_hi down to T_lo over `steps` values, `sweeps_per_step`
    simulation steps each).  With icm=True every sweep is followed by the
    cluster move of the pair (steps 2a and 2b) -- the variant the paper
    proposes for ground-state searches.  Returns the batch (caller reads it)."""
    ts = T_hi * (T_lo / T_hi) ** (np.arange(steps) / max(steps - 1, 1))
    T_icm = float("inf") if icm else 0.0
    b = icmpt.Batch(ctx, lattice, L, disorder, couplings, ts[:1], min(T_icm, 1e300), seed, spins=spins,
                    instance_ids=instance_ids)
    b.set_schedule(icm_every=1 if icm else 0, swap_every=0, t_meas=1 << 62)
    for T in ts:
        b.set_temperatures([T], min(T_icm, 1e300))
        b.run(sweeps_per_step)
    return b


# ----------------------------------------------------------------------------- Fig. 1
@dataclass
class FractionCurve:
    T: np.ndarray          # temperatures, ascending
    p: np.ndarray          # disorder average of <min(n, N - n)> / N
    se: np.ndarray         # standard error over instances


def cluster_fraction(ctx, lattice: int, L: int, disorder: int, couplings, spins, T, T_icm: float, seed: int,
                     sweeps: int, t_meas: int, instance_ids=None) -> FractionCurve:
    """p(T) of a batch of instances run with PT and cluster moves (steps 1-3)
    for `sweeps` sweeps, measured from sweep t_meas on."""
    b = icmpt.Batch(ctx, lattice, L, disorder, couplings, T, T_icm, seed, spins=spins, instance_ids=instance_ids)
    b.set_schedule(t_meas=t_meas)
    b.run(sweeps)
    o = b.read_observables(hist=False)
    b.close()
    per = o.acc_pmin / (b.N * np.maximum(o.n_meas, 1)[:, None].astype(np.float64))
    n = per.shape[0]
    se = per.std(0, ddof=1) / np.sqrt(n) if n > 1 else np.zeros(per.shape[1])
    return FractionCurve(np.asarray(T, dtype=np.float64), per.mean(0), se)


def crossing_temperature(curve: FractionCurve, p_c: float):
    """The temperature at which p(T) first reaches p_c, going up in T (linear
    interpolation between ladder points), or None if p stays below p_c."""
    T, p = curve.T, curve.p
    for k in range(len(T)):
        if p[k] >= p_c:
            if k == 0:
                return float(T[0])
            f = (p_c - p[k - 1]) / (p[k] - p[k - 1])
            return float(T[k - 1] + f * (T[k] - T[k - 1]))
    return None

