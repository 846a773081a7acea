#!/usr/bin/env python3
"""Benchmark: parallel tempering + isoenergetic cluster moves on GB300.

Workload (default): 3D Edwards-Anderson spin glass, L = 8 periodic cubic
lattice (512 spins), Gaussian couplings N(0,1) in fp32, 1000 disorder
instances in one launch, 24 temperatures geometric in [0.2, 2.0], 2 replicas
per temperature, ICM at T <= 1.0, one PT pass and one measurement per sweep.
A step = `--sweeps-per-step` full simulation steps (Metropolis sweep, step
2a/2b at the 17 ICM temperatures, PT pass, observables) of all instances.

Prints one JSON line.  `value` is spin updates per ns over the K timed steps
(device time from CUDA events on the launching stream, state resident in HBM,
L2 flushed between steps); `e2e` is the same metric through the C ABI with
host buffers (H2D of couplings and spins, run, D2H of the observables).
The default line also carries the served form (`serving`: instances
thermalized/s and latency against plain PT one instance at a time), the
mixed-size workload in one persistent kernel launch (`mixed_sizes`) and 2D
L=128 on thread-block clusters (`large_instances`: 20 and 36 instances).
`--impl reference` times the CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1501_05630_gb300 import inputs as I  # noqa: E402

WORKLOADS = {
    "3d_gauss_L8": dict(lattice=I.CUBIC3D, L=8, disorder=I.GAUSS, n_inst=1000, T=(0.2, 2.0, 24), T_icm=1.0,
                        seed=0x1501056300000002,
                        desc="3D EA L=8 periodic (512 spins), Gaussian N(0,1) fp32, 1000 instances, "
                             "24 T geometric [0.2,2.0], 2 replicas/T, ICM T<=1.0"),
    "chimera_pmj_C8": dict(lattice=I.CHIMERA, L=8, disorder=I.PM_J, n_inst=10000, T=(0.2, 3.0, 30), T_icm=1.5,
                           seed=0x1501056300000003,
                           desc="chimera C_8 (512 spins), +-J, 10^4 instances multispin-coded, "
                                "30 T geometric [0.2,3.0], ICM T<=1.5"),
    "2d_pmj_L8": dict(lattice=I.SQUARE2D, L=8, disorder=I.PM_J, n_inst=1, T=(0.2, 1.5, 16), T_icm=1.0,
                      seed=0x1501056300000001,
                      desc="2D EA L=8 periodic (64 spins), +-J, 1 instance, 16 T geometric [0.2,1.5], ICM T<=1.0"),
    # the largest 2D size of the serving menu, a few instances at a time (with --cluster: 8 SMs each)
    "2d_pmj_L128": dict(lattice=I.SQUARE2D, L=128, disorder=I.PM_J, n_inst=20, T=(0.2, 1.5, 32), T_icm=1.0,
                        seed=0x1501056300000008,
                        desc="2D EA L=128 periodic (16384 spins), +-J, 20 instances, 32 T geometric [0.2,1.5], "
                             "ICM T<=1.0"),
    # the largest 3D size of the serving menu, a few instances at a time (with --cluster: 8 SMs each)
    "3d_gauss_L16": dict(lattice=I.CUBIC3D, L=16, disorder=I.GAUSS, n_inst=20, T=(0.2, 2.0, 32), T_icm=1.0,
                         seed=0x1501056300000009,
                         desc="3D EA L=16 periodic (4096 spins), Gaussian N(0,1) fp32, 20 instances, "
                              "32 T geometric [0.2,2.0], ICM T<=1.0"),
}

# Algorithmic integer/fp operations per spin update (the per-unit figure of the
# method's cost model): Philox4x32-10 = 98 integer ops per call of 4 draws
# (10 rounds x 4 mul.lo/hi + 4 xor, 9 x 2 key increments) -> 24.5 per update;
# local field and acceptance 10..15 (midpoint 12.5) -> 37 for +-J; Gaussian
# couplings add z fp32 multiply-adds and one exponential.
ALG_OPS = {I.PM_J: lambda z: 24.5 + 12.5,
           I.GAUSS: lambda z: 24.5 + 12.5 + z + 1}



def icm_ops(N: int, Nb: int, z: int, n_icm: int, pairs: float, moves: float, scans: float,
            union_find: bool = False) -> float:
    """Algorithmic operations of the cluster moves (steps 2a/2b), the
    method's cost model of O(N + N_b) per pair plus the growth iterations:
      per ICM pair visited (`pairs` = instances x ICM temperatures x sweeps):
        the overlap q_i (N), the count n (N), step 2a (N);
      per moved pair (`moves`, n > 0, from the device counter): the seed
        draw (one Philox4x32-10 call, 98 ops), the rank search (N), the flip
        of both copies (2N), the energy update over the bonds (N_b);
      per growth scan (`scans`, from the device counter, summed over the
        instances): one pass over the site words that hold ICM pairs
        (ceil(n_icm / 16) per site, two replica bits per pair), each word
        the OR of its z neighbours' cluster words, one AND with its domain
        and one OR into its own word (z + 2).
    One operation per spin (or bond) and pair, as the method is written,
    except the growth, counted per 32-bit word of the bit-parallel flood fill
    that stands for one label-propagation pass of every pair.  Union-find
    growth (thread-block-cluster layout on request) counts instead, per moved
    pair, one label reset per site, one union per bond and one root lookup
    per site (2N + N_b); its scan counter is not used."""
    words = -(-n_icm // 16)
    growth = moves * (2 * N + Nb) if union_find else scans * words * N * (z + 2)
    return pairs * 3 * N + moves * (98 + 3 * N + Nb) + growth


def phase_fractions(b, stream, flush, S, n_inst, updates_per_step, ops_per_update, N, Nb, z, n_icm, peak):
    """Roofline fractions of the two phases, from launches that differ only in
    the public schedule flags: the sweep alone (no cluster moves, PT pass or
    measurement) and the cluster moves alone (no Metropolis sweep, PT pass or
    measurement), each timed over three launches of S sweeps after one
    untimed launch, with CUDA events on the launching stream and L2 flushed
    between launches.  The schedule is restored afterwards."""
    import torch
    sched = b.schedule()
    keep = {k: getattr(sched, k) for k in ("icm_every", "swap_every", "enable_2a", "enable_metropolis",
                                           "t_meas", "trace")}

    def timed(n=3):
        b.run(S)
        torch.cuda.synchronize()
        ts = []
        for _ in range(n):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.run(S)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.mean(ts))

    b.set_schedule(icm_every=0, swap_every=0, t_meas=1 << 62, trace=0)
    t_sweep = timed()
    b.set_schedule(icm_every=1, swap_every=0, enable_metropolis=0, t_meas=1 << 62, trace=0)
    b.clear_observables()
    t_icm = timed()
    st = b.read_icm_stats().astype(np.float64)
    b.set_schedule(**keep)
    moves, scans = st[:, 0].sum() / 4, st[:, 1].sum() / 4        # per launch (4 launches counted)
    pairs = n_inst * n_icm * S
    sweep_ach = updates_per_step * ops_per_update / (t_sweep * 1e-3) / 1e12
    icm_ach = icm_ops(N, Nb, z, n_icm, pairs, moves, scans, b.cluster_growth() > 0) / (t_icm * 1e-3) / 1e12
    return {"sweep_frac": sweep_ach / peak, "sweep_ms": t_sweep,
            "sweep_updates_per_ns": updates_per_step / (t_sweep * 1e6),
            "icm_frac": icm_ach / peak, "icm_ms": t_icm, "icm_moved_fraction": moves / pairs,
            "icm_scans_per_sweep": scans / (n_inst * S),
            "phase_note": "sweep_frac: Metropolis ops of a sweep-only launch; icm_frac: cluster-move ops "
                          "(icm_ops) of an ICM-only launch; both over the same issue peak"}


# the sources of the fused kernel (its launch shape and arithmetic); host-side
# files (the API, the request server, other kernels) do not change its traffic
FUSED_SOURCES = ("pt_icm.cu", "fused_pmj.cu", "fused_gauss.cu", "icm_device.cuh", "icm_internal.h")


def kernel_source_digest() -> str:
    """Digest of the fused kernel's code: its sources with comments removed and
    whitespace collapsed, so that a comment edit keeps the recorded counters."""
    import hashlib
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1501_05630_gb300", "csrc")
    for f in FUSED_SOURCES:
        with open(os.path.join(csrc, f)) as fh:
            code = fh.read()
        code = re.sub(r"/\*.*?\*/", " ", code, flags=re.S)
        code = re.sub(r"//[^\n]*", " ", code)
        code = " ".join(code.split())
        h.update(f.encode() + code.encode())
    return h.hexdigest()[:16]


def recorded_counter(workload: str, key: str):
    """A counter of the committed ncu summary of this workload's fused kernel
    (traffic_bytes_per_launch, instructions_per_update), or None when the
    kernel sources changed since that capture."""
    path = os.path.join(ROOT, "profiles", f"fused_kernel_{workload}.md")
    try:
        vals = {}
        for line in open(path):
            if ":" in line and line.strip().startswith((key, "kernel_source_digest")):
                k, v = line.strip().strip("`").split(":", 1)
                vals[k.strip()] = v.strip().strip("`")
        if vals.get("kernel_source_digest") != kernel_source_digest():
            return None
        return float(vals[key])
    except Exception:
        return None


def recorded_traffic(workload: str):
    """DRAM bytes per fused-kernel launch (see recorded_counter)."""
    return recorded_counter(workload, "traffic_bytes_per_launch")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons while the timed region runs."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_throughput(wl, sweeps: int, n_inst: int, threads: int):
    """The CPU oracle, as it stands, on n_inst instances x `sweeps` sweeps,
    instances spread over `threads` host threads (ctypes drops the GIL)."""
    from concurrent.futures import ThreadPoolExecutor
    from oracle import oracle as O
    g = O.Geometry(wl["lattice"], wl["L"])
    T = I.ladder(*wl["T"])
    J = I.couplings(g.Nb, wl["disorder"], wl["seed"], range(n_inst))
    s0 = I.initial_spins(g.N, 2 * len(T), wl["seed"], range(n_inst))
    insts = [O.Instance(g, J[a].astype(np.float64), T, s0[a], pm=(wl["disorder"] == I.PM_J),
                        T_icm=wl["T_icm"], seed=wl["seed"], inst=a) for a in range(n_inst)]
    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(lambda x: x.run(sweeps), insts))
    dt = time.perf_counter() - t0
    updates = n_inst * sweeps * g.N * 2 * len(T)
    return updates / dt / 1e9, dt, updates


def calibrate_sweeps(wl, cores, seconds):
    """Sweeps per instance so that 2*cores instances take about `seconds`."""
    rate, dt, _ = oracle_throughput(wl, 4, 1, 1)            # updates/ns of one core
    from oracle import oracle as O
    g = O.Geometry(wl["lattice"], wl["L"])
    per_sweep = g.N * 2 * len(I.ladder(*wl["T"]))
    sweeps = int(seconds * rate * 1e9 * cores / (2 * cores * per_sweep))
    return max(4, sweeps)


def run_reference(args, wl, rank):
    cores = os.cpu_count() or 1
    if rank != 0:
        return
    sweeps = args.ref_sweeps
    vals = []
    for _ in range(args.warmup):
        oracle_throughput(wl, sweeps, cores, cores)
    for _ in range(args.steps):
        v, dt, _ = oracle_throughput(wl, sweeps, cores, cores)
        vals.append(v)
    value = float(np.mean(vals))
    n_icm = int(np.sum(I.ladder(*wl["T"]) <= wl["T_icm"]))
    sample = f"{cores} instances x {sweeps} sweeps per step (of {wl['n_inst']} instances), {cores} threads"
    print(json.dumps({
        "impl": "reference", "metric": "spin_updates_per_ns", "value": value, "unit": "updates/ns",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if wl["disorder"] == I.GAUSS else "int64",
        "data": "synthetic", "config": {"workload": args.workload, "desc": wl["desc"], "n_icm": n_icm},
        "cpu_baseline": {"value": value, "unit": "updates/ns", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "updates/ns", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


SERVING_MENU = [
    # (lattice, L, disorder, (T_min, T_max), T_icm): 2D +-J L in {16,32,64,128}, 3D Gaussian L in {6,8,12,16},
    # chimera C_8 / C_12 +-J
    (I.SQUARE2D, 16, I.PM_J, (0.2, 1.5), 1.0), (I.SQUARE2D, 32, I.PM_J, (0.2, 1.5), 1.0),
    (I.SQUARE2D, 64, I.PM_J, (0.2, 1.5), 1.0), (I.SQUARE2D, 128, I.PM_J, (0.2, 1.5), 1.0),
    (I.CUBIC3D, 6, I.GAUSS, (0.2, 2.0), 1.0), (I.CUBIC3D, 8, I.GAUSS, (0.2, 2.0), 1.0),
    (I.CUBIC3D, 12, I.GAUSS, (0.2, 2.0), 1.0), (I.CUBIC3D, 16, I.GAUSS, (0.2, 2.0), 1.0),
    (I.CHIMERA, 8, I.PM_J, (0.2, 3.0), 1.5), (I.CHIMERA, 12, I.PM_J, (0.2, 3.0), 1.5),
]


def serving_requests(n, rate, seed, n_T_choices):
    """Poisson arrivals (mean `rate`/s) of instances drawn uniformly from the menu."""
    from paper_1501_05630_gb300 import icmpt
    from paper_1501_05630_gb300.serve import Request
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    reqs = []
    for i in range(n):
        lat, L, dis, (tl, th), ticm = SERVING_MENU[rng.integers(len(SERVING_MENU))]
        nT = int(rng.choice(n_T_choices))
        N, Nb = icmpt.lattice_size(lat, L)
        inst = 5000 + i
        reqs.append(Request(lat, L, dis, I.ladder(tl, th, nT), ticm, seed, inst,
                            I.couplings(Nb, dis, seed, [inst])[0], I.initial_spins(N, 2 * nT, seed, [inst])[0],
                            arrival=float(t[i])))
    return reqs


def _menu_name(lat, L, dis):
    return f"{['2D', '3D', 'chimera', '4D'][lat]} L={L} {['pmJ', 'gauss'][dis]}"


def serving_measurement(args):
    """Workload 5 (serving): a Poisson stream of requests over the full menu,
    run to the per-instance thermalization criterion by the native
    continuous-batching server; then the plain method one instance at a time
    (plain PT: T_icm below every temperature, so no step 2a or 2b; a one-slot
    server, the same criterion and sweep cap) on a sample stratified by menu
    kind, `alone_sample` requests of each kind taken round-robin over the
    kinds and started while `alone_seconds` last.  Returns the figures as a
    dict (rates in instances thermalized per second of wall time)."""
    import torch
    from paper_1501_05630_gb300 import build
    from paper_1501_05630_gb300.serve import Server
    torch.cuda.set_device(0)
    build.build()
    n_T = tuple(int(x) for x in args.serving_nT.split(","))
    reqs = serving_requests(args.requests, args.rate, 0x150105630000005, n_T)
    kw = dict(quantum=args.quantum, max_sweeps=args.max_sweeps, eps_e=0.005, eps_ql=0.01, need=2)
    srv = Server(slots_per_class=args.slots, **kw)
    pending = sorted(reqs, key=lambda r: r.arrival)
    tickets = {}
    i = 0
    with ClockSampler(0) as clk:
        start = time.perf_counter()
        while i < len(pending) or not srv.idle():
            now = time.perf_counter() - start
            while i < len(pending) and pending[i].arrival <= now:
                r = pending[i]
                r.arrival = start + r.arrival
                tickets[srv.submit(r)] = r
                i += 1
            if srv.idle():
                time.sleep(max(0.0, min(0.002, pending[i].arrival - (time.perf_counter() - start))))
                continue
            srv.step()
        wall = time.perf_counter() - start
    res = {t: srv.poll(t) for t in tickets}
    srv.close()
    lat = np.array([r.latency for r in res.values()])
    lat_th = np.array([r.latency for r in res.values() if r.status == "thermalized"])
    therm = sum(r.status == "thermalized" for r in res.values())
    last_arrival = max(r.arrival for r in tickets.values())
    admits = np.array([r.admitted for r in res.values()])
    per_class = {}
    for t, r in tickets.items():
        c = per_class.setdefault(_menu_name(r.lattice, r.L, r.disorder), {"requests": 0, "thermalized": 0})
        c["requests"] += 1
        c["thermalized"] += res[t].status == "thermalized"
    # the plain method, one instance at a time
    kinds = {}
    for r in pending:
        kinds.setdefault((r.lattice, r.L, r.disorder), []).append(r)
    order = [kinds[k][j] for j in range(args.alone_sample) for k in kinds if j < len(kinds[k])]
    a0 = time.perf_counter()
    alone_therm, alone_done, alone_class = 0, 0, {}
    for r in order:
        if time.perf_counter() - a0 > args.alone_seconds:
            break
        one = Server(slots_per_class=1, **kw)
        r2 = dataclasses_replace(r)
        r2.T_icm = 0.0                                      # plain PT: no cluster temperature
        tk = one.submit(r2)
        one.run_until_idle()
        ok = one.poll(tk).status == "thermalized"
        one.close()
        alone_therm += ok
        alone_done += 1
        c = alone_class.setdefault(_menu_name(r.lattice, r.L, r.disorder), {"requests": 0, "thermalized": 0})
        c["requests"] += 1
        c["thermalized"] += int(ok)
    alone_s = time.perf_counter() - a0
    return {
        "instances_thermalized_per_s": therm / wall, "latency_p50_s": float(np.percentile(lat, 50)),
        "latency_p99_s": float(np.percentile(lat, 99)),
        "latency_thermalized_p50_s": float(np.percentile(lat_th, 50)) if len(lat_th) else None,
        "latency_thermalized_p99_s": float(np.percentile(lat_th, 99)) if len(lat_th) else None,
        "requests": len(res), "offered_per_s": args.rate,
        "thermalized": int(therm), "not_thermalized": int(len(res) - therm), "wall_s": wall,
        "completed_per_s": len(res) / wall,
        "admitted_per_s": len(res) / max(float(admits.max()) - start, 1e-9),
        "backlog_at_last_arrival": int(np.sum(admits > last_arrival)),
        "sustainable": bool(len(res) / wall >= 0.95 * args.rate),
        "mean_sweeps": float(np.mean([r.sweeps for r in res.values()])),
        "per_class": per_class,
        "one_at_a_time_plain_pt": {"value": alone_therm / alone_s, "unit": "instances/s",
                                   "requests": alone_done, "thermalized": int(alone_therm), "wall_s": alone_s,
                                   "sample": f"{args.alone_sample} per menu kind, round-robin over the kinds, "
                                             f"started within {args.alone_seconds:.0f} s",
                                   "per_class": alone_class},
        "config": {"menu": [_menu_name(*m[:3]) for m in SERVING_MENU], "n_T": n_T, "quantum": args.quantum,
                   "max_sweeps": args.max_sweeps, "slots_per_class": args.slots,
                   "criterion": "block means of e and q_l at T_min agree (|de|<=0.005, |dq_l|<=0.01) on 2 "
                                "consecutive doubling windows"},
        "clocks": clk.summary(),
    }


def run_serving(args):
    out = serving_measurement(args)
    line = {"metric": "instances_thermalized_per_s", "value": out["instances_thermalized_per_s"],
            "unit": "instances/s", "n_gpus": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "data": "synthetic", "dtype": "u32/f32",
            "config": dict(out.pop("config"), workload="serving", requests=args.requests, rate_per_s=args.rate)}
    line.update(out)
    print(json.dumps(line))


def dataclasses_replace(r):
    import dataclasses
    return dataclasses.replace(r, arrival=0.0)


MIXED = dict(sizes=(4, 6, 8, 10, 12), counts=(4096, 2048, 1024, 512, 256), T=(0.2, 2.0, 24), T_icm=1.0,
             seed=0x1501056300000004,
             desc="3D EA Gaussian, L in {4,6,8,10,12} x {4096,2048,1024,512,256} instances, 24 T geometric "
                  "[0.2,2.0], ICM T<=1.0, one seed (instance ids distinct across sizes)")


def mixed_measurement(args, steps: int, warmup: int, mode: str) -> dict:
    """Workload 4: uneven sizes in one captured launch.  shared (default): the
    instances of all sizes share one persistent kernel (icm_group_create_shared),
    threads per instance tuned by timing (icmpt.tune_shared_widths); graph: one
    kernel per size on forked streams, CTA width autotuned per size.  Returns
    the bench line of the workload."""
    import torch
    from paper_1501_05630_gb300 import build, icmpt
    torch.cuda.set_device(0)
    build.build()
    stream = torch.cuda.current_stream()
    ctx = icmpt.Context(0, stream.cuda_stream)
    T = I.ladder(*MIXED["T"])
    batches, updates, tuned = [], 0, {}
    first = 0
    for L, n in zip(MIXED["sizes"], MIXED["counts"]):
        N, Nb = icmpt.lattice_size(I.CUBIC3D, L)
        ids = np.arange(first, first + n, dtype=np.uint32)
        first += n
        J = torch.from_numpy(I.couplings(Nb, I.GAUSS, MIXED["seed"], ids)).cuda()
        s0 = torch.from_numpy(I.initial_spins(N, 2 * len(T), MIXED["seed"], ids)).cuda()
        b = icmpt.Batch(ctx, I.CUBIC3D, L, I.GAUSS, J, T, MIXED["T_icm"], MIXED["seed"], spins=s0, instance_ids=ids)
        if mode == "graph":
            th, ms = b.autotune(sweeps=8)
            tuned[f"L{L}"] = {"threads": th, "ctas_per_sm": b.info()["ctas_per_sm"]}
        batches.append(b)
        updates += n * 2 * len(T) * N
    S = args.sweeps_per_step
    if mode == "shared":
        if args.team_threads:
            widths = [int(x) for x in args.team_threads.split(",")]
            table = {c: {} for c in range(len(batches))}
        else:
            widths, table = icmpt.tune_shared_widths(ctx, batches, sweeps=8)
        g = icmpt.Group(ctx, batches, S, shared=True, team_threads=widths)
        info = g.info()
        for L, w, k in zip(MIXED["sizes"], info["team_threads"], info["tile"]):
            tuned[f"L{L}"] = {"threads_per_instance": w, "instances_per_tile": k,
                              "tried_ms": {str(x): round(y, 3) for x, y in table[MIXED["sizes"].index(L)].items()}}
        tuned["kernel"] = {"grid": info["grid"], "smem_bytes": info["smem_bytes"], "tiles": info["n_items"],
                           "threads": 896}
    else:
        g = icmpt.Group(ctx, batches, S)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(warmup):
        g.run(1)
    torch.cuda.synchronize()
    times = []
    with ClockSampler(0) as clk:
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.run(1)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
    ms = float(np.sum(times))
    value = updates * S * steps / (ms * 1e6)
    desc = MIXED["desc"] + (", all sizes in one persistent kernel launch (CUDA graph), threads per instance tuned"
                            if mode == "shared" else
                            ", one CUDA graph per step (one kernel per size on forked streams), CTA width "
                            "autotuned per size")
    out = {
        "metric": "spin_updates_per_ns", "value": value, "unit": "updates/ns", "n_gpus": 1, "steps": steps,
        "warmup": warmup, "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "3d_gauss_mixed", "mode": mode, "desc": desc, "sweeps_per_step": S,
                   "tuned": tuned, "l2": "flushed between steps (256 MB write)"},
        "gpu_launches": steps if mode == "shared" else steps * len(batches),
        "clocks": clk.summary()}
    g.close()
    for b in batches:
        b.close()
    ctx.close()
    return out


def cluster_measurement(n_inst: int, steps: int = 3, warmup: int = 2, sweeps: int = 64) -> dict:
    """The largest 2D size of the serving menu on 8-CTA thread-block clusters
    (the 2d_pmj_L128 workload with n_inst instances): spin updates/ns over
    `steps` launches of `sweeps` sweeps, CUDA events, L2 flushed between."""
    import torch
    from paper_1501_05630_gb300 import icmpt
    wl = WORKLOADS["2d_pmj_L128"]
    stream = torch.cuda.current_stream()
    ctx = icmpt.Context(torch.cuda.current_device(), stream.cuda_stream)
    T = I.ladder(*wl["T"])
    N, Nb = icmpt.lattice_size(wl["lattice"], wl["L"])
    ids = np.arange(n_inst, dtype=np.uint32)
    b = icmpt.Batch(ctx, wl["lattice"], wl["L"], wl["disorder"], I.couplings(Nb, wl["disorder"], wl["seed"], ids), T,
                    wl["T_icm"], wl["seed"], spins=I.initial_spins(N, 2 * len(T), wl["seed"], ids), instance_ids=ids)
    b.set_cluster(8, 512)
    info = b.info()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(warmup):
        b.run(sweeps)
    torch.cuda.synchronize()
    ms = 0.0
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.run(sweeps)
        e1.record(stream)
        e1.synchronize()
        ms += e0.elapsed_time(e1)
    out = {"value": n_inst * 2 * len(T) * N * sweeps * steps / (ms * 1e6), "unit": "updates/ns",
           "ms_per_step": ms / steps, "sweeps_per_step": sweeps, "steps": steps, "instances": n_inst,
           "clusters": info["grid"] // 8, "gpu_launches": steps}
    b.close()
    ctx.close()
    return out


def run_mixed(args):
    print(json.dumps(mixed_measurement(args, args.steps, args.warmup, args.mixed_mode)))


THERMO = [
    # Table I (geometric ladders; N_c lowest temperatures get cluster moves), reduced instance counts
    dict(name="2D N=256", lattice=I.SQUARE2D, L=16, T=(0.2120, 1.6325, 30), n_c=30),
    dict(name="chimera N=288", lattice=I.CHIMERA, L=6, T=(0.2120, 1.6325, 30), n_c=19),
    dict(name="3D N=216", lattice=I.CUBIC3D, L=6, T=(0.4200, 1.8000, 26), n_c=13),
]


def run_thermalization(args):
    """Delta(t) of Eq. 2 for PT, PT+ICM and HCA on reduced Table I systems and
    the automated thermalization-time ratio PT / PT+ICM (Fig. 2, Fig. 3)."""
    import torch
    from paper_1501_05630_gb300 import build, icmpt
    from paper_1501_05630_gb300.experiments import delta_curve, thermalization_time
    torch.cuda.set_device(0)
    build.build()
    ctx = icmpt.Context(0)
    out = {"metric": "thermalization_speedup", "unit": "PT sweeps / PT+ICM sweeps", "higher_is_better": True,
           "n_gpus": 1, "data": "synthetic", "config": {"workload": "thermalization", "instances": args.instances,
                                                       "log2_sweeps": [4, args.log2_max]}, "systems": {}}
    t0 = time.perf_counter()
    ratios = []
    for sysd in THERMO:
        T = I.ladder(*sysd["T"])
        T_icm = float(T[sysd["n_c"] - 1]) + 1e-9
        N, Nb = icmpt.lattice_size(sysd["lattice"], sysd["L"])
        seed = 0x1501056300000006 + sysd["L"]
        J = I.couplings(Nb, I.GAUSS, seed, range(args.instances))
        s0 = I.initial_spins(N, 2 * len(T), seed, range(args.instances))
        res = {}
        for m in ("pt", "icm", "hca"):
            c = delta_curve(ctx, sysd["lattice"], sysd["L"], I.GAUSS, J, s0, T, T_icm, seed, m, 4, args.log2_max)
            res[m] = {"t": c.t.tolist(), "delta": [round(float(x), 5) for x in c.delta],
                      "se": [round(float(x), 5) for x in c.se], "t_therm": thermalization_time(c, nsig=2.0)}
        tp, ti = res["pt"]["t_therm"], res["icm"]["t_therm"]
        res["ratio_pt_over_icm"] = (tp / ti) if (tp and ti) else None
        if res["ratio_pt_over_icm"]:
            ratios.append(res["ratio_pt_over_icm"])
        out["systems"][sysd["name"]] = res
    out["value"] = float(np.exp(np.mean(np.log(ratios)))) if ratios else None
    out["wall_s"] = time.perf_counter() - t0
    print(json.dumps(out))


# Fig. 3 systems: the Table I sizes that 256 instances thermalize within 2^18 sweeps under plain PT
FIG3 = [
    dict(name="2D", lattice=I.SQUARE2D, Ls=(16, 24), T=(0.2120, 1.6325, 30), n_c=30),
    dict(name="chimera", lattice=I.CHIMERA, Ls=(4, 6, 8), T=(0.2120, 1.6325, 30), n_c=19),
    dict(name="3D", lattice=I.CUBIC3D, Ls=(4, 6, 8), T=(0.4200, 1.8000, 26), n_c=13),
]


def run_icm_frequency(args):
    """The frequency of the cluster moves judged on time to the criterion
    (experiments.icm_frequency) for the Table I systems of the thermalization
    workload: cluster moves every 1, 2, 4 or 8 sweeps."""
    import torch
    from paper_1501_05630_gb300 import build, icmpt
    from paper_1501_05630_gb300.experiments import icm_frequency
    torch.cuda.set_device(0)
    build.build()
    ctx = icmpt.Context(0)
    out = {"metric": "icm_frequency_time_to_criterion", "unit": "ms to the criterion", "higher_is_better": False,
           "n_gpus": 1, "data": "synthetic",
           "config": {"workload": "icm_frequency", "instances": args.instances, "log2_sweeps": [4, args.log2_max],
                      "candidates": [1, 2, 4, 8], "criterion": "|Delta| of Eq. 2 within 2 s.e. from a window on"},
           "systems": {}}
    t0 = time.perf_counter()
    for sysd in THERMO:
        T = I.ladder(*sysd["T"])
        T_icm = float(T[sysd["n_c"] - 1]) + 1e-9
        N, Nb = icmpt.lattice_size(sysd["lattice"], sysd["L"])
        seed = 0x1501056300000006 + sysd["L"]
        J = I.couplings(Nb, I.GAUSS, seed, range(args.instances))
        s0 = I.initial_spins(N, 2 * len(T), seed, range(args.instances))
        best, rows = icm_frequency(ctx, sysd["lattice"], sysd["L"], I.GAUSS, J, s0, T, T_icm, seed,
                                   candidates=(1, 2, 4, 8), log2_max=args.log2_max)
        out["systems"][sysd["name"]] = {"best_icm_every": best,
                                       "rows": [dict(icm_every=r.icm_every, t_therm=r.t_therm,
                                                     ms_per_sweep=round(r.ms_per_sweep, 5),
                                                     cost_ms=None if r.cost_ms is None else round(r.cost_ms, 2))
                                                for r in rows]}
    out["wall_s"] = time.perf_counter() - t0
    out["value"] = None
    print(json.dumps(out))


def run_fig3(args):
    """Thermalization times of plain PT and PT+ICM against the system size
    (reduced Fig. 3): Delta(t) of Eq. 2 over doubling windows up to
    2^log2_max_fig3 sweeps, thermalization time = first window end from which
    |Delta| stays within 2 standard errors; a time that is not reached is
    reported as None (the ratio is then a bound)."""
    import torch
    from paper_1501_05630_gb300 import build, icmpt
    from paper_1501_05630_gb300.experiments import delta_curve, thermalization_time
    torch.cuda.set_device(0)
    build.build()
    ctx = icmpt.Context(0)
    lm = args.log2_max_fig3
    out = {"metric": "thermalization_speedup_vs_N", "unit": "PT sweeps / PT+ICM sweeps", "higher_is_better": True,
           "n_gpus": 1, "data": "synthetic", "config": {"workload": "fig3", "instances": args.instances,
                                                       "log2_sweeps": [4, lm], "disorder": "Gaussian"},
           "systems": {}}
    t0 = time.perf_counter()
    for sysd in FIG3:
        T = I.ladder(*sysd["T"])
        T_icm = float(T[sysd["n_c"] - 1]) + 1e-9
        rows = []
        for L in sysd["Ls"]:
            N, Nb = icmpt.lattice_size(sysd["lattice"], L)
            seed = 0x1501056300000009 + L
            J = I.couplings(Nb, I.GAUSS, seed, range(args.instances))
            s0 = I.initial_spins(N, 2 * len(T), seed, range(args.instances))
            tt = {}
            for m in ("pt", "icm"):
                c = delta_curve(ctx, sysd["lattice"], L, I.GAUSS, J, s0, T, T_icm, seed, m, 4, lm)
                tt[m] = thermalization_time(c, nsig=2.0)
            ratio = (tt["pt"] / tt["icm"]) if (tt["pt"] and tt["icm"]) else None
            row = {"N": N, "t_pt": tt["pt"], "t_icm": tt["icm"], "ratio": ratio}
            if tt["pt"] is None and tt["icm"]:
                row["ratio_at_least"] = (1 << lm) / tt["icm"]     # PT not thermalized by the last window
            rows.append(row)
        out["systems"][sysd["name"]] = rows
    largest = [r[-1]["ratio"] for r in out["systems"].values() if r[-1]["ratio"]]
    out["value"] = float(np.exp(np.mean(np.log(largest)))) if largest else None
    out["wall_s"] = time.perf_counter() - t0
    print(json.dumps(out))


# Fig. 1 systems: Table I ladders and sizes (N_c cluster temperatures), Gaussian
# disorder; p_c = site-percolation thresholds the paper quotes
FIG1 = [
    dict(name="2D", lattice=I.SQUARE2D, Ls=(16, 24, 32), T=(0.212, 1.6325, 30), n_c=30, p_c=0.592),
    dict(name="chimera", lattice=I.CHIMERA, Ls=(4, 6, 8, 10, 12), T=(0.212, 1.6325, 30), n_c=19, p_c=0.3866),
    dict(name="3D", lattice=I.CUBIC3D, Ls=(4, 6, 8, 10, 12), T=(0.42, 1.8, 26), n_c=13, p_c=0.311),
]


def run_fig1(args):
    """Fraction p(T) of potential cluster sites for the Table I systems (Fig. 1
    at reduced instance counts) and the temperature where it reaches the
    lattice's site-percolation threshold."""
    import torch
    from paper_1501_05630_gb300 import build, icmpt
    from paper_1501_05630_gb300.experiments import cluster_fraction, crossing_temperature
    torch.cuda.set_device(0)
    build.build()
    ctx = icmpt.Context(0)
    sweeps = 1 << args.log2_max_fig1
    out = {"metric": "fig1_crossing_temperature", "unit": "T at p(T) = p_c (largest N)", "higher_is_better": None,
           "n_gpus": 1, "data": "synthetic",
           "config": {"workload": "fig1", "instances": args.instances, "sweeps": sweeps, "t_meas": sweeps // 2,
                      "disorder": "Gaussian", "method": "PT + ICM at the lowest N_c temperatures (Table I)"},
           "systems": {}}
    t0 = time.perf_counter()
    updates = 0
    for sysd in FIG1:
        T = I.ladder(*sysd["T"])
        T_icm = float(T[sysd["n_c"] - 1]) + 1e-9
        res = {"p_c": sysd["p_c"], "sizes": {}}
        for L in sysd["Ls"]:
            N, Nb = icmpt.lattice_size(sysd["lattice"], L)
            seed = 0x1501056300000010 + L
            J = I.couplings(Nb, I.GAUSS, seed, range(args.instances))
            s0 = I.initial_spins(N, 2 * len(T), seed, range(args.instances))
            c = cluster_fraction(ctx, sysd["lattice"], L, I.GAUSS, J, s0, T, T_icm, seed, sweeps, sweeps // 2)
            updates += args.instances * N * 2 * len(T) * sweeps
            res["sizes"][N] = {"p": [round(float(x), 4) for x in c.p], "se": [round(float(x), 4) for x in c.se],
                               "T_cross": crossing_temperature(c, sysd["p_c"]), "p_max": round(float(c.p.max()), 4)}
        res["T"] = [round(float(x), 4) for x in T]
        out["systems"][sysd["name"]] = res
    largest = {k: v["sizes"][max(v["sizes"])]["T_cross"] for k, v in out["systems"].items()}
    out["value"] = largest
    out["wall_s"] = time.perf_counter() - t0
    out["updates_per_ns"] = updates / out["wall_s"] / 1e9
    print(json.dumps(out))


def run_annealing(args):
    """Simulated annealing with and without isoenergetic cluster moves at
    equal sweeps (the ground-state use the paper proposes): mean final energy
    per spin and how often each variant reaches the lowest energy found."""
    import torch
    from paper_1501_05630_gb300 import build, icmpt
    from paper_1501_05630_gb300.experiments import anneal
    torch.cuda.set_device(0)
    build.build()
    ctx = icmpt.Context(0)
    out = {"metric": "annealing_residual_energy_per_spin", "unit": "energy/spin", "higher_is_better": False,
           "n_gpus": 1, "data": "synthetic", "config": {"workload": "annealing", "instances": args.instances,
                                                       "schedule": "T 3.0 -> 0.05 geometric, 64 steps x 32 sweeps"},
           "systems": {}}
    t0 = time.perf_counter()
    for name, lat, L in (("3D L=6 Gaussian", I.CUBIC3D, 6), ("chimera C_6 Gaussian", I.CHIMERA, 6),
                         ("2D L=16 Gaussian", I.SQUARE2D, 16)):
        N, Nb = icmpt.lattice_size(lat, L)
        seed = 0x1501056300000007 + L
        J = I.couplings(Nb, I.GAUSS, seed, range(args.instances))
        s0 = I.initial_spins(N, 2, seed, range(args.instances))
        e = {}
        for icm in (False, True):
            b = anneal(ctx, lat, L, I.GAUSS, J, s0, 3.0, 0.05, 64, 32, icm, seed)
            e[icm] = b.read_energies().min(axis=1) / N
            b.close()
        best = np.minimum(e[False], e[True])
        out["systems"][name] = {
            "mean_e_sa": float(e[False].mean()), "mean_e_sa_icm": float(e[True].mean()),
            "residual_sa": float((e[False] - best).mean()), "residual_sa_icm": float((e[True] - best).mean()),
            "frac_best_sa": float(np.mean(e[False] <= best + 1e-6)),
            "frac_best_sa_icm": float(np.mean(e[True] <= best + 1e-6))}
    out["value"] = float(np.mean([v["residual_sa_icm"] for v in out["systems"].values()]))
    out["wall_s"] = time.perf_counter() - t0
    print(json.dumps(out))


def run_percolation(args):
    """Binder ratio of the largest-cluster fraction on chimera C_8 .. C_48
    (device-drawn masks), the crossing estimate of p_c and the exponent nu
    from the growth of the slope dg/dp with M (the Supplemental Material
    prints p_c = 0.3866(3), nu = 1.39(1))."""
    import torch
    from paper_1501_05630_gb300 import build, icmpt
    torch.cuda.set_device(0)
    build.build()
    ctx = icmpt.Context(0)
    sizes, n = (8, 16, 32, 48), args.masks
    ps = np.round(np.linspace(0.370, 0.400, 7), 4)
    g = {}
    total_sites, t0 = 0, time.perf_counter()
    for M in sizes:
        N, _ = icmpt.lattice_size(I.CHIMERA, M)
        row = []
        for p in ps:
            s = icmpt.largest_clusters_random(ctx, I.CHIMERA, M, float(p), 0x1501056300000005 + M, n) / N
            row.append(0.5 * (3.0 - np.mean(s ** 4) / np.mean(s ** 2) ** 2))
            total_sites += n * N
        g[M] = np.array(row)
    wall = time.perf_counter() - t0

    def cross(a, b):
        d = b - a
        i = np.flatnonzero(np.diff(np.sign(d)) != 0)
        return [float(ps[j] - d[j] * (ps[j + 1] - ps[j]) / (d[j + 1] - d[j])) for j in i]
    out = {"metric": "percolation_sites_per_ns", "value": total_sites / wall / 1e9, "unit": "sites/ns",
           "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
           "config": {"workload": "percolation", "lattice": "chimera", "sizes": list(sizes), "masks_per_p": n,
                      "p": ps.tolist()},
           "binder": {f"C{M}": [round(float(x), 4) for x in g[M]] for M in sizes},
           "crossings": {f"C{a}_C{b}": cross(g[a], g[b]) for a, b in zip(sizes[:-1], sizes[1:])},
           "paper_pc": 0.3866, "wall_s": wall}
    # finite-size scaling: near p_c, g depends on (p - p_c) M^(1/nu), so the
    # slope dg/dp at p_c grows as M^(1/nu).  Slopes: derivative of a cubic fit
    # of g(p) at the crossing of the two largest sizes; nu from a line through
    # (log M, log slope) over all sizes but the smallest (the largest
    # corrections to scaling are there)
    last = out["crossings"][f"C{sizes[-2]}_C{sizes[-1]}"]
    p0 = last[0] if last else 0.3866
    slope = {M: float(np.polyval(np.polyder(np.polyfit(ps, g[M], 3)), p0)) for M in sizes}
    lm = np.log(np.array(sizes[1:], dtype=np.float64))
    ls = np.log(np.abs([slope[M] for M in sizes[1:]]))
    out["binder_slope_at"] = round(float(p0), 4)
    out["binder_slope"] = {f"C{M}": round(slope[M], 3) for M in sizes}
    out["nu_pairs"] = {f"C{a}_C{b}": round(float(np.log(b / a) / np.log(slope[b] / slope[a])), 3)
                       for a, b in zip(sizes[:-1], sizes[1:])}
    out["nu_fit"] = round(float(1.0 / np.polyfit(lm, ls, 1)[0]), 3)
    out["paper_nu"] = 1.39
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="3d_gauss_L8", choices=sorted(WORKLOADS) + ["serving", "3d_gauss_mixed", "percolation", "thermalization",
                                                                   "annealing", "fig1", "fig3", "icm_frequency"])
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--quantum", type=int, default=64)
    ap.add_argument("--max-sweeps", type=int, default=1 << 14)
    ap.add_argument("--slots", type=int, default=64)
    ap.add_argument("--serving-nT", default="16,24,32")
    ap.add_argument("--alone-sample", type=int, default=3, help="serving: one-at-a-time requests per menu kind")
    ap.add_argument("--alone-seconds", type=float, default=40.0,
                    help="serving: start one-at-a-time requests while this many seconds last")
    ap.add_argument("--no-serving", action="store_true",
                    help="default workload: leave out the serving leg (and the mixed-size leg)")
    ap.add_argument("--no-phases", action="store_true", help="leave out the sweep-only / ICM-only launches")
    ap.add_argument("--no-mixed", action="store_true", help="default workload: leave out the mixed-size leg")
    ap.add_argument("--team-threads", default="",
                    help="3d_gauss_mixed shared: threads per instance of each size (comma list) instead of tuning")
    ap.add_argument("--mixed-mode", default="shared", choices=["shared", "graph"],
                    help="3d_gauss_mixed: one shared persistent kernel, or one kernel per size in a graph")
    ap.add_argument("--masks", type=int, default=200000)
    ap.add_argument("--instances", type=int, default=256)
    ap.add_argument("--log2-max", type=int, default=17)
    ap.add_argument("--log2-max-fig1", type=int, default=14, help="fig1: sweeps = 2^this, measured over the second half")
    ap.add_argument("--log2-max-fig3", type=int, default=18, help="fig3: the last doubling window ends at 2^this")
    ap.add_argument("--sweeps-per-step", type=int, default=256)
    ap.add_argument("--cluster", type=int, default=0, help="run each instance on a thread-block cluster of K CTAs")
    ap.add_argument("--cluster-threads", type=int, default=512)
    ap.add_argument("--n-inst", type=int, default=0, help="instances per GPU instead of the workload's own count")
    ap.add_argument("--cluster-growth", type=int, default=-1,
                    help="cluster layout's growth: 1 union-find, 0 label propagation, -1 the library's choice")
    ap.add_argument("--ref-sweeps", type=int, default=32)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()
    if args.workload == "serving":
        if int(os.environ.get("RANK", "0")) == 0:
            run_serving(args)
        return
    if args.workload == "thermalization":
        if int(os.environ.get("RANK", "0")) == 0:
            run_thermalization(args)
        return
    if args.workload == "icm_frequency":
        if int(os.environ.get("RANK", "0")) == 0:
            run_icm_frequency(args)
        return
    if args.workload == "fig3":
        if int(os.environ.get("RANK", "0")) == 0:
            run_fig3(args)
        return
    if args.workload == "fig1":
        if int(os.environ.get("RANK", "0")) == 0:
            run_fig1(args)
        return
    if args.workload == "annealing":
        if int(os.environ.get("RANK", "0")) == 0:
            run_annealing(args)
        return
    if args.workload == "percolation":
        if int(os.environ.get("RANK", "0")) == 0:
            run_percolation(args)
        return
    if args.workload == "3d_gauss_mixed":
        if int(os.environ.get("RANK", "0")) == 0:
            run_mixed(args)
        return
    wl = WORKLOADS[args.workload]
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, wl, rank)
        return

    import torch
    import torch.distributed as dist
    from paper_1501_05630_gb300 import build, icmpt

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    stream = torch.cuda.current_stream()
    ctx = icmpt.Context(local, stream.cuda_stream)

    n = args.n_inst or wl["n_inst"]
    T = I.ladder(*wl["T"])
    N, Nb = icmpt.lattice_size(wl["lattice"], wl["L"])
    R = 2 * len(T)
    from paper_1501_05630_gb300 import sharding
    ids = sharding.instance_range(rank, world, n)               # weak scaling: disjoint instances per rank
    J = I.couplings(Nb, wl["disorder"], wl["seed"], ids)
    s0 = I.initial_spins(N, R, wl["seed"], ids)
    J_pin = torch.from_numpy(J).pin_memory()
    s_pin = torch.from_numpy(s0).pin_memory()
    J_dev, s_dev = J_pin.cuda(), s_pin.cuda()
    b = icmpt.Batch(ctx, wl["lattice"], wl["L"], wl["disorder"], J_dev, T, wl["T_icm"], wl["seed"],
                    spins=s_dev, instance_ids=ids)
    if args.cluster:
        b.set_cluster_growth(args.cluster_growth)
        b.set_cluster(args.cluster, args.cluster_threads)     # one instance per thread-block cluster
    info = b.info()
    S = args.sweeps_per_step
    n_icm = int(np.sum(T <= wl["T_icm"]))
    updates_per_step = n * R * N * S
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # > L2 (129 MB)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        b.run(S)
    barrier()
    launches0 = b.info()["launches"]
    b.clear_observables()                                         # cluster-move counters of the timed steps
    barrier()
    times = []
    with ClockSampler(local) as clk:
        barrier()
        t_wall = time.perf_counter()
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.run(S)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        barrier()
        t_wall = time.perf_counter() - t_wall
    launches = b.info()["launches"] - launches0
    ms = float(np.sum(times))
    if world > 1:
        tt = torch.tensor([ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    value = updates_per_step * args.steps * world / (ms * 1e6)
    icm_attempts_per_s = n * n_icm * S * args.steps * world / (ms * 1e-3)
    stats = b.read_icm_stats().astype(np.float64)
    icm_moves_per_s = stats[:, 0].sum() * world / (ms * 1e-3)     # pairs with n > 0 (a cluster moved)

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        hb = icmpt.Batch(ctx, wl["lattice"], wl["L"], wl["disorder"], J_pin.numpy(), T, wl["T_icm"], wl["seed"],
                         spins=s_pin.numpy(), instance_ids=ids)
        if args.cluster:
            hb.set_cluster_growth(args.cluster_growth)
            hb.set_cluster(args.cluster, args.cluster_threads)
        for _ in range(2):
            hb.load(J_pin.numpy(), s_pin.numpy())
            hb.run(S)
            hb.read_observables(hist=False)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            hb.load(J_pin.numpy(), s_pin.numpy())          # H2D: couplings + spins
            hb.run(S)
            o = hb.read_observables(hist=False)            # D2H: accumulators (waits)
        barrier()
        dt = time.perf_counter() - t0
        if world > 1:
            tt = torch.tensor([dt], device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            dt = float(tt.item())
        h2d = J.nbytes + s0.nbytes
        d2h = o.accE.nbytes + 4 * o.acc_n.nbytes + o.n_meas.nbytes
        e2e = {"value": updates_per_step * args.steps * world / (dt * 1e9), "unit": "updates/ns",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}
        hb.close()

    peaks, peak_src = _peaks()
    z = {I.SQUARE2D: 4, I.CUBIC3D: 6, I.CHIMERA: 6, I.HYPERCUBIC4D: 8}[wl["lattice"]]
    ops_per_update = ALG_OPS[wl["disorder"]](z)
    per_launch_ms = ms / max(args.steps, 1)
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    peak = n_sm * 128 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12                  # issue limit, Tops/s
    # the whole step: the sweep's algorithmic ops plus the cluster moves' (from
    # the device counters of the timed steps), over the fused kernel's time
    icm_ops_step = icm_ops(N, Nb, z, n_icm, n * n_icm * S, stats[:, 0].sum() / args.steps,
                           stats[:, 1].sum() / args.steps, b.cluster_growth() > 0)
    achieved = (updates_per_step * ops_per_update + icm_ops_step) / (per_launch_ms * 1e-3) / 1e12
    # executed thread-instructions per update (ncu) give the issue utilisation
    # beside the algorithmic fraction
    ipu = None if args.cluster else recorded_counter(args.workload, "instructions_per_update")
    issue_frac = (updates_per_step * ipu / (per_launch_ms * 1e-3) / 1e12) / peak if ipu else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                "frac": achieved / peak, "traffic": None if args.cluster else recorded_traffic(args.workload),
                "kernel": "cluster_kernel" if args.cluster else "fused_kernel",
                "ops_per_update": ops_per_update, "icm_ops_per_step": icm_ops_step,
                "instructions_per_update": ipu, "issue_frac": issue_frac,
                "peak_note": f"issue limit: {n_sm} SMs x 128 thread-instr/clk x sm_max_mhz ({peak_src}); "
                             "frac = algorithmic ops (Metropolis per update + cluster moves from the device "
                             "counters), issue_frac = executed instructions (ncu); traffic = DRAM bytes per launch"}
    if not args.no_phases:
        roofline.update(phase_fractions(b, stream, flush, S, n, updates_per_step, ops_per_update, N, Nb, z,
                                        n_icm, peak))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        ref_sweeps = calibrate_sweeps(wl, cores, args.cpu_seconds)
        v, dt, _ = oracle_throughput(wl, ref_sweeps, 2 * cores, cores)
        cpu = {"value": v, "unit": "updates/ns", "cores": cores, "kind": "oracle",
               "sample": f"{2 * cores} of the {wl['n_inst']} instances x {ref_sweeps} sweeps "
                         f"({dt:.1f} s on {cores} threads)"}

    if rank == 0:
        out = {
            "metric": "spin_updates_per_ns", "value": value, "unit": "updates/ns", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if wl["disorder"] == I.GAUSS else "u32",
            "data": "synthetic",
            "config": {"workload": args.workload,
                       "desc": wl["desc"] + (f"; run with {n} instances per GPU" if args.n_inst else ""),
                       "instances_per_gpu": n,
                       "sweeps_per_step": S, "n_icm": n_icm, "l2": "flushed between steps (256 MB write)",
                       "threads": info["threads"], "ctas_per_sm": info["ctas_per_sm"], "grid": info["grid"],
                       "smem_bytes": info["smem_bytes"],
                       "cluster": {"K": args.cluster, "clusters": info["grid"] // args.cluster,
                                   "union_find_pairs_per_group": b.cluster_growth()} if args.cluster else None},
            "icm_moves_per_s": icm_moves_per_s, "icm_attempts_per_s": icm_attempts_per_s,
            "e2e": e2e, "gpu_launches": int(launches), "roofline": roofline, "cpu_baseline": cpu,
            "clocks": clk.summary(), "wall_s": t_wall,
        }
        if world == 1 and args.workload == "3d_gauss_L8" and not args.no_serving:
            # the metric's second half: instances thermalized/s and latency of
            # the served form (workload 5), against the plain method one at a time
            sv = serving_measurement(args)
            out.update({k: sv[k] for k in ("instances_thermalized_per_s", "latency_p50_s", "latency_p99_s")})
            sv.pop("clocks", None)
            out["serving"] = sv
        if world == 1 and args.workload == "3d_gauss_L8" and not (args.no_mixed or args.no_serving):
            # uneven sizes (3D L = 4..12) sharing one persistent kernel launch
            mx = mixed_measurement(args, 5, 3, "shared")
            out["mixed_sizes"] = {k: mx[k] for k in ("value", "unit", "ms_per_step", "steps", "warmup", "gpu_launches",
                                                     "clocks")}
            out["mixed_sizes"]["config"] = mx["config"]
            # the largest serving size on 8-CTA thread-block clusters: 20 instances,
            # and one per resident cluster of 8 x 512 (36 on a full GB300)
            out["large_instances"] = {"workload": "2D EA L=128 periodic (16384 spins), +-J, 32 T geometric [0.2,1.5], "
                                                  "ICM T<=1.0, one instance per 8-CTA cluster of 512 threads",
                                      "x20": cluster_measurement(20), "x36": cluster_measurement(36)}
        print(json.dumps(out))
    b.close()
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
