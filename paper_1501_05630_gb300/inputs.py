"""Seeded synthetic inputs shared by the CUDA path, the CPU oracle and the benchmark.

This module holds no arithmetic of the method (no energies, no Monte Carlo, no
cluster building).  It only turns (seed, instance id) into the arrays a run
starts from, so that both sides of every comparison receive identical inputs:

* temperature ladders, geometric between T_min and T_max (the paper's Table I
  lists T_min, T_max and N_T per topology);
* disorder: Gaussian couplings N(0, 1) ("Benchmark model and observables") or
  bimodal +-1 couplings (the paper's remark on bimodal disorder), one value
  per bond in the caller's bond order;
* bond dilution: each bond absent (J = 0) independently with a given
  probability, the diluted lattices the paper's introduction cites;
* initial spins, uniformly random +-1 for every replica;
* random site masks with occupation probability p (site percolation, as in
  the Supplemental Material).

Sizes (number of sites and bonds) are passed in by the caller, which takes
them from its own geometry.
"""
from __future__ import annotations

import numpy as np

#: lattice kinds, in the order used by the C ABI
SQUARE2D, CUBIC3D, CHIMERA, HYPERCUBIC4D = 0, 1, 2, 3
#: disorder kinds, in the order used by the C ABI
PM_J, GAUSS = 0, 1


def _rng(seed: int, instance_id: int, stream: int) -> np.random.Generator:
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    ss = np.random.SeedSequence([seed & 0xFFFFFFFF, seed >> 32, int(instance_id), int(stream)])
    return np.random.Generator(np.random.PCG64(ss))


def ladder(T_min: float, T_max: float, n_T: int) -> np.ndarray:
    """Geometric temperature ladder T_k = T_min (T_max/T_min)^(k/(n_T-1)), ascending."""
    if n_T == 1:
        return np.array([float(T_min)])
    k = np.arange(n_T, dtype=np.float64)
    return float(T_min) * (float(T_max) / float(T_min)) ** (k / (n_T - 1))


def couplings(n_bonds: int, disorder: int, seed: int, instance_ids) -> np.ndarray:
    """Couplings J[instance][bond]: int8 +-1 for PM_J, float32 N(0,1) for GAUSS."""
    ids = list(instance_ids)
    if disorder == PM_J:
        out = np.empty((len(ids), n_bonds), dtype=np.int8)
        for a, inst in enumerate(ids):
            out[a] = 1 - 2 * _rng(seed, inst, 3).integers(0, 2, size=n_bonds, dtype=np.int8)
    elif disorder == GAUSS:
        out = np.empty((len(ids), n_bonds), dtype=np.float32)
        for a, inst in enumerate(ids):
            out[a] = _rng(seed, inst, 3).standard_normal(n_bonds).astype(np.float32)
    else:
        raise ValueError(f"unknown disorder kind {disorder}")
    return out


def dilute(J: np.ndarray, fraction: float, seed: int, instance_ids) -> np.ndarray:
    """Copy of J[instance][bond] with each bond set to 0 (absent) independently
    with probability `fraction`; the pattern depends on (seed, instance id)."""
    ids = list(instance_ids)
    out = np.array(J, copy=True)
    if out.shape[0] != len(ids):
        raise ValueError("one row of couplings per instance id")
    for a, inst in enumerate(ids):
        out[a][_rng(seed, inst, 6).random(out.shape[1]) < fraction] = 0
    return out


def initial_spins(n_sites: int, n_replicas: int, seed: int, instance_ids) -> np.ndarray:
    """Random +-1 spins s[instance][replica][site] (int8)."""
    ids = list(instance_ids)
    out = np.empty((len(ids), n_replicas, n_sites), dtype=np.int8)
    for a, inst in enumerate(ids):
        out[a] = 1 - 2 * _rng(seed, inst, 4).integers(0, 2, size=(n_replicas, n_sites), dtype=np.int8)
    return out


def site_masks(n_sites: int, p: float, seed: int, n: int) -> np.ndarray:
    """n random occupation masks (uint8 0/1) with site probability p."""
    rng = _rng(seed, 0, 5)
    return (rng.random((n, n_sites)) < p).astype(np.uint8)


# The five workloads of the benchmark table, as plain parameters.
WORKLOADS = {
    "2d_pmj_L8": dict(lattice=SQUARE2D, L=8, disorder=PM_J, n_inst=1, T=(0.2, 1.5, 16),
                      T_icm=1.0, sweeps=4096, seed=0x1501056300000001),
    "3d_gauss_L8": dict(lattice=CUBIC3D, L=8, disorder=GAUSS, n_inst=1000, T=(0.2, 2.0, 24),
                        T_icm=1.0, sweeps=1 << 16, seed=0x1501056300000002),
    "chimera_pmj_C8": dict(lattice=CHIMERA, L=8, disorder=PM_J, n_inst=10000, T=(0.2, 3.0, 30),
                           T_icm=1.5, sweeps=1 << 16, seed=0x1501056300000003),
}
