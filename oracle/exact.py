"""Exact enumeration of small Ising spin glasses (test infrastructure only).

For N <= 20 spins every configuration is enumerated, which gives the
equilibrium values that the Monte Carlo chain must reproduce:

* the mean energy per spin, <H>/N with H = -sum_<ij> J_ij s_i s_j
  ("Benchmark model and observables");
* the link overlap of two independent replicas,
  <q_l> = (1/N_b) sum_<ij> <s_i s_j>^2  (the replicas are independent, so
  <s_i^1 s_j^1 s_i^2 s_j^2> factorises into <s_i s_j>^2);
* the distribution of n = #{i : s_i^1 != s_i^2} between two independent
  replicas, P(n) = sum_v g(v) [popcount(v) = n] with
  g(v) = sum_s p(s) p(s xor v), computed by a Walsh-Hadamard transform.
"""
from __future__ import annotations

import numpy as np


def all_states(N: int) -> np.ndarray:
    """int8 [2^N][N]; bit i of the state index set means s_i = -1."""
    idx = np.arange(1 << N, dtype=np.int64)
    bits = (idx[:, None] >> np.arange(N)) & 1
    return (1 - 2 * bits).astype(np.int8)


def energies(bi, bj, J, states: np.ndarray) -> np.ndarray:
    s = states.astype(np.float64)
    return -(s[:, bi] * s[:, bj]) @ np.asarray(J, dtype=np.float64)


def _wht(a: np.ndarray) -> np.ndarray:
    a = a.copy()
    h = 1
    n = a.shape[0]
    while h < n:
        a = a.reshape(-1, 2, h)
        x, y = a[:, 0, :].copy(), a[:, 1, :].copy()
        a[:, 0, :], a[:, 1, :] = x + y, x - y
        a = a.reshape(n)
        h *= 2
    return a


def thermal(bi, bj, J, N: int, T: float, states=None, E=None) -> dict:
    """Exact equilibrium observables at temperature T."""
    if states is None:
        states = all_states(N)
    if E is None:
        E = energies(bi, bj, J, states)
    w = np.exp(-(E - E.min()) / T)
    p = w / w.sum()
    Nb = len(bi)
    s = states.astype(np.float64)
    links = s[:, bi] * s[:, bj]                  # [states][bonds]
    corr = p @ links                             # <s_i s_j> per bond
    g = _wht(_wht(p) ** 2) / float(1 << N)       # g(v) = sum_s p(s) p(s^v)
    pop = np.array([bin(v).count("1") for v in range(1 << N)])
    P_n = np.bincount(pop, weights=g, minlength=N + 1)
    n = np.arange(N + 1)
    return dict(
        e=float(p @ E) / N,
        q_l=float(np.sum(corr ** 2) / Nb),
        P_n=P_n,
        q2=float(np.sum(P_n * ((N - 2 * n) / N) ** 2)),
        n_frac=float(np.sum(P_n * n) / N),
        p=float(np.sum(P_n * np.minimum(n, N - n)) / N),
        E_min=float(E.min()),
    )
