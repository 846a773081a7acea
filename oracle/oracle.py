"""Python front end of the CPU oracle (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may use
this module.  It compiles ``icm_oracle.c`` with gcc into ``oracle/_build`` and
calls it through ctypes.  It imports nothing from the CUDA library package.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "icm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

SQUARE2D, CUBIC3D, CHIMERA, HYPERCUBIC4D = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle shared library (plain C, gcc)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Problem(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int32), ("Nb", ctypes.c_int32), ("nT", ctypes.c_int32), ("pm", ctypes.c_int32),
        ("bi", ctypes.c_void_p), ("bj", ctypes.c_void_p), ("J", ctypes.c_void_p),
        ("color", ctypes.c_void_p), ("T", ctypes.c_void_p), ("T_icm", ctypes.c_double),
        ("icm_every", ctypes.c_int32), ("swap_every", ctypes.c_int32),
        ("enable_2a", ctypes.c_int32), ("enable_metropolis", ctypes.c_int32),
        ("t_meas", ctypes.c_int64), ("seed", ctypes.c_uint64),
        ("inst", ctypes.c_uint32), ("pad2_", ctypes.c_uint32),
    ]


class _State(ctypes.Structure):
    _fields_ = [
        ("s", ctypes.c_void_p), ("E", ctypes.c_void_p), ("accE", ctypes.c_void_p),
        ("acc_n", ctypes.c_void_p), ("acc_q2", ctypes.c_void_p), ("acc_pmin", ctypes.c_void_p),
        ("acc_d", ctypes.c_void_p), ("hist", ctypes.c_void_p), ("n_meas", ctypes.c_void_p),
        ("t", ctypes.c_uint32), ("pad_", ctypes.c_uint32),
    ]


class _Trace(ctypes.Structure):
    _fields_ = [
        ("n_pre", ctypes.c_void_p), ("flip2a", ctypes.c_void_p), ("seed_site", ctypes.c_void_p),
        ("csize", ctypes.c_void_p), ("esum_before", ctypes.c_void_p), ("esum_after", ctypes.c_void_p),
        ("swap_acc", ctypes.c_void_p), ("cmask", ctypes.c_void_p),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.orc_philox4x32_10.argtypes = [ctypes.c_void_p] * 3
            L.orc_geometry_sizes.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
            L.orc_geometry.argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.c_void_p] * 3
            L.orc_run.argtypes = [ctypes.POINTER(_Problem), ctypes.POINTER(_State), ctypes.c_uint32,
                                  ctypes.POINTER(_Trace)]
            L.orc_largest_clusters.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
            L.orc_energy.argtypes = [ctypes.POINTER(_Problem), ctypes.c_void_p]
            L.orc_energy.restype = ctypes.c_double
            _lib = L
    return _lib


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one counter (4 x uint32) under one key (2 x uint32)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def philox_couplings(n_bonds: int, pm: bool, seed: int, instance_ids) -> np.ndarray:
    """Disorder drawn from the seed (the paper's "Benchmark model and
    observables": J = +-1 with probability 1/2, or Gaussian with mean 0 and
    variance 1), Philox domain 3 keyed by instance id and bond index:
      +-J bond b: the top bit of word b & 3 of counter {b >> 2, 0, 0, 3<<24 | id},
        0 -> +1, 1 -> -1 (int8);
      Gaussian bond b: words o0, o1 of counter {b, 1, 0, 3<<24 | id}, Box-Muller
        in double, J = sqrt(-2 ln u1) cos(2 pi u2), u1 = (o0 + 1) 2^-32,
        u2 = o1 2^-32, rounded to fp32.
    Returns [len(instance_ids)][n_bonds]."""
    import math
    key = [int(seed) & 0xFFFFFFFF, (int(seed) >> 32) & 0xFFFFFFFF]
    ids = list(instance_ids)
    out = np.empty((len(ids), n_bonds), dtype=np.int8 if pm else np.float32)
    for a, inst in enumerate(ids):
        c3 = (3 << 24) | int(inst)
        for b in range(n_bonds):
            if pm:
                o = philox([b >> 2, 0, 0, c3], key)
                out[a, b] = -1 if (int(o[b & 3]) >> 31) else 1
            else:
                o = philox([b, 1, 0, c3], key)
                u1 = (int(o[0]) + 1) / 4294967296.0
                u2 = int(o[1]) / 4294967296.0
                out[a, b] = np.float32(math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2))
    return out


class Geometry:
    """Sites, bonds (in bond order) and the two-colouring of one lattice."""

    def __init__(self, kind: int, L: int):
        N = ctypes.c_int32()
        Nb = ctypes.c_int32()
        if lib().orc_geometry_sizes(kind, L, ctypes.byref(N), ctypes.byref(Nb)):
            raise ValueError("bad lattice")
        self.kind, self.L, self.N, self.Nb = kind, L, N.value, Nb.value
        self.bi = np.zeros(self.Nb, dtype=np.int32)
        self.bj = np.zeros(self.Nb, dtype=np.int32)
        self.color = np.zeros(self.N, dtype=np.uint8)
        if lib().orc_geometry(kind, L, _p(self.bi), _p(self.bj), _p(self.color)):
            raise RuntimeError("geometry failed")


class Instance:
    """One disorder instance with 2 N_T replicas, run by the oracle."""

    def __init__(self, geom: Geometry, J, T, spins, *, pm: bool, T_icm: float, seed: int,
                 inst: int, icm_every: int = 1, swap_every: int = 1, enable_2a: bool = True,
                 enable_metropolis: bool = True, t_meas: int = 0, t0: int = 0):
        self.g = geom
        self.pm = bool(pm)
        self.J = np.ascontiguousarray(J, dtype=np.float64)
        self.nb_present = int(np.count_nonzero(self.J))     # bonds with J = 0 are absent (dilution)
        self.T = np.ascontiguousarray(T, dtype=np.float64)
        nT = len(self.T)
        self.nT = nT
        self.s = np.ascontiguousarray(spins, dtype=np.int8).reshape(2 * nT, geom.N).copy()
        self.E = np.zeros(2 * nT)
        self.accE = np.zeros(nT)
        self.acc_n = np.zeros(nT, dtype=np.int64)
        self.acc_q2 = np.zeros(nT, dtype=np.int64)
        self.acc_pmin = np.zeros(nT, dtype=np.int64)
        self.acc_d = np.zeros(nT, dtype=np.int64)
        self.hist = np.zeros((nT, geom.N + 1), dtype=np.int64)
        self.n_meas = np.zeros(1, dtype=np.int64)
        self._P = _Problem(geom.N, geom.Nb, nT, int(self.pm), _p(geom.bi), _p(geom.bj), _p(self.J),
                           _p(geom.color), _p(self.T), float(T_icm), int(icm_every), int(swap_every),
                           int(enable_2a), int(enable_metropolis), int(t_meas),
                           int(seed) & 0xFFFFFFFFFFFFFFFF, int(inst), 0)
        self._S = _State(_p(self.s), _p(self.E), _p(self.accE), _p(self.acc_n), _p(self.acc_q2),
                         _p(self.acc_pmin), _p(self.acc_d), _p(self.hist), _p(self.n_meas), int(t0), 0)

    @property
    def t(self) -> int:
        return self._S.t

    def run(self, n_sweeps: int, trace: bool = False):
        tr = None
        if trace:
            nT = self.nT
            tr = dict(n_pre=np.zeros(nT, np.int32), flip2a=np.zeros(nT, np.int32),
                      seed_site=np.zeros(nT, np.int32), csize=np.zeros(nT, np.int32),
                      esum_before=np.zeros(nT), esum_after=np.zeros(nT),
                      swap_acc=np.zeros((2, max(nT - 1, 1)), np.uint8),
                      cmask=np.zeros((nT, self.g.N), np.uint8))
            ct = _Trace(*[_p(tr[f]) for f in ("n_pre", "flip2a", "seed_site", "csize",
                                              "esum_before", "esum_after", "swap_acc", "cmask")])
            ptr = ctypes.byref(ct)
        else:
            ptr = None
        rc = lib().orc_run(ctypes.byref(self._P), ctypes.byref(self._S), int(n_sweeps), ptr)
        if rc:
            raise RuntimeError(f"orc_run failed: {rc}")
        return tr

    def energy(self, s) -> float:
        s = np.ascontiguousarray(s, dtype=np.int8)
        return lib().orc_energy(ctypes.byref(self._P), _p(s))

    def observables(self) -> dict:
        """Per-temperature averages over the measured sweeps."""
        m = max(int(self.n_meas[0]), 1)
        N, Nb = self.g.N, max(self.nb_present, 1)
        return dict(
            e=self.accE / (2.0 * N * m),
            q_l=1.0 - 2.0 * self.acc_d / (Nb * m),
            q2=self.acc_q2 / (float(N) * N * m),
            p=self.acc_pmin / (float(N) * m),
            n_frac=self.acc_n / (float(N) * m),
            P_n=self.hist / float(m),
            n_meas=int(self.n_meas[0]),
        )


def largest_clusters(geom: Geometry, masks) -> np.ndarray:
    """Largest occupied cluster of every mask (site percolation), int32 [n]."""
    m = np.ascontiguousarray(masks, dtype=np.uint8).reshape(-1, geom.N)
    out = np.zeros(m.shape[0], dtype=np.int32)
    if lib().orc_largest_clusters(geom.N, geom.Nb, _p(geom.bi), _p(geom.bj), m.shape[0], _p(m), _p(out)):
        raise RuntimeError("orc_largest_clusters failed")
    return out


def binder_ratio(smax_fraction) -> float:
    """g = (1/2)(3 - <s^4>/<s^2>^2) of the largest-cluster fraction (Supplemental Material)."""
    s = np.asarray(smax_fraction, dtype=np.float64)
    return 0.5 * (3.0 - np.mean(s ** 4) / np.mean(s ** 2) ** 2)
