"""Run by tests/test_checked_build.py in a child process (it is not a test
module): loads the checked build of the library (every guarded index of the
fused and cluster kernels tested against its bound), runs +-J cases of several
shapes and layouts against the oracle, bit for bit, and a Gaussian case, then
prints the check words as JSON.  A child process, so that the checked library is the only
one loaded."""
import ctypes
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import oracle as O  # noqa: E402
from paper_1501_05630_gb300 import build, icmpt, inputs as I  # noqa: E402

lib = icmpt.load_library(build.build(checked=True))
lib.icm_debug_check.argtypes = [ctypes.c_void_p, ctypes.c_int]
lib.icm_debug_check.restype = ctypes.c_int
lib.icm_debug_check_cluster.argtypes = [ctypes.c_void_p, ctypes.c_int]
lib.icm_debug_check_cluster.restype = ctypes.c_int
ctx = icmpt.Context(0)

CASES = [  # lattice, L, n_T, T_max, T_icm, dilution, threads or (K, threads) of a thread-block cluster
    (O.SQUARE2D, 8, 16, 1.5, 1.0, 0.0, None),
    (O.CUBIC3D, 4, 24, 2.0, 1.0, 0.0, None),
    (O.CHIMERA, 3, 30, 3.0, 1.5, 0.0, None),
    (O.HYPERCUBIC4D, 4, 8, 3.0, 1.5, 0.0, None),
    (O.SQUARE2D, 8, 12, 1.5, 1.0, 0.3, None),
    (O.CUBIC3D, 6, 10, 2.0, 1.0, 0.0, 256),
    (O.SQUARE2D, 16, 16, 1.5, 1.0, 0.0, (4, 64)),
    (O.CUBIC3D, 8, 10, 2.0, 1.0, 0.3, (2, 128)),
    (O.HYPERCUBIC4D, 4, 8, 3.0, 1.5, 0.0, (4, 32)),
]
mismatch = []
for ci, (lat, L, nT, th, ticm, dil, threads) in enumerate(CASES):
    g = O.Geometry(lat, L)
    T = I.ladder(0.2, th, nT)
    J = I.couplings(g.Nb, I.PM_J, 50 + ci, range(2))
    if dil:
        J = I.dilute(J, dil, 50 + ci, range(2))
    s0 = I.initial_spins(g.N, 2 * nT, 50 + ci, range(2))
    b = icmpt.Batch(ctx, lat, L, I.PM_J, J, T, ticm, 50 + ci, spins=s0)
    if isinstance(threads, tuple):
        b.set_cluster(*threads)
    elif threads:
        b.set_threads(threads)
    b.set_schedule(trace=1, t_meas=5)
    b.run(20)
    spins, E, o = b.read_spins(), b.read_energies(), b.read_observables()
    for a in range(2):
        r = O.Instance(g, J[a].astype(np.float64), T, s0[a], pm=True, T_icm=ticm, seed=50 + ci, inst=a, t_meas=5)
        r.run(20)
        if not (np.array_equal(spins[a], r.s) and np.array_equal(E[a], r.E) and np.array_equal(o.hist[a], r.hist)):
            mismatch.append([ci, a])
    b.close()
g = O.Geometry(O.CUBIC3D, 8)
T = I.ladder(0.2, 2.0, 24)
b = icmpt.Batch(ctx, O.CUBIC3D, 8, I.GAUSS, I.couplings(g.Nb, I.GAUSS, 9, range(16)), T, 1.0, 9,
                spins=I.initial_spins(g.N, 48, 9, range(16)))
b.set_schedule(trace=1)
b.run(30)
b.read_trace()
ctx.sync()
word = (ctypes.c_uint * 4)()
rc = lib.icm_debug_check(word, 1)
cword = (ctypes.c_uint * 4)()
rc_cluster = lib.icm_debug_check_cluster(cword, 1)
print(json.dumps({"rc": rc, "check": list(word), "rc_cluster": rc_cluster, "check_cluster": list(cword),
                  "mismatch": mismatch}))
