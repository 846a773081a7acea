"""Oracle pins for the widened geometry: 4D hypercubic lattices and diluted
lattices (bonds with J = 0 absent from the lattice).

* 4D geometry: bond count 4N, degree 8, proper two-colouring; the chain
  (Metropolis + ICM + PT) on the L = 2 hypercube (N = 16) agrees with exact
  enumeration.
* Dilution, closed form: a 2D torus with every vertical bond absent is L
  independent rings.  A ring with couplings J_1..J_L has
  Z = prod 2 cosh(beta J_b) + prod 2 sinh(beta J_b) (transfer matrix), hence
  <s_i s_j>_b = (a tanh(beta J_b) + b coth(beta J_b)) / (a + b) with
  a = prod 2 cosh, b = prod 2 sinh; e = -sum_b J_b <s s>_b / N and, for two
  independent replicas, q_l = sum_b <s s>_b^2 / N_b(present).  A cluster of
  the isoenergetic move cannot leave its ring, so its size is at most L.
  On diluted instances a zero-energy proposal is accepted with probability
  1/2: with the deterministic flip, the checkerboard sweep is not ergodic
  on such rings and misses the closed form by many standard errors.
* All bonds absent: every energy is 0, every proposal has Delta E = 0 and is
  accepted with probability 1/2, clusters are single sites and every swap is
  accepted.
"""

import numpy as np
import pytest
import statcheck

from oracle import exact
from oracle import oracle as O
from paper_1501_05630_gb300 import inputs as I


# ----------------------------------------------------------------------------- 4D geometry
@pytest.mark.parametrize("L", [4, 6])
def test_geometry_4d_invariants(L):
    g = O.Geometry(O.HYPERCUBIC4D, L)
    N = L ** 4
    assert (g.N, g.Nb) == (N, 4 * N)
    assert np.all(g.bi != g.bj)
    assert np.all(g.color[g.bi] != g.color[g.bj])
    assert np.sum(g.color == 0) == N // 2
    d = np.bincount(np.concatenate([g.bi, g.bj]), minlength=N)
    assert np.all(d == 8)
    pairs = set(zip(np.minimum(g.bi, g.bj), np.maximum(g.bi, g.bj)))
    assert len(pairs) == g.Nb
    # bond 4i + d joins i to its +1 neighbour along axis d
    i = np.arange(N)
    x = np.stack([(i // L ** a) % L for a in range(4)], 1)
    for a in range(4):
        y = x.copy()
        y[:, a] = (y[:, a] + 1) % L
        j = (y * (L ** np.arange(4))).sum(1)
        assert np.array_equal(g.bi[4 * i + a], i) and np.array_equal(g.bj[4 * i + a], j)


def test_geometry_4d_smallest_torus_keeps_doubled_bonds():
    g = O.Geometry(O.HYPERCUBIC4D, 2)
    assert (g.N, g.Nb) == (16, 64)
    d = np.bincount(np.concatenate([g.bi, g.bj]), minlength=16)
    assert np.all(d == 8)


def _agree(samples, target):
    """Samples agree with target at three standard errors (one Hotelling test
    over all components, statcheck); returns (ok, sample mean, test figures)."""
    d = np.asarray(samples, dtype=np.float64) - np.asarray(target, dtype=np.float64)
    r = statcheck.hotelling(d)
    return r["p"] >= statcheck.P_3SIGMA, d.mean(0) + target, r


@pytest.mark.parametrize("disorder", [I.PM_J, I.GAUSS])
def test_4d_chain_matches_exact_enumeration(disorder):
    g = O.Geometry(O.HYPERCUBIC4D, 2)
    seed = 44
    J = I.couplings(g.Nb, disorder, seed, [0])[0].astype(np.float64)
    T = I.ladder(0.6, 3.0, 6)
    obs = []
    for c in range(40):
        s0 = I.initial_spins(g.N, 2 * len(T), seed, [1000 + c])[0]
        inst = O.Instance(g, J, T, s0, pm=(disorder == I.PM_J), T_icm=1.5, seed=seed, inst=c, t_meas=500)
        inst.run(2500)
        obs.append(inst.observables())
    st = exact.all_states(g.N)
    E = exact.energies(g.bi, g.bj, J, st)
    ex = [exact.thermal(g.bi, g.bj, J, g.N, t, st, E) for t in T]
    for name in ("e", "q_l", "q2"):
        ok, mean, se = _agree([o[name] for o in obs], np.array([x[name] for x in ex]))
        assert ok, (name, mean, se, [x[name] for x in ex])


# ----------------------------------------------------------------------------- dilution
def _ring_correlations(Jring, beta):
    """<s_i s_j> of every bond of one ring (transfer matrix, closed form)."""
    K = beta * np.asarray(Jring, dtype=np.float64)
    a = np.prod(2 * np.cosh(K))
    b = np.prod(2 * np.sinh(K))
    return (a * np.tanh(K) + b / np.tanh(K)) / (a + b)


@pytest.mark.parametrize("disorder", [I.PM_J, I.GAUSS])
def test_diluted_torus_of_rings_matches_closed_form(disorder):
    L = 6
    g = O.Geometry(O.SQUARE2D, L)
    seed = 61
    J = I.couplings(g.Nb, disorder, seed, [0])[0].astype(np.float64)
    J[1::2] = 0.0                           # every +y bond absent: L rings along x
    T = I.ladder(0.5, 2.5, 6)
    obs, max_csize = [], 0
    for c in range(40):
        s0 = I.initial_spins(g.N, 2 * len(T), seed, [2000 + c])[0]
        inst = O.Instance(g, J, T, s0, pm=(disorder == I.PM_J), T_icm=1.2, seed=seed, inst=c, t_meas=400)
        inst.run(400)
        for _ in range(40):                 # the traced sweeps: cluster sizes
            tr = inst.run(40, trace=True)
            max_csize = max(max_csize, int(tr["csize"].max()))
        obs.append(inst.observables())
    assert 1 < max_csize <= L
    want_e, want_ql = [], []
    for t in T:
        ss = np.concatenate([_ring_correlations(J[2 * L * y:2 * L * (y + 1):2], 1.0 / t) for y in range(L)])
        Jx = J[0::2]
        want_e.append(-np.sum(Jx * ss) / g.N)
        want_ql.append(np.sum(ss ** 2) / (g.Nb // 2))
    for name, want in (("e", want_e), ("q_l", want_ql)):
        ok, mean, se = _agree([o[name] for o in obs], np.array(want))
        assert ok, (name, mean, se, want)


def test_fully_diluted_lattice_is_free_spins():
    g = O.Geometry(O.CUBIC3D, 4)
    T = I.ladder(0.3, 2.0, 5)
    J = np.zeros(g.Nb)
    s0 = I.initial_spins(g.N, 10, 3, [0])[0]
    inst = O.Instance(g, J, T, s0, pm=True, T_icm=1.0, seed=3, inst=0)
    assert inst.nb_present == 0
    for _ in range(20):
        tr = inst.run(1, trace=True)
        assert np.all(inst.E == 0)
        assert np.all(tr["csize"] <= 1)
        assert np.all(tr["swap_acc"] == 1)
    # Metropolis alone: Delta E = 0 everywhere, each proposal accepted with
    # probability 1/2 (a deterministic flip would reverse every spin)
    sweep = O.Instance(g, J, T, s0, pm=True, T_icm=1.0, seed=3, inst=0, icm_every=0, swap_every=0)
    flips = 0
    for _ in range(20):
        before = sweep.s.copy()
        sweep.run(1)
        flips += np.count_nonzero(sweep.s != before)
    assert abs(flips / (20 * sweep.s.size) - 0.5) < 0.02
