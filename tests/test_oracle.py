"""Pins of the CPU oracle against facts that do not come from the oracle itself.

* Philox4x32-10: the published known-answer vectors (Salmon et al., SC'11)
  and cuRAND's independent host implementation.
* Geometry: bond counts, degrees and the two-colouring of the lattices.
* Exact enumeration: Kaufman's closed-form partition function of the 2D
  ferromagnet on a torus, and the Gaussian-disorder identity of Eq. 1.
* Monte Carlo chain (Metropolis + ICM + PT): equilibrium values from exact
  enumeration, a chi-square test of sampled states against Boltzmann weights,
  the invariance of E_a + E_b under every cluster move (the move is
  "isoenergetic"), the cluster = connected component of the negative-overlap
  sites, and the limits p -> 1/2 (T -> infinity) and p -> 0 (T -> 0, Gaussian).
"""
import ctypes
import math

import numpy as np
import pytest
import statcheck

from oracle import exact
from oracle import oracle as O
from paper_1501_05630_gb300 import inputs as I


# ----------------------------------------------------------------------------- Philox
def test_philox_known_answers():
    kat = [
        ([0, 0, 0, 0], [0, 0], [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
        ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2, [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
        ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
         [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]),
    ]
    for ctr, key, want in kat:
        assert list(O.philox(ctr, key)) == want


def _curand_host():
    for name in ("libcurand.so", "libcurand.so.10", "/usr/local/cuda/lib64/libcurand.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    return None


def test_philox_matches_curand_host_generator():
    lib = _curand_host()
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) != 0:  # PHILOX4_32_10
        pytest.skip("cuRAND host generator unavailable")
    try:
        for seed in (0, 0x1501056300000002, 0xDEADBEEF12345678):
            assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
            assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(0)) == 0
            n = 64
            buf = (ctypes.c_uint32 * (4 * n))()
            assert lib.curandGenerate(gen, buf, ctypes.c_size_t(4 * n)) == 0
            got = np.frombuffer(buf, dtype=np.uint32).reshape(n, 4)
            key = [seed & 0xFFFFFFFF, seed >> 32]
            for c in range(n):
                assert list(O.philox([0, 0, c, 0], key)) == list(got[c])   # block c = ctr {0,0,c,0}
    finally:
        lib.curandDestroyGenerator(gen)


# ----------------------------------------------------------------------------- geometry
@pytest.mark.parametrize("kind,L,N,Nb,deg", [
    (O.SQUARE2D, 4, 16, 32, {4}), (O.SQUARE2D, 8, 64, 128, {4}),
    (O.CUBIC3D, 4, 64, 192, {6}), (O.CUBIC3D, 8, 512, 1536, {6}),
    (O.CHIMERA, 1, 8, 16, {4}), (O.CHIMERA, 8, 512, 1472, {5, 6}),
    (O.CHIMERA, 12, 1152, 3360, {5, 6}),
])
def test_geometry_invariants(kind, L, N, Nb, deg):
    g = O.Geometry(kind, L)
    assert (g.N, g.Nb) == (N, Nb)
    assert np.all(g.bi != g.bj)
    assert np.all(g.color[g.bi] != g.color[g.bj])            # proper two-colouring
    assert np.sum(g.color == 0) == N // 2
    d = np.bincount(np.concatenate([g.bi, g.bj]), minlength=N)
    assert set(np.unique(d)) == deg
    pairs = set(zip(np.minimum(g.bi, g.bj), np.maximum(g.bi, g.bj)))
    assert len(pairs) == Nb                                  # no doubled bond for L >= 3
    if kind == O.CHIMERA and L > 1:
        # 4 in-cell bonds + 2 inter-cell bonds, one fewer on the boundary rows/columns
        assert np.sum(d == 5) == 16 * L
        assert np.sum(d == 6) == N - 16 * L


def test_geometry_small_torus_keeps_doubled_bonds():
    g = O.Geometry(O.CUBIC3D, 2)
    assert (g.N, g.Nb) == (8, 24)
    d = np.bincount(np.concatenate([g.bi, g.bj]), minlength=8)
    assert np.all(d == 6)


# ----------------------------------------------------------------------------- exact enumeration
def _kaufman_logZ(K: float, m: int, n: int) -> float:
    """ln Z of the m x n periodic ferromagnet, J = 1, K = J/T (Kaufman 1949).

    Z = 1/2 (2 sinh 2K)^{mn/2} (Z1 + Z2 + Z3 + Z4),
    Z1 = prod_r 2 cosh(m g_{2r+1}/2), Z2 = prod_r 2 sinh(m g_{2r+1}/2),
    Z3 = prod_r 2 cosh(m g_{2r}/2),   Z4 = prod_r 2 sinh(m g_{2r}/2),  r = 0..n-1,
    cosh g_l = cosh 2K coth 2K - cos(l pi / n), and g_0 = 2K + ln tanh K.
    """
    def gamma(l):
        if l == 0:
            return 2 * K + math.log(math.tanh(K))
        return math.acosh(math.cosh(2 * K) / math.tanh(2 * K) - math.cos(l * math.pi / n))
    Z1 = Z2 = Z3 = Z4 = 1.0
    for r in range(n):
        g1, g0 = gamma(2 * r + 1), gamma(2 * r)
        Z1 *= 2 * math.cosh(m * g1 / 2)
        Z2 *= 2 * math.sinh(m * g1 / 2)
        Z3 *= 2 * math.cosh(m * g0 / 2)
        Z4 *= 2 * math.sinh(m * g0 / 2)
    return math.log(0.5) + (m * n / 2) * math.log(2 * math.sinh(2 * K)) + math.log(Z1 + Z2 + Z3 + Z4)


@pytest.mark.parametrize("T", [1.0, 2.0, 2.269, 3.5])
def test_exact_enumeration_matches_kaufman(T):
    g = O.Geometry(O.SQUARE2D, 4)
    st = exact.all_states(g.N)
    E = exact.energies(g.bi, g.bj, np.ones(g.Nb), st)
    logZ = np.log(np.sum(np.exp(-E / T)))
    assert abs(logZ - _kaufman_logZ(1.0 / T, 4, 4)) < 1e-9
    # mean energy by a central difference of the closed form in K
    K, h = 1.0 / T, 1e-5
    e_kauf = -(_kaufman_logZ(K + h, 4, 4) - _kaufman_logZ(K - h, 4, 4)) / (2 * h) / g.N
    assert abs(exact.thermal(g.bi, g.bj, np.ones(g.Nb), g.N, T, st, E)["e"] - e_kauf) < 1e-6


def test_exact_overlap_distribution_is_normalised_and_symmetric():
    g = O.Geometry(O.SQUARE2D, 4)
    J = I.couplings(g.Nb, I.GAUSS, 7, [0])[0].astype(np.float64)
    th = exact.thermal(g.bi, g.bj, J, g.N, 0.7)
    assert abs(th["P_n"].sum() - 1.0) < 1e-12
    assert np.allclose(th["P_n"], th["P_n"][::-1], atol=1e-12)   # spin-reversal symmetry


@pytest.mark.parametrize("kind,L,T", [(O.CHIMERA, 1, 0.7), (O.CUBIC3D, 2, 1.3)])
def test_exact_overlap_distribution_equals_direct_double_sum(kind, L, T):
    """P(n) of two independent replicas, written out as the double sum over
    state pairs sum_s sum_t p(s) p(t) [popcount(s xor t) = n] (N = 8), equals
    the transform-based P(n) of exact.thermal, and so do <q^2>, <n>/N and p
    from it."""
    g = O.Geometry(kind, L)
    assert g.N == 8
    J = I.couplings(g.Nb, I.GAUSS, 17, [0])[0].astype(np.float64)
    st = exact.all_states(g.N)
    E = -(st[:, g.bi].astype(np.float64) * st[:, g.bj]) @ J
    p = np.exp(-(E - E.min()) / T)
    p /= p.sum()
    P = np.zeros(g.N + 1)
    for s in range(1 << g.N):
        for t in range(1 << g.N):
            P[bin(s ^ t).count("1")] += p[s] * p[t]
    th = exact.thermal(g.bi, g.bj, J, g.N, T)
    assert np.allclose(th["P_n"], P, rtol=0, atol=1e-14)
    n = np.arange(g.N + 1)
    assert th["q2"] == pytest.approx(np.sum(P * (1 - 2 * n / g.N) ** 2), abs=1e-14)
    assert th["n_frac"] == pytest.approx(np.sum(P * n) / g.N, abs=1e-14)
    assert th["p"] == pytest.approx(np.sum(P * np.minimum(n, g.N - n)) / g.N, abs=1e-14)


def test_eq1_identity_for_gaussian_disorder_exact():
    """[<H>]/N = -(N_b/N)(1 - [q_l])/T, averaged over Gaussian disorder (Eq. 1)."""
    g = O.Geometry(O.SQUARE2D, 4)
    st = exact.all_states(g.N)
    T = 1.1
    d = []
    for inst in range(300):
        J = I.couplings(g.Nb, I.GAUSS, 11, [inst])[0].astype(np.float64)
        th = exact.thermal(g.bi, g.bj, J, g.N, T, st)
        d.append(th["e"] + (g.Nb / g.N) * (1.0 - th["q_l"]) / T)
    d = np.array(d)
    statcheck.agree(d, "Eq. 1")
    # the identity is a disorder average: single instances do deviate
    assert d.std() > 1e-3


# ----------------------------------------------------------------------------- Monte Carlo chain
def _chains(kind, L, disorder, T, T_icm, n_chains, sweeps, seed=5, t_meas=None, **kw):
    g = O.Geometry(kind, L)
    J = I.couplings(g.Nb, disorder, seed, [0])[0].astype(np.float64)
    R = 2 * len(T)
    obs = []
    for c in range(n_chains):
        s0 = I.initial_spins(g.N, R, seed, [1000 + c])[0]
        inst = O.Instance(g, J, T, s0, pm=(disorder == I.PM_J), T_icm=T_icm, seed=seed,
                          inst=c, t_meas=sweeps // 4 if t_meas is None else t_meas, **kw)
        inst.run(sweeps)
        obs.append(inst.observables())
    return g, J, obs


def _agree(samples, target):
    """Samples agree with target at three standard errors (one Hotelling test
    over all components, statcheck); returns (ok, sample mean, test figures)."""
    d = np.asarray(samples, dtype=np.float64) - np.asarray(target, dtype=np.float64)
    r = statcheck.hotelling(d)
    return r["p"] >= statcheck.P_3SIGMA, d.mean(0) + target, r


@pytest.mark.parametrize("kind,L,disorder", [
    (O.SQUARE2D, 4, I.PM_J), (O.SQUARE2D, 4, I.GAUSS),
    (O.CUBIC3D, 2, I.GAUSS), (O.CHIMERA, 1, I.PM_J),
])
def test_oracle_chain_matches_exact_enumeration(kind, L, disorder):
    T = I.ladder(0.4, 2.0, 6)
    g, J, obs = _chains(kind, L, disorder, T, T_icm=1.0, n_chains=48, sweeps=3000)
    st = exact.all_states(g.N)
    E = exact.energies(g.bi, g.bj, J, st)
    ex = [exact.thermal(g.bi, g.bj, J, g.N, t, st, E) for t in T]
    for name in ("e", "q_l", "q2"):
        ok, mean, se = _agree([o[name] for o in obs], np.array([x[name] for x in ex]))
        assert ok, (name, mean, se, [x[name] for x in ex])
    # Full overlap distribution at the lowest and highest temperature.  Step 2a
    # flips copy 1 whenever n > N/2, so the chain is stationary only for
    # observables invariant under a global flip of copy 1: compare P(q)
    # symmetrised, (P(n) + P(N - n))/2, with the (symmetric) exact P(n).
    for k in (0, len(T) - 1):
        sym = [(o["P_n"][k] + o["P_n"][k][::-1]) / 2 for o in obs]
        statcheck.agree_distribution(sym, ex[k]["P_n"], [o["n_meas"] for o in obs], (k, "P(n)"))


def test_oracle_samples_boltzmann_distribution_chi2():
    """Independent chains' final states at T_0 follow exp(-E/T_0)/Z (N = 8)."""
    from scipy import stats
    g = O.Geometry(O.CHIMERA, 1)
    J = I.couplings(g.Nb, I.GAUSS, 3, [0])[0].astype(np.float64)
    T = I.ladder(0.8, 2.5, 4)
    st = exact.all_states(g.N)
    E = exact.energies(g.bi, g.bj, J, st)
    p = np.exp(-(E - E.min()) / T[0]); p /= p.sum()
    counts = np.zeros(1 << g.N)
    n = 3000
    for c in range(n):
        s0 = I.initial_spins(g.N, 2 * len(T), 3, [c])[0]
        inst = O.Instance(g, J, T, s0, pm=False, T_icm=1.0, seed=99, inst=c)
        inst.run(60)
        bits = (inst.s[0] < 0).astype(np.int64)
        counts[int(np.sum(bits << np.arange(g.N)))] += 1
    exp_ = p * n
    # pool states with small expectation into one bin
    big = exp_ >= 5
    obs_b = np.append(counts[big], counts[~big].sum())
    exp_b = np.append(exp_[big], exp_[~big].sum())
    chi2 = np.sum((obs_b - exp_b) ** 2 / np.maximum(exp_b, 1e-12))
    dof = len(obs_b) - 1
    assert stats.chi2.sf(chi2, dof) > 1e-4, (chi2, dof)


@pytest.mark.parametrize("disorder", [I.PM_J, I.GAUSS])
def test_cluster_move_is_isoenergetic_and_flips_a_component(disorder):
    """Steps 2a/2b alone: E_a + E_b unchanged; the flipped set is the connected
    component of the seed among the q = -1 sites (checked with scipy)."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    g = O.Geometry(O.CUBIC3D, 6)
    J = I.couplings(g.Nb, disorder, 21, [0])[0].astype(np.float64)
    T = I.ladder(0.3, 1.5, 8)
    R = 2 * len(T)
    s0 = I.initial_spins(g.N, R, 21, [0])[0]
    inst = O.Instance(g, J, T, s0, pm=(disorder == I.PM_J), T_icm=1.0, seed=21, inst=0,
                      swap_every=0, enable_metropolis=False)
    moves = 0
    for step in range(40):
        before = inst.s.copy()
        tr = inst.run(1, trace=True)
        for k in range(len(T)):
            sa, sb = before[2 * k].copy(), before[2 * k + 1].copy()
            if T[k] > 1.0:
                assert tr["n_pre"][k] == -1
                assert np.array_equal(inst.s[2 * k], sa) and np.array_equal(inst.s[2 * k + 1], sb)
                continue
            Eb = inst.energy(sb)
            if tr["flip2a"][k]:
                sb = -sb
                assert inst.energy(sb) == pytest.approx(Eb, abs=1e-9)   # spin reversal
            neg = (sa * sb == -1)
            assert neg.sum() <= g.N // 2
            if disorder == I.PM_J:
                assert tr["esum_after"][k] == tr["esum_before"][k]
            else:
                assert abs(tr["esum_after"][k] - tr["esum_before"][k]) <= 1e-12 * np.abs(J).sum()
            if not neg.any():
                assert tr["seed_site"][k] == -1
                continue
            moves += 1
            seed = tr["seed_site"][k]
            assert neg[seed]
            m = neg[g.bi] & neg[g.bj]
            A = coo_matrix((np.ones(m.sum()), (g.bi[m], g.bj[m])), shape=(g.N, g.N))
            _, lab = connected_components(A, directed=False)
            comp = neg & (lab == lab[seed])
            assert comp.sum() == tr["csize"][k]
            want_a = np.where(comp, -sa, sa)
            want_b = np.where(comp, -sb, sb)
            assert np.array_equal(inst.s[2 * k], want_a)
            assert np.array_equal(inst.s[2 * k + 1], want_b)
    assert moves > 50


def test_seed_is_uniform_over_negative_sites():
    """rank = floor(x n / 2^32) picks each q = -1 site equally often."""
    g = O.Geometry(O.SQUARE2D, 6)
    J = I.couplings(g.Nb, I.PM_J, 4, [0])[0].astype(np.float64)
    T = np.array([0.5])
    s0 = I.initial_spins(g.N, 2, 4, [0])[0]
    inst = O.Instance(g, J, T, s0, pm=True, T_icm=1.0, seed=4, inst=0,
                      swap_every=0, enable_metropolis=False, enable_2a=False)
    # freeze a fixed negative set: undo each move by re-loading the start state
    neg = np.flatnonzero(s0[0] * s0[1] == -1)
    hits = np.zeros(g.N)
    for step in range(4000):
        inst.s[:] = s0
        tr = inst.run(1, trace=True)
        hits[tr["seed_site"][0]] += 1
    from scipy import stats
    f = hits[neg]
    assert hits.sum() == f.sum()
    chi2 = np.sum((f - f.mean()) ** 2 / f.mean())
    assert stats.chi2.sf(chi2, len(f) - 1) > 1e-4


def test_high_temperature_limit_p_half():
    """T -> infinity: the fraction of q = -1 sites tends to 1/2 (Fig. 1)."""
    g, J, obs = _chains(O.CUBIC3D, 4, I.GAUSS, np.array([1e6, 2e6]), T_icm=0.0,
                        n_chains=16, sweeps=400, t_meas=10)
    ok, mean, se = _agree([o["n_frac"] for o in obs], np.array([0.5, 0.5]))
    assert ok, (mean, se)


def test_low_temperature_gaussian_reaches_ground_state():
    """Gaussian disorder, T -> 0: both replicas in the unique ground state, p -> 0."""
    g = O.Geometry(O.CHIMERA, 1)
    J = I.couplings(g.Nb, I.GAUSS, 8, [0])[0].astype(np.float64)
    st = exact.all_states(g.N)
    E_gs = exact.energies(g.bi, g.bj, J, st).min()
    T = I.ladder(0.02, 1.5, 8)
    s0 = I.initial_spins(g.N, 16, 8, [0])[0]
    inst = O.Instance(g, J, T, s0, pm=False, T_icm=1.0, seed=8, inst=0, t_meas=1500)
    inst.run(2000)
    ob = inst.observables()
    assert inst.E[0] == pytest.approx(E_gs, abs=1e-9)
    assert inst.E[1] == pytest.approx(E_gs, abs=1e-9)
    assert ob["n_frac"][0] < 1e-3 or ob["n_frac"][0] > 1 - 1e-3
    assert ob["p"][0] < 1e-3


def test_bimodal_keeps_clusters_at_low_temperature():
    """+-J: degenerate ground states leave q = -1 sites at the lowest T."""
    g, J, obs = _chains(O.SQUARE2D, 6, I.PM_J, I.ladder(0.1, 1.5, 8), T_icm=1.0,
                        n_chains=6, sweeps=1500)
    assert np.mean([o["p"][0] for o in obs]) > 0.01


# ----------------------------------------------------------------------------- site percolation
def _thresholds():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "percolation_thresholds.txt")
    out = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            f = line.split()
            out[f[0]] = (float(f[1]), float(f[2]))
    return out


@pytest.mark.parametrize("kind,L", [(O.SQUARE2D, 6), (O.CUBIC3D, 4), (O.CHIMERA, 3), (O.CHIMERA, 1)])
def test_largest_cluster_matches_scipy(kind, L):
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    g = O.Geometry(kind, L)
    masks = np.concatenate([I.site_masks(g.N, p, 17, 40) for p in (0.0, 0.2, 0.4, 0.6, 1.0)])
    got = O.largest_clusters(g, masks)
    for m, s in zip(masks, got):
        occ = m.astype(bool)
        keep = occ[g.bi] & occ[g.bj]
        A = coo_matrix((np.ones(keep.sum()), (g.bi[keep], g.bj[keep])), shape=(g.N, g.N))
        _, lab = connected_components(A, directed=False)
        want = np.bincount(lab[occ]).max() if occ.any() else 0
        assert s == want


@pytest.mark.parametrize("name,kind,sizes,half_window,tol", [
    ("square2d", O.SQUARE2D, (8, 16), 0.05, 0.02),
    ("cubic3d", O.CUBIC3D, (4, 8), 0.05, 0.03),
    ("chimera", O.CHIMERA, (8, 16), 0.03, 0.012),
])
def test_binder_crossing_near_printed_threshold(name, kind, sizes, half_window, tol):
    """The Binder ratios g = (3 - <s^4>/<s^2>^2)/2 of the largest-cluster
    fraction of two sizes cross near the threshold the paper prints (Fig. 1
    caption, Supplemental Material).  The sizes are small, so a finite-size
    shift of the crossing (toward lower p here) is part of the tolerance."""
    pc, _ = _thresholds()[name]
    ps = np.linspace(pc - half_window, pc + half_window, 9)
    curves = []
    for L in sizes:
        g = O.Geometry(kind, L)
        curves.append([O.binder_ratio(O.largest_clusters(g, I.site_masks(g.N, p, 100 + L, 6000)) / g.N)
                       for p in ps])
    d = np.array(curves[1]) - np.array(curves[0])
    i = np.flatnonzero(np.diff(np.sign(d)) != 0)
    assert len(i) >= 1
    cross = [ps[j] - d[j] * (ps[j + 1] - ps[j]) / (d[j + 1] - d[j]) for j in i]
    best = min(cross, key=lambda c: abs(c - pc))
    assert abs(best - pc) < tol, (cross, pc)


def test_trace_cluster_masks_are_the_moved_components():
    """The oracle's traced cluster of each move: csize sites, including the
    seed, connected through bonds present, all with q = -1 in the final state
    (both copies flip, so the overlap of a moved site stays -1); without PT
    the configurations stay at their temperatures, so this is checkable."""
    scipy_sparse = pytest.importorskip("scipy.sparse")
    from scipy.sparse.csgraph import connected_components
    g = O.Geometry(O.SQUARE2D, 8)
    T = I.ladder(0.3, 1.5, 8)
    J = I.couplings(g.Nb, I.PM_J, 5, [0])[0].astype(np.float64)
    s0 = I.initial_spins(g.N, 16, 5, [0])[0]
    r = O.Instance(g, J, T, s0, pm=True, T_icm=1.2, seed=5, inst=0, swap_every=0)
    moved = 0
    for _ in range(20):
        tr = r.run(1, trace=True)
        for k in range(len(T)):
            m = tr["cmask"][k].astype(bool)
            assert m.sum() == tr["csize"][k]
            if tr["csize"][k] == 0:
                continue
            moved += 1
            assert m[tr["seed_site"][k]]
            q = r.s[2 * k] * r.s[2 * k + 1]
            assert np.all(q[m] == -1)
            sel = np.flatnonzero(m)
            keep = m[g.bi] & m[g.bj]
            A = scipy_sparse.coo_matrix((np.ones(keep.sum()), (g.bi[keep], g.bj[keep])), shape=(g.N, g.N))
            _, lab = connected_components(A, directed=False)
            assert len(set(lab[sel])) == 1
    assert moved > 20
