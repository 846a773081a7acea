"""Parity of the CUDA library (through its C ABI) with the CPU oracle.

+-J couplings: bit-exact, sweep by sweep (spins, integer energies, n before
step 2a, step-2a decisions, seed sites, cluster sizes, PT decisions) and for
the accumulated observables.  Gaussian couplings: statistical agreement
(energy per spin, link overlap, overlap distribution within three standard
errors over instances, one Hotelling test per observable: statcheck),
energy conservation of every cluster move to 1e-5 of sum |J| in fp32 (the
kernel's own E_a + E_b and float64 energies of the spins), and the Eq. 1
identity.
"""
import numpy as np
import pytest
import statcheck

from oracle import exact
from oracle import oracle as O
from paper_1501_05630_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def icm():
    import torch
    from paper_1501_05630_gb300 import build, icmpt
    build.build()
    torch.cuda.set_device(0)
    ctx = icmpt.Context(0)
    yield icmpt, ctx
    ctx.close()


def _setup(kind, L, dis, n_inst, T, seed, ids=None):
    g = O.Geometry(kind, L)
    ids = list(range(n_inst)) if ids is None else list(ids)
    J = I.couplings(g.Nb, dis, seed, ids)
    s0 = I.initial_spins(g.N, 2 * len(T), seed, ids)
    return g, J, s0, ids


def _oracle(g, J, s0, T, T_icm, seed, inst, dis, **kw):
    return O.Instance(g, J.astype(np.float64), T, s0, pm=(dis == I.PM_J), T_icm=T_icm, seed=seed,
                      inst=inst, **kw)


TRACE_KEYS = ("n_pre", "flip2a", "seed_site", "csize", "esum_before", "esum_after")


def _compare_sweeps(icm, kind, L, nT, T_lo, T_hi, T_icm, n_inst, sweeps, seed, check_every=1, threads=None,
                    setup=None, **sched):
    icmpt, ctx = icm
    T = I.ladder(T_lo, T_hi, nT)
    g, J, s0, ids = _setup(kind, L, I.PM_J, n_inst, T, seed)
    b = icmpt.Batch(ctx, kind, L, I.PM_J, J, T, T_icm, seed, spins=s0)
    if threads is not None:
        b.set_threads(threads)
        assert b.info()["threads"] == threads
    if setup is not None:
        setup(b)
    b.set_schedule(trace=1, **sched)
    refs = [_oracle(g, J[a], s0[a], T, T_icm, seed, ids[a], I.PM_J, **sched) for a in range(n_inst)]
    b.clear_observables()
    moves = np.zeros(n_inst, dtype=np.int64)            # the oracle's cluster moves (seeded pairs)
    done = 0
    while done < sweeps:
        step = min(check_every, sweeps - done)
        b.run(step)
        trs = [r.run(step, trace=True) for r in refs]
        moves += [int((tr["seed_site"] >= 0).sum()) for tr in trs]
        done += step
        spins, E, tr = b.read_spins(), b.read_energies(), b.read_trace()
        cm = b.read_cluster_masks()
        for a, r in enumerate(refs):
            assert np.array_equal(spins[a], r.s), (a, done, "spins")
            assert np.array_equal(cm[a], trs[a]["cmask"]), (a, done, "cluster masks")
            assert np.array_equal(E[a], r.E), (a, done, E[a], r.E)
            for key in TRACE_KEYS:
                assert np.array_equal(tr[key][a], trs[a][key]), (a, done, key, tr[key][a], trs[a][key])
            if nT > 1:
                assert np.array_equal(tr["swap_acc"][a], trs[a]["swap_acc"]), (a, done, "swap")
    if check_every == 1:
        st = b.read_icm_stats()
        assert np.array_equal(st[:, 0].astype(np.int64), moves), (st[:, 0], moves)   # cluster moves
        assert np.all(st[:, 1] >= (st[:, 0] > 0))                                      # growth scans
    o = b.read_observables()
    for a, r in enumerate(refs):
        assert np.array_equal(o.accE[a], r.accE)
        assert np.array_equal(o.acc_n[a], r.acc_n)
        assert np.array_equal(o.acc_q2[a], r.acc_q2)
        assert np.array_equal(o.acc_pmin[a], r.acc_pmin)
        assert np.array_equal(o.acc_d[a], r.acc_d)
        assert np.array_equal(o.hist[a], r.hist)
        assert o.n_meas[a] == r.n_meas[0]
    assert np.all(b.read_sweeps() == sweeps)
    b.close()


# ----------------------------------------------------------------------------- +-J, bit-exact
def test_pmj_2d_L8_sweep_by_sweep(icm):
    """2D L=8 +-J, 16 temperatures in [0.2, 1.5], ICM for T <= 1: every sweep."""
    _compare_sweeps(icm, O.SQUARE2D, 8, 16, 0.2, 1.5, 1.0, 1, 200, 0x1501056300000001)


def test_pmj_2d_L8_full_run_4096_sweeps(icm):
    """The full 2D L=8 workload: 4096 sweeps, measured from sweep 2048."""
    icmpt, ctx = icm
    seed = 0x1501056300000001
    T = I.ladder(0.2, 1.5, 16)
    g, J, s0, ids = _setup(O.SQUARE2D, 8, I.PM_J, 1, T, seed)
    b = icmpt.Batch(ctx, O.SQUARE2D, 8, I.PM_J, J, T, 1.0, seed, spins=s0)
    b.set_schedule(t_meas=2048)
    b.run(4096)
    r = _oracle(g, J[0], s0[0], T, 1.0, seed, 0, I.PM_J, t_meas=2048)
    r.run(4096)
    assert np.array_equal(b.read_spins()[0], r.s)
    assert np.array_equal(b.read_energies()[0], r.E)
    o = b.read_observables()
    assert np.array_equal(o.hist[0], r.hist) and np.array_equal(o.acc_d[0], r.acc_d)
    assert np.array_equal(o.accE[0], r.accE) and o.n_meas[0] == 2048


@pytest.mark.parametrize("kind,L,nT,T_hi,T_icm,n_inst", [
    (O.CUBIC3D, 4, 24, 2.0, 1.0, 3),     # two spin words per site (48 replicas)
    (O.CUBIC3D, 6, 10, 2.0, 1.0, 2),     # 108 sites per colour: ragged against 128 threads
    (O.CHIMERA, 3, 30, 3.0, 1.5, 2),     # per-site degree 5/6, padded neighbour lists
    (O.SQUARE2D, 2, 4, 1.5, 1.0, 2),     # doubled bonds of the smallest torus
    (O.CUBIC3D, 2, 3, 2.0, 1.0, 2),
    (O.SQUARE2D, 6, 2, 1.5, 1.0, 1),     # fewest temperatures
    (O.CHIMERA, 1, 32, 3.0, 1.5, 1),     # most temperatures: 64 replicas, two full words
])
def test_pmj_sweep_by_sweep_shapes(icm, kind, L, nT, T_hi, T_icm, n_inst):
    _compare_sweeps(icm, kind, L, nT, 0.2, T_hi, T_icm, n_inst, 40, 0xC0FFEE + L)


@pytest.mark.parametrize("sched", [
    dict(enable_2a=0), dict(icm_every=0), dict(swap_every=0), dict(icm_every=3, swap_every=2),
    dict(enable_metropolis=0), dict(t_meas=10**9),
])
def test_pmj_schedule_variants(icm, sched):
    _compare_sweeps(icm, O.CUBIC3D, 4, 8, 0.3, 2.0, 1.2, 2, 25, 77, **sched)


def test_pmj_multi_sweep_launches(icm):
    """Several sweeps per launch give the same state as one sweep per launch."""
    _compare_sweeps(icm, O.CHIMERA, 4, 12, 0.2, 3.0, 1.5, 3, 90, 5, check_every=30)


def test_pmj_chimera_C8_full_batch_sampled(icm):
    """The chimera C_8 workload's shape: 10^4 instances, 30 temperatures, in one
    launch; sampled instances re-run alone by the oracle must match bit for bit."""
    icmpt, ctx = icm
    seed = 0x1501056300000003
    T = I.ladder(0.2, 3.0, 30)
    n = 10000
    g = O.Geometry(O.CHIMERA, 8)
    J = I.couplings(g.Nb, I.PM_J, seed, range(n))
    s0 = I.initial_spins(g.N, 60, seed, range(n))
    b = icmpt.Batch(ctx, O.CHIMERA, 8, I.PM_J, J, T, 1.5, seed, spins=s0)
    b.run(24)
    spins, E = b.read_spins(), b.read_energies()
    for a in (0, 1, 4999, 9998, 9999):
        r = _oracle(g, J[a], s0[a], T, 1.5, seed, a, I.PM_J)
        r.run(24)
        assert np.array_equal(spins[a], r.s), a
        assert np.array_equal(E[a], r.E), a
    # every instance: integer energies consistent with its spins
    for a in range(0, n, 997):
        e = -(J[a][None, :].astype(np.int64) * spins[a][:, g.bi] * spins[a][:, g.bj]).sum(1)
        assert np.array_equal(e, E[a].astype(np.int64))


def test_pmj_chimera_C8_planned_scale(icm):
    """The chimera C_8 workload at its planned parity scale: 10^4 instances,
    30 temperatures, in the launch shape of the bench; 64 instances sampled
    across the batch are bit-exact with the oracle (spins, integer energies,
    P(q) histograms, accumulated link disagreements) after 2^12 sweeps, and 4
    of them after the full 2^16 sweeps.  The oracle runs on the host cores
    while the GPU runs."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    icmpt, ctx = icm
    seed = 0x1501056300000003
    T = I.ladder(0.2, 3.0, 30)
    n = 10000
    g = O.Geometry(O.CHIMERA, 8)
    J = I.couplings(g.Nb, I.PM_J, seed, range(n))
    s0 = I.initial_spins(g.N, 60, seed, range(n))
    sample = np.linspace(0, n - 1, 64).astype(int)
    full = sample[[0, 21, 42, 63]]
    refs = {a: _oracle(g, J[a], s0[a], T, 1.5, seed, a, I.PM_J) for a in sample}
    b = icmpt.Batch(ctx, O.CHIMERA, 8, I.PM_J, J, T, 1.5, seed, spins=s0)
    with ThreadPoolExecutor(os.cpu_count() or 1) as ex:
        fut = {a: ex.submit(refs[a].run, 1 << 12) for a in sample}
        b.run(1 << 12)
        spins, E, o = b.read_spins(), b.read_energies(), b.read_observables()
        for a in sample:
            fut[a].result()
            r = refs[a]
            assert np.array_equal(spins[a], r.s), a
            assert np.array_equal(E[a], r.E), a
            assert np.array_equal(o.hist[a], r.hist) and np.array_equal(o.acc_d[a], r.acc_d), a
        del spins, o
        fut = {a: ex.submit(refs[a].run, (1 << 16) - (1 << 12)) for a in full}
        b.run((1 << 16) - (1 << 12))
        spins, E = b.read_spins(), b.read_energies()
        for a in full:
            fut[a].result()
            assert np.array_equal(spins[a], refs[a].s), a
            assert np.array_equal(E[a], refs[a].E), a
    assert np.all(b.read_sweeps() == 1 << 16)
    b.close()


def test_mix_invariance(icm):
    """An instance gives the same result alone and inside a larger batch."""
    icmpt, ctx = icm
    T = I.ladder(0.2, 2.0, 12)
    seed = 99
    g = O.Geometry(O.CUBIC3D, 4)
    for dis in (I.PM_J, I.GAUSS):
        J = I.couplings(g.Nb, dis, seed, range(40))
        s0 = I.initial_spins(g.N, 24, seed, range(40))
        big = icmpt.Batch(ctx, O.CUBIC3D, 4, dis, J, T, 1.0, seed, spins=s0)
        big.run(50)
        alone = icmpt.Batch(ctx, O.CUBIC3D, 4, dis, J[17:18].copy(), T, 1.0, seed, spins=s0[17:18].copy(),
                            instance_ids=[17])
        alone.run(50)
        assert np.array_equal(big.read_spins()[17], alone.read_spins()[0])
        assert np.array_equal(big.read_energies()[17], alone.read_energies()[0])


# ----------------------------------------------------------------------------- Gaussian, statistical
def _e64(J, spins, g):
    """H = -sum_b J_b s_i s_j of every replica, in float64 ([n][R])."""
    out = np.empty(spins.shape[:2])
    for a0 in range(0, spins.shape[0], 64):
        sl = slice(a0, a0 + 64)
        out[sl] = -np.einsum("nb,nrb->nr", J[sl].astype(np.float64),
                             (spins[sl][:, :, g.bi] * spins[sl][:, :, g.bj]).astype(np.float64))
    return out


def _check_icm_only_step(b, g, J, T, T_icm, tol=1e-5):
    """One step with only steps 2a/2b (no Metropolis sweep, no PT pass) on the
    batch's current state, checked on the host against the spins:
      * the spins change exactly on the traced clusters (copy b also by the
        step-2a reversal), and each cluster is the connected component of its
        traced seed among the q = -1 sites (the paper's cluster);
      * E_a + E_b of each pair, recomputed from the spins in float64, is the
        same before and after the move (the move is isoenergetic);
      * the device energies after the move equal the float64 energies of the
        spins, to tol * sum|J| (the benchmark spec's 1e-5 in fp32);
      * the traced E_a + E_b, both recomputed by the kernel from the flipped
        spins, equals the traced value before the move to tol * sum|J|.
    Returns the number of moves checked."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    nT = len(T)
    sched = b.schedule()
    b.set_schedule(enable_metropolis=0, swap_every=0, t_meas=1 << 40, trace=1)
    s0 = b.read_spins()
    b.run(1)
    s1, E1, tr, cm = b.read_spins(), b.read_energies(), b.read_trace(), b.read_cluster_masks()
    b.set_schedule(icm_every=sched.icm_every, swap_every=sched.swap_every, enable_2a=sched.enable_2a,
                   enable_metropolis=sched.enable_metropolis, t_meas=sched.t_meas, trace=sched.trace)
    scale = np.abs(J).astype(np.float64).sum(1)
    e0, e1 = _e64(J, s0, g), _e64(J, s1, g)
    icm_k = np.flatnonzero(T <= T_icm)
    assert np.all(tr["n_pre"][:, icm_k] >= 0) and np.all(tr["n_pre"][:, len(icm_k):] == -1)
    # conservation in float64 from the spins, every instance and ICM pair
    d = (e1[:, 0::2] + e1[:, 1::2]) - (e0[:, 0::2] + e0[:, 1::2])
    assert np.all(np.abs(d[:, icm_k]) <= 1e-9 * scale[:, None]), np.abs(d).max()
    # device energies = float64 energies of the spins
    assert np.all(np.abs(E1 - e1) <= tol * scale[:, None]), np.abs(E1 - e1).max()
    # traced E_a + E_b: both recomputed by the kernel from the flipped spins
    err = np.abs(tr["esum_after"] - tr["esum_before"])[:, icm_k]
    assert np.all(err <= tol * scale[:, None]), err.max()
    # the moved sets: spins change exactly on the cluster, which is the seed's component
    moves = 0
    for a in range(s0.shape[0]):
        for k in icm_k:
            sa, sb = s0[a, 2 * k], s0[a, 2 * k + 1].copy()
            if tr["flip2a"][a, k]:
                sb = -sb
            neg = sa * sb == -1
            comp = cm[a, k].astype(bool)
            assert np.array_equal(s1[a, 2 * k] != sa, comp) and np.array_equal(s1[a, 2 * k + 1] != sb, comp)
            assert comp.sum() == tr["csize"][a, k]
            if not neg.any():
                assert tr["seed_site"][a, k] == -1 and not comp.any()
                continue
            seed = tr["seed_site"][a, k]
            assert neg[seed] and comp[seed]
            if a % 50 == 0:                      # connectivity on a sample (scipy per pair)
                m = neg[g.bi] & neg[g.bj] & (J[a] != 0)      # bonds present (dilution)
                A = coo_matrix((np.ones(m.sum()), (g.bi[m], g.bj[m])), shape=(g.N, g.N))
                _, lab = connected_components(A, directed=False)
                assert np.array_equal(comp, neg & (lab == lab[seed]))
            moves += 1
    return moves


def test_gauss_energy_conservation_and_consistency(icm):
    """Every cluster move keeps E_a + E_b to 1e-5 sum|J| (fp32; the traced sum
    is of E_a and E_b each recomputed from the flipped spins); device energies
    agree with energies recomputed from the spins in float64."""
    icmpt, ctx = icm
    T = I.ladder(0.2, 2.0, 24)
    seed = 0x1501056300000002
    g, J, s0, ids = _setup(O.CUBIC3D, 8, I.GAUSS, 64, T, seed)
    b = icmpt.Batch(ctx, O.CUBIC3D, 8, I.GAUSS, J, T, 1.0, seed, spins=s0)
    b.set_schedule(trace=1)
    scale = np.abs(J).astype(np.float64).sum(1)
    moves = 0
    for rep in range(6):
        b.run(7)
        tr = b.read_trace()
        icm_k = tr["n_pre"] >= 0
        moves += int((tr["csize"] > 0).sum())
        err = np.abs(tr["esum_after"] - tr["esum_before"])[icm_k]
        assert np.all(err <= 1e-5 * np.repeat(scale[:, None], 24, 1)[icm_k])
        spins, E = b.read_spins(), b.read_energies()
        assert np.all(np.abs(E - _e64(J, spins, g)) <= 1e-5 * scale[:, None])
    assert moves > 100


def test_gauss_3d_L8_full_workload_invariants(icm):
    """The 3D L=8 Gaussian workload at its full size and launch shape (1000
    instances, 24 temperatures, ICM at 17, one launch of 256 sweeps, 128
    threads, every instance resident at once): every cluster move of the last sweep keeps
    E_a + E_b to 1e-5 sum|J|, every instance's device energies equal the
    energies recomputed from its spins in fp64 to 1e-5 sum|J|; then one step
    of cluster moves alone on that state, checked move by move against the
    spins (see _check_icm_only_step)."""
    icmpt, ctx = icm
    T = I.ladder(0.2, 2.0, 24)
    seed = 0x1501056300000002
    n = 1000
    g, J, s0, ids = _setup(O.CUBIC3D, 8, I.GAUSS, n, T, seed)
    b = icmpt.Batch(ctx, O.CUBIC3D, 8, I.GAUSS, J, T, 1.0, seed, spins=s0)
    info = b.info()
    import torch
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    assert (info["threads"], info["grid"]) == (128, 1000) and info["ctas_per_sm"] * n_sm >= n   # all resident
    b.set_schedule(trace=1)
    b.run(256)
    tr = b.read_trace()
    scale = np.abs(J).astype(np.float64).sum(1)
    icm_k = tr["n_pre"] >= 0
    assert icm_k.sum() == 17 * n
    err = np.abs(tr["esum_after"] - tr["esum_before"])[icm_k]
    assert np.all(err <= 1e-5 * np.repeat(scale[:, None], 24, 1)[icm_k])
    spins, E = b.read_spins(), b.read_energies()
    assert np.all(np.abs(E - _e64(J, spins, g)) <= 1e-5 * scale[:, None])
    assert np.array_equal(b.read_sweeps(), np.full(n, 256))
    assert _check_icm_only_step(b, g, J, T, 1.0) > 5000
    b.close()


def _paired(gpu_obs, refs, g):
    """Per-instance GPU-minus-oracle differences of e, q_l and the coarse
    symmetrised P(q), each [n][n_T(, bins)]."""
    m = gpu_obs.n_meas[:, None].astype(np.float64)
    ge = gpu_obs.accE / (2 * g.N * m)
    gq = 1 - 2 * gpu_obs.acc_d / (g.Nb * m)
    gp = statcheck.pq_bins(gpu_obs.hist)
    oe = np.array([r.observables()["e"] for r in refs])
    oq = np.array([r.observables()["q_l"] for r in refs])
    op = statcheck.pq_bins(np.array([r.hist for r in refs]))
    return dict(e=ge - oe, q_l=gq - oq, P_q=gp - op)


def _run_oracles(refs, sweeps):
    """The oracle instances, spread over the host cores (ctypes drops the GIL)."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(os.cpu_count() or 1) as ex:
        list(ex.map(lambda r: r.run(sweeps), refs))


@pytest.mark.parametrize("L", [4, 6])
def test_gauss_statistical_agreement_with_oracle(icm, L):
    """3D L=4 and L=6 Gaussian, 256 instances, 2^14 sweeps (measured over the
    second half), 24 temperatures in [0.2, 2.0], ICM for T <= 1: the energy per
    spin, the link overlap and the symmetrised overlap distribution P(q)
    (coarse bins of |q|) of every temperature agree between the GPU and the
    oracle, on the same instances, at three standard errors over instances
    (one Hotelling test per observable, see statcheck)."""
    icmpt, ctx = icm
    T = I.ladder(0.2, 2.0, 24)
    seed = 0x1501056300000020 + L
    n, sweeps = 256, 1 << 14
    g, J, s0, ids = _setup(O.CUBIC3D, L, I.GAUSS, n, T, seed)
    b = icmpt.Batch(ctx, O.CUBIC3D, L, I.GAUSS, J, T, 1.0, seed, spins=s0)
    b.set_schedule(t_meas=sweeps // 2)
    b.run(sweeps)
    o = b.read_observables()
    refs = [_oracle(g, J[a], s0[a], T, 1.0, seed, a, I.GAUSS, t_meas=sweeps // 2) for a in range(n)]
    _run_oracles(refs, sweeps)
    for key, d in _paired(o, refs, g).items():
        statcheck.agree(d, (L, key))
    b.close()


def test_gauss_matches_exact_enumeration(icm):
    """2D L=4 Gaussian (N = 16): 64 independent chains of one instance agree
    with exact enumeration (energy, link overlap, symmetrised P(q) at the
    lowest and highest temperature), three standard errors (statcheck)."""
    icmpt, ctx = icm
    T = I.ladder(0.4, 2.0, 6)
    seed = 5
    g = O.Geometry(O.SQUARE2D, 4)
    J1 = I.couplings(g.Nb, I.GAUSS, seed, [0])[0]
    n = 64
    J = np.repeat(J1[None], n, 0)
    s0 = I.initial_spins(g.N, 12, seed, range(1000, 1000 + n))
    b = icmpt.Batch(ctx, O.SQUARE2D, 4, I.GAUSS, J, T, 1.0, seed, spins=s0)
    b.set_schedule(t_meas=1000)
    b.run(5000)
    o = b.read_observables()
    m = o.n_meas[:, None].astype(np.float64)
    st = exact.all_states(g.N)
    E = exact.energies(g.bi, g.bj, J1.astype(np.float64), st)
    ex = [exact.thermal(g.bi, g.bj, J1.astype(np.float64), g.N, t, st, E) for t in T]
    for name, vals in (("e", o.accE / (2 * g.N * m)), ("q_l", 1 - 2 * o.acc_d / (g.Nb * m))):
        want = np.array([x[name] for x in ex])
        statcheck.agree(vals - want[None, :], name)
    P = o.hist / m[:, :, None]
    for k in (0, len(T) - 1):
        statcheck.agree_distribution((P[:, k] + P[:, k, ::-1]) / 2, ex[k]["P_n"], o.n_meas, (k, "P(q)"))


def test_gauss_eq1_identity(icm):
    """Eq. 1: disorder-averaged e = -(N_b/N)(1 - [q_l])/T at equilibrium
    (3D L=4, 200 instances, well-thermalised moderate temperatures), three
    standard errors over instances (statcheck)."""
    icmpt, ctx = icm
    T = I.ladder(0.6, 2.0, 8)
    seed = 31
    n = 200
    g, J, s0, ids = _setup(O.CUBIC3D, 4, I.GAUSS, n, T, seed)
    b = icmpt.Batch(ctx, O.CUBIC3D, 4, I.GAUSS, J, T, 1.0, seed, spins=s0)
    b.set_schedule(t_meas=2000)
    b.run(10000)
    o = b.read_observables()
    m = o.n_meas[:, None].astype(np.float64)
    e = o.accE / (2 * g.N * m)
    ql = 1 - 2 * o.acc_d / (g.Nb * m)
    statcheck.agree(e + (g.Nb / g.N) * (1 - ql) / T[None, :], "Eq. 1")


# ----------------------------------------------------------------------------- limits and errors
def test_largest_shared_memory_instance(icm):
    """3D L=12 (1728 sites), 48 replicas: one CTA's shared memory holds the whole instance."""
    _compare_sweeps(icm, O.CUBIC3D, 12, 24, 0.2, 2.0, 1.0, 2, 6, 12, check_every=3, threads=128)


# ----------------------------------------------------------------------------- global-resident (wide) layout
@pytest.mark.parametrize("kind,L,nT,T_hi,T_icm,n_inst,threads", [
    (O.CUBIC3D, 4, 24, 2.0, 1.0, 3, 256),      # two spin words, more threads than sites per colour
    (O.CUBIC3D, 6, 10, 2.0, 1.0, 2, 160),      # ragged against the CTA width
    (O.CHIMERA, 3, 30, 3.0, 1.5, 2, 512),      # per-site degrees, padded neighbour lists
    (O.SQUARE2D, 2, 4, 1.5, 1.0, 2, 1024),     # doubled bonds; widest CTA on the smallest torus
    (O.CHIMERA, 1, 32, 3.0, 1.5, 1, 192),      # 64 replicas
])
def test_wide_layout_pmj_sweep_by_sweep(icm, kind, L, nT, T_hi, T_icm, n_inst, threads):
    """Widths above 128 threads keep the instance in global memory: the same
    chain as the oracle, bit for bit, sweep by sweep."""
    _compare_sweeps(icm, kind, L, nT, 0.2, T_hi, T_icm, n_inst, 30, 0xBEEF + L, threads=threads)


def test_wide_layout_2d_L128_64_replicas(icm):
    """2D L=128 (16384 sites) +-J with 32 temperatures (64 replicas), the
    largest serving size: too large for shared memory, so the default layout
    is the global-resident one; bit-exact with the oracle."""
    icmpt, ctx = icm
    _compare_sweeps(icm, O.SQUARE2D, 128, 32, 0.2, 1.5, 1.0, 1, 6, 0x1501, check_every=3)


def test_wide_layout_default_for_large_instances(icm):
    """The shared-memory layout while several instances fit one SM, else the wide one."""
    icmpt, ctx = icm
    for kind, L, dis, nT, wide in ((O.SQUARE2D, 128, I.PM_J, 32, True), (O.SQUARE2D, 128, I.PM_J, 8, True),
                                   (O.SQUARE2D, 64, I.PM_J, 32, True), (O.CUBIC3D, 12, I.GAUSS, 24, True),
                                   (O.CUBIC3D, 22, I.PM_J, 16, True), (O.CUBIC3D, 8, I.GAUSS, 24, False),
                                   (O.CHIMERA, 8, I.PM_J, 30, False), (O.SQUARE2D, 8, I.PM_J, 16, False)):
        T = I.ladder(0.2, 2.0, nT)
        g = O.Geometry(kind, L)
        b = icmpt.Batch(ctx, kind, L, dis, I.couplings(g.Nb, dis, 1, [0]), T, 1.0, 1,
                        spins=I.initial_spins(g.N, 2 * nT, 1, [0]))
        info = b.info()
        assert (info["threads"] > 128) == wide, (kind, L, info)
        b.close()


@pytest.mark.parametrize("threads", [None, 1024])
def test_gauss_3d_L16_conservation_and_consistency(icm, threads):
    """3D L=16 Gaussian (4096 sites, 64 replicas), default and wide layout:
    every cluster move keeps E_a + E_b to 1e-5 sum|J|; device energies equal
    energies from the spins."""
    icmpt, ctx = icm
    T = I.ladder(0.2, 2.0, 32)
    seed = 0x1501056300000016
    n = 6
    g, J, s0, ids = _setup(O.CUBIC3D, 16, I.GAUSS, n, T, seed)
    b = icmpt.Batch(ctx, O.CUBIC3D, 16, I.GAUSS, J, T, 1.0, seed, spins=s0)
    if threads:
        b.set_threads(threads)
    b.set_schedule(trace=1)
    scale = np.abs(J).astype(np.float64).sum(1)
    moves = 0
    for rep in range(4):
        b.run(5)
        tr = b.read_trace()
        icm_k = tr["n_pre"] >= 0
        moves += int((tr["csize"] > 0).sum())
        err = np.abs(tr["esum_after"] - tr["esum_before"])[icm_k]
        assert np.all(err <= 1e-5 * np.repeat(scale[:, None], 32, 1)[icm_k])
        spins, E = b.read_spins(), b.read_energies()
        for a in range(n):
            e_ref = -np.einsum("b,rb->r", J[a].astype(np.float64),
                               (spins[a][:, g.bi] * spins[a][:, g.bj]).astype(np.float64))
            assert np.allclose(E[a], e_ref, rtol=0, atol=2e-5 * scale[a])
    assert moves > 50


def test_wide_layout_gauss_statistical_agreement_with_oracle(icm):
    """3D L=4 Gaussian forced into the wide layout: per-temperature energy,
    link overlap and P(q) agree with the oracle's on the same instances at
    three standard errors (statcheck)."""
    icmpt, ctx = icm
    T = I.ladder(0.3, 2.0, 8)
    seed = 4343
    n = 64
    g, J, s0, ids = _setup(O.CUBIC3D, 4, I.GAUSS, n, T, seed)
    sweeps, t_meas = 3000, 1000
    b = icmpt.Batch(ctx, O.CUBIC3D, 4, I.GAUSS, J, T, 1.0, seed, spins=s0)
    b.set_threads(256)
    b.set_schedule(t_meas=t_meas)
    b.run(sweeps)
    o = b.read_observables()
    refs = [_oracle(g, J[a], s0[a], T, 1.0, seed, a, I.GAUSS, t_meas=t_meas) for a in range(n)]
    _run_oracles(refs, sweeps)
    for key, d in _paired(o, refs, g).items():
        statcheck.agree(d, key)


def test_wide_layout_autotune_keeps_state(icm):
    icmpt, ctx = icm
    T = I.ladder(0.2, 1.5, 16)
    g = O.Geometry(O.SQUARE2D, 128)
    b = icmpt.Batch(ctx, O.SQUARE2D, 128, I.PM_J, I.couplings(g.Nb, I.PM_J, 2, range(3)), T, 1.0, 2,
                    spins=I.initial_spins(g.N, 32, 2, range(3)))
    b.run(2)
    before = (b.read_spins(), b.read_energies(), b.read_sweeps())
    th, ms = b.autotune(sweeps=2)
    assert th in (256, 512, 1024) and ms > 0
    for x, y in zip(before, (b.read_spins(), b.read_energies(), b.read_sweeps())):
        assert np.array_equal(x, y)
    b.close()


def test_invalid_arguments(icm):
    icmpt, ctx = icm
    T = I.ladder(0.2, 2.0, 4)
    J = I.couplings(48, I.PM_J, 0, [0])
    with pytest.raises(icmpt.IcmError):
        icmpt.Batch(ctx, O.SQUARE2D, 5, I.PM_J, I.couplings(50, I.PM_J, 0, [0]), T, 1.0, 0)   # odd L
    with pytest.raises(icmpt.IcmError):
        icmpt.Batch(ctx, O.CUBIC3D, 4, I.PM_J, I.couplings(192, I.PM_J, 0, [0]), T[::-1].copy(), 1.0, 0)
    with pytest.raises(icmpt.IcmError):
        icmpt.Batch(ctx, O.CUBIC3D, 4, I.PM_J, I.couplings(192, I.PM_J, 0, [0]), I.ladder(0.2, 2, 33), 1.0, 0)
    with pytest.raises(icmpt.IcmError):
        icmpt.Batch(ctx, O.SQUARE2D, 256, I.PM_J, I.couplings(2 * 256 * 256, I.PM_J, 0, [0]), T, 1.0, 0)
    del J


def test_read_overlaps_equals_oracle_averages(icm):
    """icm_read_overlaps normalises the accumulators into <q>, <q^2>, <q_l> and
    the counts of n; for +-J they equal the oracle's averages (same chain)."""
    icmpt, ctx = icm
    T = I.ladder(0.3, 2.0, 8)
    g, J, s0, ids = _setup(O.CUBIC3D, 4, I.PM_J, 2, T, 0x0E)
    b = icmpt.Batch(ctx, O.CUBIC3D, 4, I.PM_J, J, T, 1.2, 0x0E, spins=s0)
    b.set_schedule(t_meas=30)
    b.run(90)
    q, q2, ql, h = b.read_overlaps()
    for a in range(2):
        r = _oracle(g, J[a], s0[a], T, 1.2, 0x0E, a, I.PM_J, t_meas=30)
        r.run(90)
        ob = r.observables()
        assert np.allclose(q[a], 1.0 - 2.0 * ob["n_frac"], rtol=0, atol=1e-12)
        assert np.allclose(q2[a], ob["q2"], rtol=0, atol=1e-12)
        assert np.allclose(ql[a], ob["q_l"], rtol=0, atol=1e-12)
        assert np.array_equal(h[a], r.hist)
    b.clear_observables()
    q, q2, ql, _ = b.read_overlaps(hist=False)
    assert np.all(np.isnan(q)) and np.all(np.isnan(ql))      # nothing measured yet
    b.close()
