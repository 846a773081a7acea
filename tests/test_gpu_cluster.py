"""The thread-block-cluster layout: one instance per cluster of K CTAs that
share its sites through distributed shared memory.

+-J: the same chain as the oracle, bit for bit, sweep by sweep (spins,
integer energies, step-2a decisions, seeds, cluster sizes, PT decisions,
observables), for K = 2, 4, 8 and several CTA widths, up to 2D L=128.
Gaussian: energy conservation of every cluster move, energies consistent
with the spins, and the same equilibrium as the one-CTA layout.  A captured
group with a cluster batch equals its separate launches; a batch that
becomes diluted leaves the cluster layout by itself.
"""
import numpy as np
import pytest
import statcheck

from oracle import oracle as O
from paper_1501_05630_gb300 import inputs as I
from test_gpu_parity import _check_icm_only_step, _compare_sweeps, _e64, _setup, icm  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu


def _cluster(K, threads, growth=-1):
    def setup(b):
        b.set_cluster_growth(growth)
        b.set_cluster(K, threads)
        assert b.cluster() == K and b.info()["threads"] == threads
        assert (b.cluster_growth() > 0) == (growth == 1)    # union-find only when asked for
    return setup


@pytest.mark.parametrize("growth", [1, 0], ids=["union_find", "propagation"])
@pytest.mark.parametrize("kind,L,nT,T_hi,T_icm,n_inst,K,threads", [
    (O.CUBIC3D, 8, 24, 2.0, 1.0, 3, 2, 128),      # two spin words, slabs of 4 planes
    (O.CUBIC3D, 8, 12, 2.0, 1.0, 2, 8, 32),       # one plane per CTA: every z-neighbour remote
    (O.SQUARE2D, 16, 16, 1.5, 1.0, 3, 4, 64),
    (O.CHIMERA, 4, 30, 3.0, 1.5, 2, 2, 32),       # per-site degrees, padded neighbour lists
    (O.SQUARE2D, 32, 32, 1.5, 1.0, 1, 8, 256),    # 64 replicas
    (O.SQUARE2D, 32, 32, 1.5, 1.0, 2, 4, 64),     # four sites per thread: growth by 2 x 2 blocks
])
def test_cluster_pmj_sweep_by_sweep(icm, kind, L, nT, T_hi, T_icm, n_inst, K, threads, growth):
    _compare_sweeps(icm, kind, L, nT, 0.2, T_hi, T_icm, n_inst, 30, 0xC1 + L + K, setup=_cluster(K, threads, growth))


@pytest.mark.parametrize("growth,K,threads", [(1, 8, 1024), (1, 8, 512), (0, 8, 1024), (0, 8, 512)],
                         ids=["union_find_1024", "union_find_512", "propagation_1024", "propagation_512_blocks"])
def test_cluster_2d_L128_64_replicas(icm, growth, K, threads):
    _compare_sweeps(icm, O.SQUARE2D, 128, 32, 0.2, 1.5, 1.0, 1, 6, 0x1502, check_every=3,
                    setup=_cluster(K, threads, growth))


def test_cluster_growth_modes_and_ladder_change(icm):
    """The growth mode switches on a clustered batch without changing the
    chain; a new ladder keeps the batch on clusters; modes outside -1..1
    are refused."""
    icmpt, ctx = icm
    T = I.ladder(0.2, 1.5, 16)
    g, J, s0, ids = _setup(O.SQUARE2D, 32, I.PM_J, 2, T, 0x77)
    runs = []
    for modes in ((1, 1), (0, 1), (1, 0)):
        b = icmpt.Batch(ctx, O.SQUARE2D, 32, I.PM_J, J, T, 1.0, 0x77, spins=s0)
        b.set_cluster(4, 128)
        b.set_cluster_growth(modes[0])
        b.run(5)
        b.set_cluster_growth(modes[1])
        assert b.cluster() == 4 and (b.cluster_growth() > 0) == (modes[1] == 1)
        b.run(5)
        runs.append((b.read_spins(), b.read_energies()))
        with pytest.raises(icmpt.IcmError):
            b.set_cluster_growth(2)
        b.set_temperatures(I.ladder(0.25, 1.5, 16), 1.1)
        assert b.cluster() == 4
        b.close()
    for r in runs[1:]:
        assert np.array_equal(r[0], runs[0][0]) and np.array_equal(r[1], runs[0][1])
    ref = [O.Instance(g, J[a].astype(np.float64), T, s0[a], pm=True, T_icm=1.0, seed=0x77, inst=a) for a in range(2)]
    for a, r in enumerate(ref):
        r.run(10)
        assert np.array_equal(runs[0][0][a], r.s) and np.array_equal(runs[0][1][a], r.E)


def test_cluster_schedule_and_multi_sweep_launches(icm):
    _compare_sweeps(icm, O.CUBIC3D, 8, 10, 0.2, 2.0, 1.0, 2, 40, 77, check_every=7, setup=_cluster(4, 64),
                    icm_every=3, swap_every=2, t_meas=11)


def test_cluster_gauss_conservation_and_consistency(icm):
    """3D L=16 Gaussian on clusters of 8 CTAs: every traced cluster move keeps
    E_a + E_b (each recomputed from the flipped spins by the kernel) to 1e-5
    sum|J|; device energies equal float64 energies of the spins to 1e-5
    sum|J|; then steps of cluster moves alone, checked move by move against
    the spins (conservation in float64, moved sets = the seeds' components)."""
    icmpt, ctx = icm
    T = I.ladder(0.2, 2.0, 24)
    seed = 0x15010563000000C1
    n = 6
    g, J, s0, ids = _setup(O.CUBIC3D, 16, I.GAUSS, n, T, seed)
    b = icmpt.Batch(ctx, O.CUBIC3D, 16, I.GAUSS, J, T, 1.0, seed, spins=s0)
    b.set_cluster(8, 256)
    b.set_schedule(trace=1)
    scale = np.abs(J).astype(np.float64).sum(1)
    moves = 0
    for rep in range(4):
        b.run(5)
        tr = b.read_trace()
        k = tr["n_pre"] >= 0
        moves += int((tr["csize"] > 0).sum())
        err = np.abs(tr["esum_after"] - tr["esum_before"])[k]
        assert np.all(err <= 1e-5 * np.repeat(scale[:, None], 24, 1)[k])
        spins, E = b.read_spins(), b.read_energies()
        assert np.all(np.abs(E - _e64(J, spins, g)) <= 1e-5 * scale[:, None])
        moves += _check_icm_only_step(b, g, J, T, 1.0)
    assert moves > 100


def test_cluster_gauss_equilibrium_equals_one_cta_layout(icm):
    """3D L=8 Gaussian, 96 instances: per-temperature energy and link overlap
    of the cluster layout agree with the one-CTA layout's (paired by
    instance), three standard errors (statcheck)."""
    icmpt, ctx = icm
    T = I.ladder(0.4, 2.0, 8)
    seed = 515
    n = 96
    g, J, s0, ids = _setup(O.CUBIC3D, 8, I.GAUSS, n, T, seed)
    out = []
    for K in (0, 4):
        b = icmpt.Batch(ctx, O.CUBIC3D, 8, I.GAUSS, J, T, 1.0, seed, spins=s0)
        if K:
            b.set_cluster(K, 64)
        b.set_schedule(t_meas=1000)
        b.run(4000)
        o = b.read_observables()
        m = o.n_meas[:, None].astype(np.float64)
        out.append((o.accE / (2 * g.N * m), 1 - 2 * o.acc_d / (g.Nb * m)))
        b.close()
    for i in range(2):
        statcheck.agree(out[1][i] - out[0][i], ("e", "q_l")[i])


def test_group_with_cluster_batch_equals_separate_launches(icm):
    icmpt, ctx = icm
    T = I.ladder(0.2, 2.0, 12)
    batches = []
    for rep in range(2):
        row = []
        for L, n, K in ((8, 5, 4), (4, 7, 0)):
            g, J, s0, ids = _setup(O.CUBIC3D, L, I.PM_J, n, T, 31 + L)
            b = icmpt.Batch(ctx, O.CUBIC3D, L, I.PM_J, J, T, 1.0, 31 + L, spins=s0)
            if K:
                b.set_cluster(K, 64)
            row.append(b)
        batches.append(row)
    grp = icmpt.Group(ctx, batches[0], sweeps_per_launch=5)
    grp.run(3)
    ctx.sync()
    for b in batches[1]:
        b.run(15)
    for a, b in zip(*batches):
        assert np.array_equal(a.read_spins(), b.read_spins())
        assert np.array_equal(a.read_energies(), b.read_energies())
    grp.close()


@pytest.mark.parametrize("lattice,L,K,threads", [(O.CUBIC3D, 8, 4, 64), (O.SQUARE2D, 32, 4, 64)],
                         ids=["3d", "2d_blocks"])
def test_diluted_couplings_keep_the_cluster_layout(icm, lattice, L, K, threads):
    """Loading diluted couplings into a clustered batch keeps it on clusters
    (kernels with per-instance tables); the chain equals the oracle's (2D:
    with the 2 x 2 growth blocks, four sites per thread)."""
    icmpt, ctx = icm
    T = I.ladder(0.3, 2.0, 8)
    g, J, s0, ids = _setup(lattice, L, I.PM_J, 2, T, 5)
    b = icmpt.Batch(ctx, lattice, L, I.PM_J, J, T, 1.0, 5, spins=s0)
    b.set_cluster(K, threads)
    Jd = I.dilute(J, 0.2, 5, ids)
    b.load(couplings=Jd)
    assert b.cluster() == K
    b.run(9)
    spins, E = b.read_spins(), b.read_energies()
    for a in range(2):
        r = O.Instance(g, Jd[a].astype(np.float64), T, s0[a], pm=True, T_icm=1.0, seed=5, inst=a)
        r.run(9)
        assert np.array_equal(spins[a], r.s) and np.array_equal(E[a], r.E)
    b.load(couplings=J)                                   # back to undiluted couplings
    assert b.cluster() == K
    b.close()
