"""Parity of the CUDA library with the oracle on the widened geometry:
4D hypercubic lattices and diluted lattices (bonds with J = 0 absent).

+-J: bit-exact sweep by sweep (spins, integer energies, step-2a decisions,
seeds, cluster sizes, PT decisions, observables), in both layouts, with
diluted and undiluted instances in one batch (the zero-energy rule is per
instance).  Gaussian: statistical agreement and energy conservation.  Site
percolation on 4D lattices: largest clusters equal the oracle's.
"""

import numpy as np
import pytest
import statcheck

from oracle import oracle as O
from paper_1501_05630_gb300 import inputs as I
from test_gpu_parity import _check_icm_only_step, _e64

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


TRACE_KEYS = ("n_pre", "flip2a", "seed_site", "csize", "esum_before", "esum_after")


def _couplings(g, dis, seed, ids, dilution, diluted_rows):
    J = I.couplings(g.Nb, dis, seed, ids)
    if dilution > 0:
        Jd = I.dilute(J, dilution, seed, ids)
        rows = list(range(len(ids))) if diluted_rows is None else list(diluted_rows)
        J[rows] = Jd[rows]
    return J


def _compare(icm, kind, L, nT, T_hi, T_icm, n_inst, sweeps, seed, dilution=0.0, diluted_rows=None,
             threads=None, check_every=1, cluster=None):
    icmpt, ctx = icm
    T = I.ladder(0.2, T_hi, nT)
    g = O.Geometry(kind, L)
    ids = list(range(n_inst))
    J = _couplings(g, I.PM_J, seed, ids, dilution, diluted_rows)
    s0 = I.initial_spins(g.N, 2 * nT, seed, ids)
    b = icmpt.Batch(ctx, kind, L, I.PM_J, J, T, T_icm, seed, spins=s0)
    if threads is not None:
        b.set_threads(threads)
    if cluster is not None:
        b.set_cluster(*cluster)
        assert b.cluster() == cluster[0]
    b.set_schedule(trace=1, t_meas=sweeps // 3)
    assert np.array_equal(b.bond_counts(), np.count_nonzero(J, axis=1))
    refs = [O.Instance(g, J[a].astype(np.float64), T, s0[a], pm=True, T_icm=T_icm, seed=seed, inst=a,
                       t_meas=sweeps // 3) for a in range(n_inst)]
    done = 0
    while done < sweeps:
        step = min(check_every, sweeps - done)
        b.run(step)
        trs = [r.run(step, trace=True) for r in refs]
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
    o = b.read_observables()
    for a, r in enumerate(refs):
        for f in ("accE", "acc_n", "acc_q2", "acc_pmin", "acc_d", "hist"):
            assert np.array_equal(getattr(o, f)[a], getattr(r, f)), f
        assert o.n_meas[a] == r.n_meas[0]
        assert o.nb[a] == r.nb_present
    b.close()


@pytest.mark.parametrize("L,nT,n_inst,threads", [
    (4, 12, 2, None),        # 256 sites, 24 replicas, shared memory
    (2, 6, 2, None),         # doubled bonds of the smallest hypercube
    (4, 30, 1, 256),         # 60 replicas, wide layout
    (6, 16, 1, None),        # 1296 sites
])
def test_4d_pmj_sweep_by_sweep(icm, L, nT, n_inst, threads):
    _compare(icm, O.HYPERCUBIC4D, L, nT, 3.0, 1.5, n_inst, 24, 0x4D + L, threads=threads)


@pytest.mark.parametrize("kind,L,nT,T_hi,T_icm,dilution,rows,threads", [
    (O.SQUARE2D, 8, 12, 1.5, 1.0, 0.3, None, None),         # every instance diluted
    (O.SQUARE2D, 8, 12, 1.5, 1.0, 0.3, [1], None),          # one diluted, two undiluted: per-instance rule
    (O.CUBIC3D, 4, 16, 2.0, 1.0, 0.25, [0, 2], None),
    (O.CUBIC3D, 6, 10, 2.0, 1.0, 0.4, None, 256),           # wide layout
    (O.CHIMERA, 3, 20, 3.0, 1.5, 0.2, None, None),          # per-site degrees below 4
    (O.HYPERCUBIC4D, 4, 8, 3.0, 1.5, 0.3, [0], None),
    (O.SQUARE2D, 6, 4, 1.5, 1.0, 0.9, None, None),          # mostly isolated sites (degree 0)
])
def test_diluted_pmj_sweep_by_sweep(icm, kind, L, nT, T_hi, T_icm, dilution, rows, threads):
    _compare(icm, kind, L, nT, T_hi, T_icm, 3, 30, 0xD1 + L, dilution=dilution, diluted_rows=rows,
             threads=threads)


def test_fully_diluted_every_swap_accepted(icm):
    """Every bond absent: all energies are 0, so every PT swap is accepted and
    each copy's pass is one run over all 32 temperatures (the longest run the
    decision warp can form); sweep by sweep equal to the oracle."""
    icmpt, ctx = icm
    _compare(icm, O.CUBIC3D, 4, 32, 2.0, 1.0, 2, 6, 0xF0, dilution=1.0)
    _compare(icm, O.SQUARE2D, 4, 2, 1.5, 1.0, 1, 6, 0xF1, dilution=1.0)   # one pair: a run of one swap


@pytest.mark.parametrize("kind,L,nT,T_hi,T_icm,dilution,rows,cluster", [
    (O.SQUARE2D, 16, 12, 1.5, 1.0, 0.3, None, (4, 64)),
    (O.SQUARE2D, 16, 16, 1.5, 1.0, 0.3, [1], (2, 128)),      # diluted and undiluted instances together
    (O.CUBIC3D, 8, 24, 2.0, 1.0, 0.25, None, (8, 32)),      # two spin words; every z-neighbour remote
    (O.CHIMERA, 4, 20, 3.0, 1.5, 0.2, None, (2, 64)),       # per-site degrees below 4
    (O.SQUARE2D, 16, 8, 1.5, 1.0, 0.9, None, (4, 32)),      # mostly isolated sites
    (O.HYPERCUBIC4D, 4, 12, 3.0, 1.5, 0.3, [0], (4, 32)),   # 4D (Z = 8), one diluted instance
    (O.HYPERCUBIC4D, 8, 8, 3.0, 1.5, 0.0, None, (8, 64)),   # 4D L=8 undiluted, 4096 sites
])
def test_diluted_cluster_layout_sweep_by_sweep(icm, kind, L, nT, T_hi, T_icm, dilution, rows, cluster):
    """Diluted batches and 4D lattices on thread-block clusters: per-instance
    neighbour tables in every CTA's slice, a fourth bit-plane for Z = 8;
    bit-exact with the oracle sweep by sweep."""
    _compare(icm, kind, L, nT, T_hi, T_icm, 3, 24, 0xC1D + L, dilution=dilution, diluted_rows=rows,
             cluster=cluster)


def test_diluted_instance_admitted_into_undiluted_batch(icm):
    """A slot replaced by a diluted instance switches the batch to its diluted
    kernels; every slot still evolves like its instance alone."""
    icmpt, ctx = icm
    T = I.ladder(0.3, 2.0, 10)
    g = O.Geometry(O.CUBIC3D, 4)
    J = I.couplings(g.Nb, I.PM_J, 9, range(4))
    s0 = I.initial_spins(g.N, 20, 9, range(4))
    b = icmpt.Batch(ctx, O.CUBIC3D, 4, I.PM_J, J[:3].copy(), T, 1.0, 9, spins=s0[:3].copy())
    b.run(5)
    Jd = I.dilute(J[3:4], 0.3, 9, [3])[0]
    b.set_slot(1, Jd, s0[3], instance_id=3)
    assert list(b.bond_counts()) == [g.Nb, int(np.count_nonzero(Jd)), g.Nb]
    b.run(11)
    spins, E = b.read_spins(), b.read_energies()
    for slot, Jrow, s_init, inst, sweeps in ((0, J[0], s0[0], 0, 16), (1, Jd, s0[3], 3, 11), (2, J[2], s0[2], 2, 16)):
        r = O.Instance(g, Jrow.astype(np.float64), T, s_init, pm=True, T_icm=1.0, seed=9, inst=inst)
        r.run(sweeps)
        assert np.array_equal(spins[slot], r.s), slot
        assert np.array_equal(E[slot], r.E), slot
    b.close()


def test_diluted_gauss_statistics_and_conservation(icm):
    """3D L=4 Gaussian with 30% of the bonds absent: per-temperature energy and
    link overlap agree with the oracle's (paired by instance, three standard
    errors: statcheck); every cluster move keeps E_a + E_b to 1e-5 sum|J|."""
    icmpt, ctx = icm
    T = I.ladder(0.3, 2.0, 8)
    seed = 777
    n = 64
    g = O.Geometry(O.CUBIC3D, 4)
    ids = list(range(n))
    J = I.dilute(I.couplings(g.Nb, I.GAUSS, seed, ids), 0.3, seed, ids)
    s0 = I.initial_spins(g.N, 16, seed, ids)
    sweeps, t_meas = 3000, 1000
    b = icmpt.Batch(ctx, O.CUBIC3D, 4, I.GAUSS, J, T, 1.0, seed, spins=s0)
    b.set_schedule(t_meas=t_meas, trace=1)
    b.run(sweeps)
    tr = b.read_trace()
    scale = np.abs(J).astype(np.float64).sum(1)
    k = tr["n_pre"] >= 0
    assert np.all(np.abs(tr["esum_after"] - tr["esum_before"])[k] <= 1e-5 * np.repeat(scale[:, None], 8, 1)[k])
    o = b.read_observables()
    assert np.array_equal(o.nb, np.count_nonzero(J, axis=1))
    m = o.n_meas[:, None].astype(np.float64)
    gpu = dict(e=o.accE / (2 * g.N * m), q_l=1 - 2 * o.acc_d / (o.nb[:, None] * m))
    cpu = {key: [] for key in gpu}
    for a in range(n):
        r = O.Instance(g, J[a].astype(np.float64), T, s0[a], pm=False, T_icm=1.0, seed=seed, inst=a, t_meas=t_meas)
        r.run(sweeps)
        ob = r.observables()
        for key in cpu:
            cpu[key].append(ob[key])
    for key in gpu:
        statcheck.agree(gpu[key] - np.asarray(cpu[key]), key)


def test_diluted_gauss_cluster_layout_conservation(icm):
    """3D L=8 Gaussian with 30% of the bonds absent on clusters of 8 CTAs:
    every cluster move keeps E_a + E_b to 1e-5 sum|J|, the device energies
    equal fp64 energies of the spins over the bonds present, and steps of
    cluster moves alone conserve E_a + E_b of the spins in float64 and move
    the seeds' components through the bonds present."""
    icmpt, ctx = icm
    T = I.ladder(0.3, 2.0, 12)
    seed, n = 778, 4
    g = O.Geometry(O.CUBIC3D, 8)
    ids = list(range(n))
    J = I.dilute(I.couplings(g.Nb, I.GAUSS, seed, ids), 0.3, seed, ids)
    s0 = I.initial_spins(g.N, 24, seed, ids)
    b = icmpt.Batch(ctx, O.CUBIC3D, 8, I.GAUSS, J, T, 1.0, seed, spins=s0)
    b.set_cluster(8, 32)
    assert b.cluster() == 8
    b.set_schedule(trace=1)
    scale = np.abs(J).astype(np.float64).sum(1)
    moves = 0
    for _ in range(5):
        b.run(9)
        tr = b.read_trace()
        k = tr["n_pre"] >= 0
        moves += int((tr["csize"] > 0).sum())
        assert np.all(np.abs(tr["esum_after"] - tr["esum_before"])[k] <= 1e-5 * np.repeat(scale[:, None], 12, 1)[k])
        spins, E = b.read_spins(), b.read_energies()
        assert np.all(np.abs(E - _e64(J, spins, g)) <= 1e-5 * scale[:, None])
        moves += _check_icm_only_step(b, g, J, T, 1.0)
    assert moves > 20
    b.close()


def test_percolation_4d_matches_oracle(icm):
    icmpt, ctx = icm
    g = O.Geometry(O.HYPERCUBIC4D, 6)
    masks = I.site_masks(g.N, 0.2, 5, 64)
    got = icmpt.largest_clusters(ctx, O.HYPERCUBIC4D, 6, masks)
    assert np.array_equal(got, O.largest_clusters(g, masks))
