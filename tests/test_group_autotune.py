"""Mixed-size groups (CUDA graph) and the CTA-width autotuner.

A group replays the batches' kernels as one captured graph; for +-J
couplings the results must equal separate launches bit for bit, whatever the
CTA width; autotuning must leave the state untouched."""
import numpy as np
import pytest

from paper_1501_05630_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1501_05630_gb300 import build, icmpt
    build.build()
    torch.cuda.set_device(0)
    ctx = icmpt.Context(0)
    yield icmpt, ctx
    ctx.close()


def _batch(icmpt, ctx, L, n, seed, dis=I.PM_J):
    T = I.ladder(0.2, 2.0, 12)
    N, Nb = icmpt.lattice_size(I.CUBIC3D, L)
    J = I.couplings(Nb, dis, seed, range(n))
    s0 = I.initial_spins(N, 24, seed, range(n))
    return icmpt.Batch(ctx, I.CUBIC3D, L, dis, J, T, 1.0, seed, spins=s0)


def _state(b):
    o = b.read_observables()
    return b.read_spins(), b.read_energies(), b.read_sweeps(), o.accE, o.acc_d, o.hist


def test_group_graph_equals_separate_launches_and_widths(env):
    icmpt, ctx = env
    sizes = [(4, 40), (6, 20), (10, 6)]
    grouped = [_batch(icmpt, ctx, L, n, 3 + L) for L, n in sizes]
    alone = [_batch(icmpt, ctx, L, n, 3 + L) for L, n in sizes]
    grouped[1].set_threads(64)                       # any width gives the same +-J result
    g = icmpt.Group(ctx, grouped, sweeps_per_launch=7)
    g.run(3)
    ctx.sync()
    for b in alone:
        b.run(21)
    for a, b in zip(grouped, alone):
        for x, y in zip(_state(a), _state(b)):
            assert np.array_equal(x, y)
    g.close()


def test_autotune_keeps_state(env):
    icmpt, ctx = env
    b = _batch(icmpt, ctx, 8, 50, 9, dis=I.GAUSS)
    b.run(5)
    before = _state(b)
    th, ms = b.autotune(sweeps=4)
    assert th in (32, 64, 96, 128, 256, 512, 1024) and ms > 0   # wide CTAs too: 256 sites per colour
    assert b.info()["threads"] == th
    for x, y in zip(before, _state(b)):
        assert np.array_equal(x, y)


# ----------------------------------------------------------------------------- shared persistent kernel
def _oracle_batch(g, J, s0, T, T_icm, seed, ids, dis):
    from oracle import oracle as O
    return [O.Instance(g, J[a].astype(np.float64), T, s0[a], pm=(dis == I.PM_J), T_icm=T_icm, seed=seed,
                       inst=int(ids[a])) for a in range(len(ids))]


@pytest.mark.parametrize("lattice,sizes,widths", [
    (I.CUBIC3D, [(4, 5), (6, 3), (8, 2)], None),                 # widths picked: 32, 64, 128
    (I.CUBIC3D, [(4, 3), (6, 2), (8, 2), (10, 1)], [64, 128, 64, 224]),   # named barriers; general growth path
    (I.SQUARE2D, [(8, 6), (16, 3), (32, 2)], [32, 32, 128]),    # degree 4, one-warp teams
    (I.CHIMERA, [(2, 4), (4, 3)], [32, 896]),                    # per-site degrees; one team of the whole CTA
])
def test_shared_group_equals_oracle(env, lattice, sizes, widths):
    """Uneven sizes in one persistent launch of the shared group kernel: every
    +-J instance equals the oracle's chain bit for bit (spins, energies,
    last-sweep decisions, cluster masks, observables) after two launches."""
    from oracle import oracle as O
    icmpt, ctx = env
    seed = 0x5EED
    nT = 10
    T = I.ladder(0.2, 2.0, nT)
    batches, refs, geoms = [], [], []
    for c, (L, n) in enumerate(sizes):
        g = O.Geometry(lattice, L)
        ids = np.arange(n, dtype=np.uint32) + 1000 * c            # one seed: instance ids tell them apart
        J = I.couplings(g.Nb, I.PM_J, seed, ids)
        s0 = I.initial_spins(g.N, 2 * nT, seed, ids)
        b = icmpt.Batch(ctx, lattice, L, I.PM_J, J, T, 1.0, seed, spins=s0, instance_ids=ids)
        b.set_schedule(trace=1)
        batches.append(b)
        refs.append(_oracle_batch(g, J, s0, T, 1.0, seed, ids, I.PM_J))
        geoms.append(g)
    grp = icmpt.Group(ctx, batches, sweeps_per_launch=13, shared=True, team_threads=widths)
    info = grp.info()
    if widths is not None:
        assert info["team_threads"] == widths
    assert info["grid"] >= 1 and info["n_items"] >= len(sizes)
    for launch in range(2):
        grp.run(1)
        for b, rs in zip(batches, refs):
            trs = [r.run(13, trace=True) for r in rs]
            spins, E, tr, cm = b.read_spins(), b.read_energies(), b.read_trace(), b.read_cluster_masks()
            for a, r in enumerate(rs):
                assert np.array_equal(spins[a], r.s), (b.L, a, launch)
                assert np.array_equal(E[a], r.E), (b.L, a, launch)
                assert np.array_equal(cm[a], trs[a]["cmask"]), (b.L, a, launch)
                for key in ("n_pre", "flip2a", "seed_site", "csize", "esum_before", "esum_after"):
                    assert np.array_equal(tr[key][a], trs[a][key]), (b.L, a, key)
                assert np.array_equal(tr["swap_acc"][a], trs[a]["swap_acc"])
    for b, rs in zip(batches, refs):
        o = b.read_observables()
        for a, r in enumerate(rs):
            assert np.array_equal(o.hist[a], r.hist) and np.array_equal(o.acc_d[a], r.acc_d)
            assert np.array_equal(o.accE[a], r.accE) and o.n_meas[a] == r.n_meas[0]
        assert np.all(b.read_sweeps() == 26)
    grp.close()


def test_shared_group_gauss_conservation(env):
    """Gaussian couplings in the shared kernel: every traced cluster move keeps
    E_a + E_b to 1e-5 sum|J|; device energies equal float64 energies of the
    spins to 1e-5 sum|J|, for every size of the group."""
    from oracle import oracle as O
    icmpt, ctx = env
    seed, nT = 77, 24
    T = I.ladder(0.2, 2.0, nT)
    batches, Js, geoms = [], [], []
    for c, (L, n) in enumerate([(4, 30), (6, 14), (8, 7), (12, 2)]):
        g = O.Geometry(I.CUBIC3D, L)
        ids = np.arange(n, dtype=np.uint32) + 1000 * c
        J = I.couplings(g.Nb, I.GAUSS, seed, ids)
        b = icmpt.Batch(ctx, I.CUBIC3D, L, I.GAUSS, J, T, 1.0, seed,
                        spins=I.initial_spins(g.N, 2 * nT, seed, ids), instance_ids=ids)
        b.set_schedule(trace=1)
        batches.append(b)
        Js.append(J)
        geoms.append(g)
    grp = icmpt.Group(ctx, batches, sweeps_per_launch=32, shared=True)
    assert grp.info()["team_threads"] == [32, 64, 128, 448]
    grp.run(3)
    for b, J, g in zip(batches, Js, geoms):
        tr, spins, E = b.read_trace(), b.read_spins(), b.read_energies()
        scale = np.abs(J).astype(np.float64).sum(1)
        k = tr["n_pre"] >= 0
        assert k.sum() == 17 * b.n_inst
        assert np.all(np.abs(tr["esum_after"] - tr["esum_before"])[k] <= 1e-5 * np.repeat(scale[:, None], nT, 1)[k])
        e64 = -np.einsum("nb,nrb->nr", J.astype(np.float64),
                         (spins[:, :, g.bi] * spins[:, :, g.bj]).astype(np.float64))
        assert np.all(np.abs(E - e64) <= 1e-5 * scale[:, None]), b.L
        assert np.all(b.read_sweeps() == 96)
    grp.close()


def test_shared_group_refuses_mixed_kinds(env):
    icmpt, ctx = env
    a = _batch(icmpt, ctx, 4, 2, 5)
    b = _batch(icmpt, ctx, 4, 2, 5, dis=I.GAUSS)
    c = _batch(icmpt, ctx, 4, 2, 6)
    with pytest.raises(icmpt.IcmError):
        icmpt.Group(ctx, [a, b], 4, shared=True)                 # two disorder kinds
    with pytest.raises(icmpt.IcmError):
        icmpt.Group(ctx, [a, c], 4, shared=True)                 # two seeds
    with pytest.raises(icmpt.IcmError):
        icmpt.Group(ctx, [a], 4, shared=True, team_threads=[96])  # not a divisor of 896


def test_group_holds_its_batches(env):
    """A batch of a live group cannot be destroyed (the captured launches
    point at its memory); after the group is closed it can."""
    icmpt, ctx = env
    a = _batch(icmpt, ctx, 4, 2, 5)
    b = _batch(icmpt, ctx, 6, 2, 5)
    for shared in (False, True):
        g = icmpt.Group(ctx, [a, b], 4, shared=shared)
        with pytest.raises(icmpt.IcmError):
            a.close()
        g.run(1)
        g.close()
    a.close()
    b.close()
