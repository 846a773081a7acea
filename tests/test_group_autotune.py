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
