"""Disorder drawn from the seed (couplings = NULL at batch creation).

CPU: the oracle's generator follows the paper's distributions ("Benchmark
model and observables": J = +-1 with probability 1/2, Gaussian N(0, 1)),
checked by binomial and Kolmogorov-Smirnov tests, and is keyed by (seed,
instance id) only.  The Philox stream it reads is pinned separately by the
published known-answer vectors.

GPU: a batch created without couplings holds exactly the oracle's draws
(+-J and Gaussian), a slot replaced without couplings draws its instance id's
couplings, and the +-J chain on them equals the oracle's sweep by sweep."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1501_05630_gb300 import inputs as I


def test_pmj_draws_are_fair_coins_in_every_word():
    J = O.philox_couplings(4000, True, 0x1501, range(4)).astype(np.int64)
    assert set(np.unique(J)) == {-1, 1}
    for w in range(4):                        # each of the four Philox words
        x = J[:, w::4].ravel()
        n, plus = x.size, int(np.count_nonzero(x == 1))
        assert abs(plus - n / 2) <= 4.5 * math.sqrt(n / 4), (w, plus, n)


def test_gauss_draws_are_standard_normal():
    scipy_stats = pytest.importorskip("scipy.stats")
    G = O.philox_couplings(6000, False, 0x1502, range(2)).astype(np.float64).ravel()
    assert G.dtype == np.float64 and np.all(np.isfinite(G))
    n = G.size
    assert abs(G.mean()) <= 4.5 / math.sqrt(n)
    assert abs(G.var() - 1.0) <= 4.5 * math.sqrt(2.0 / n)
    assert scipy_stats.kstest(G, "norm").pvalue > 1e-4


def test_draws_keyed_by_seed_and_instance_only():
    a = O.philox_couplings(64, True, 7, [3, 9])
    b = O.philox_couplings(64, True, 7, [9])
    assert np.array_equal(a[1], b[0])                  # the same id gives the same row
    assert not np.array_equal(a[0], a[1])
    assert not np.array_equal(O.philox_couplings(64, True, 8, [3])[0], a[0])
    g = O.philox_couplings(32, False, 7, [3])
    assert g.dtype == np.float32 and not np.array_equal(g, O.philox_couplings(32, False, 7, [4]))


@pytest.fixture(scope="module")
def icm():
    import torch
    from paper_1501_05630_gb300 import build, icmpt
    build.build()
    torch.cuda.set_device(0)
    ctx = icmpt.Context(0)
    yield icmpt, ctx
    ctx.close()


@pytest.mark.gpu
@pytest.mark.parametrize("kind,L,dis", [(O.CUBIC3D, 4, I.PM_J), (O.CHIMERA, 2, I.PM_J), (O.SQUARE2D, 6, I.GAUSS),
                                        (O.CUBIC3D, 4, I.GAUSS)])
def test_batch_draws_the_oracle_disorder(icm, kind, L, dis):
    icmpt, ctx = icm
    g = O.Geometry(kind, L)
    ids = [5, 9, 200]
    seed = 0xD15C0
    T = I.ladder(0.3, 2.0, 6)
    b = icmpt.Batch(ctx, kind, L, dis, None, T, 1.0, seed, instance_ids=ids)
    want = O.philox_couplings(g.Nb, dis == I.PM_J, seed, ids)
    got = b.read_couplings()
    assert got.dtype == want.dtype and np.array_equal(got, want)
    # a slot replaced without couplings draws those of its new instance id
    b.set_slot(1, None, None, instance_id=77)
    got = b.read_couplings()
    assert np.array_equal(got[1], O.philox_couplings(g.Nb, dis == I.PM_J, seed, [77])[0])
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[2], want[2])
    b.close()


@pytest.mark.gpu
def test_chain_on_drawn_pmj_disorder_equals_oracle(icm):
    icmpt, ctx = icm
    kind, L, nT, seed = O.CUBIC3D, 4, 10, 0xD15C1
    g = O.Geometry(kind, L)
    ids = [0, 1]
    T = I.ladder(0.2, 2.0, nT)
    s0 = I.initial_spins(g.N, 2 * nT, seed, ids)
    b = icmpt.Batch(ctx, kind, L, I.PM_J, None, T, 1.0, seed, spins=s0, instance_ids=ids)
    J = O.philox_couplings(g.Nb, True, seed, ids)
    refs = [O.Instance(g, J[a].astype(np.float64), T, s0[a], pm=True, T_icm=1.0, seed=seed, inst=ids[a])
            for a in range(len(ids))]
    for _ in range(12):
        b.run(1)
        for r in refs:
            r.run(1)
        spins, E = b.read_spins(), b.read_energies()
        for a, r in enumerate(refs):
            assert np.array_equal(spins[a], r.s)
            assert np.array_equal(E[a], r.E)
    b.close()
