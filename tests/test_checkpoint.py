"""Checkpoint / resume of a batch.

The random numbers are counter-based (Philox keyed by seed, instance, sweep
and site), so a batch's whole state is its device arrays: running 2n sweeps
must equal running n, saving, restoring into a fresh batch of the same shape
and seed, and running n more -- bit for bit, for +-J and Gaussian couplings,
with and without serving-slot state."""
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


def _batch(icmpt, ctx, lattice, L, n, dis, seed, J=None, s0=None):
    T = I.ladder(0.2, 2.0, 10)
    N, Nb = icmpt.lattice_size(lattice, L)
    if J is None:
        J = I.couplings(Nb, dis, seed, range(n))
        s0 = I.initial_spins(N, 20, seed, range(n))
    b = icmpt.Batch(ctx, lattice, L, dis, J, T, 1.0, seed, spins=s0)
    b.set_schedule(t_meas=4)
    return b


def _state(b):
    o = b.read_observables()
    return (b.read_spins(), b.read_energies(), b.read_sweeps(), o.accE, o.acc_n, o.acc_q2,
            o.acc_pmin, o.acc_d, o.hist, o.n_meas)


@pytest.mark.parametrize("lattice,L,dis", [(I.CUBIC3D, 6, I.GAUSS), (I.CUBIC3D, 6, I.PM_J),
                                           (I.CHIMERA, 4, I.PM_J), (I.SQUARE2D, 10, I.GAUSS)])
def test_resume_equals_uninterrupted(env, lattice, L, dis):
    icmpt, ctx = env
    n = 7
    ref = _batch(icmpt, ctx, lattice, L, n, dis, 5)
    ref.run(12)
    a = _batch(icmpt, ctx, lattice, L, n, dis, 5)
    a.run(6)
    blob = a.checkpoint()
    a.close()
    # a fresh batch with other couplings and spins: the checkpoint replaces both
    N, Nb = icmpt.lattice_size(lattice, L)
    other_J = I.couplings(Nb, dis, 99, range(n))
    other_s = I.initial_spins(N, 20, 99, range(n))
    b = _batch(icmpt, ctx, lattice, L, n, dis, 5, other_J, other_s)
    b.restore(blob)
    b.run(6)
    for x, y in zip(_state(ref), _state(b)):
        assert np.array_equal(x, y)


def test_resume_keeps_slot_state(env):
    icmpt, ctx = env
    n = 6
    lattice, L, dis = I.CUBIC3D, 4, I.PM_J
    N, Nb = icmpt.lattice_size(lattice, L)
    J_new = I.couplings(Nb, dis, 11, [1000])[0]
    s_new = I.initial_spins(N, 20, 11, [1000])[0]

    def prepare(b):
        b.run(3)
        b.set_slot(2, J_new, s_new, instance_id=1000)
        b.set_active(4, False)
        b.start_window(1, 5)
        b.run(4)

    ref = _batch(icmpt, ctx, lattice, L, n, dis, 8)
    prepare(ref)
    ref.run(5)
    a = _batch(icmpt, ctx, lattice, L, n, dis, 8)
    prepare(a)
    blob = a.checkpoint()
    b = _batch(icmpt, ctx, lattice, L, n, dis, 8)
    b.restore(blob)
    b.run(5)
    for x, y in zip(_state(ref), _state(b)):
        assert np.array_equal(x, y)
    # the inactive slot did not move after the restore either
    assert b.read_sweeps()[4] == ref.read_sweeps()[4]


def test_restore_rejects_mismatch(env):
    icmpt, ctx = env
    a = _batch(icmpt, ctx, I.CUBIC3D, 4, 3, I.PM_J, 1)
    blob = a.checkpoint()
    other_shape = _batch(icmpt, ctx, I.CUBIC3D, 4, 4, I.PM_J, 1)
    with pytest.raises(icmpt.IcmError):
        other_shape.restore(blob)
    other_seed = _batch(icmpt, ctx, I.CUBIC3D, 4, 3, I.PM_J, 2)
    with pytest.raises(icmpt.IcmError):
        other_seed.restore(blob)
    with pytest.raises(icmpt.IcmError):
        a.restore(blob[:-1])
    with pytest.raises(icmpt.IcmError):
        a.restore(b"not a checkpoint" + blob[16:])
    a.restore(blob)                        # the untouched blob still loads
