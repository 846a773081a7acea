"""Device memory of a context: the budget and the allocator hooks.

* A batch that does not fit the budget fails with ICM_ERR_BUDGET and leaves
  nothing allocated; one that fits is counted while alive and released on
  close.  Scratch of the percolation calls counts against the budget too.
* With PyTorch's caching allocator as the hook, the library's blocks show in
  torch.cuda.memory_allocated() and go back when the batch closes, and the
  chain is the same as on a plain context (+-J, bit for bit)."""
import numpy as np
import pytest

from paper_1501_05630_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ERR_BUDGET = -3


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_1501_05630_gb300 import build, icmpt
    build.build()
    torch.cuda.set_device(0)
    return icmpt


def _batch(icmpt, ctx, lattice, L, dis, n, seed=21):
    N, Nb = icmpt.lattice_size(lattice, L)
    T = I.ladder(0.3, 2.0, 8)
    J = I.couplings(Nb, dis, seed, range(n))
    s0 = I.initial_spins(N, 16, seed, range(n))
    return icmpt.Batch(ctx, lattice, L, dis, J, T, 1.0, seed, spins=s0)


def test_budget_refuses_and_counts(lib):
    icmpt = lib
    ctx = icmpt.Context(0, hbm_budget=1 << 20)
    with pytest.raises(icmpt.IcmError) as ei:
        _batch(icmpt, ctx, I.CUBIC3D, 8, I.GAUSS, 200)
    assert ei.value.code == ERR_BUDGET
    assert ctx.memory() == (0, 1 << 20)                      # the failed creation freed its blocks
    b = _batch(icmpt, ctx, I.SQUARE2D, 4, I.PM_J, 2)
    used, budget = ctx.memory()
    assert 0 < used <= budget
    b.run(3)
    b.close()
    assert ctx.memory()[0] == 0
    with pytest.raises(icmpt.IcmError) as ei:               # 5000 chimera C_16 masks need ~10 MB
        icmpt.largest_clusters(ctx, I.CHIMERA, 16, np.zeros((5000, 8 * 16 * 16), dtype=np.uint8))
    assert ei.value.code == ERR_BUDGET and ctx.memory()[0] == 0
    ctx.close()


def test_torch_allocator_owns_the_blocks(lib):
    import torch
    icmpt = lib
    plain = icmpt.Context(0)
    hooked = icmpt.Context(0, allocator="torch")
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    a = _batch(icmpt, plain, I.CUBIC3D, 4, I.PM_J, 3)
    b = _batch(icmpt, hooked, I.CUBIC3D, 4, I.PM_J, 3)
    used = hooked.memory()[0]
    assert used > 0 and plain.memory()[0] > 0
    assert torch.cuda.memory_allocated() - before >= used
    a.run(20)
    b.run(20)
    assert np.array_equal(a.read_spins(), b.read_spins())
    assert np.array_equal(a.read_energies(), b.read_energies())
    b.close()
    torch.cuda.synchronize()
    assert hooked.memory()[0] == 0
    assert torch.cuda.memory_allocated() == before
    a.close()
    plain.close()
    hooked.close()
