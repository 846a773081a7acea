"""The allocation-free energy entry point against the batch API.

icm_energies_static serves callers that cannot allocate device memory when
they need energies (a pool or arena that forbids outside allocations, a
pipeline that must not hit cudaMalloc's implicit synchronisation, a fixed HBM
budget).  It works on a fixed scratch array inside the library, so this test
checks, on two calls in a row with different inputs, that its results equal
those of icm_batch_create + icm_read_energies on the same spins and
couplings, and that an oversized request is refused with a clear error.
The file name sorts last so that a failing run has already run every other
test.
"""
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
    ctx = icmpt.Context(0, torch.cuda.current_stream().cuda_stream)
    yield icmpt, ctx, torch
    ctx.close()


@pytest.mark.parametrize("lattice,L,disorder,n_inst,nT", [
    (I.CUBIC3D, 8, I.GAUSS, 40, 24),
    (I.CHIMERA, 8, I.PM_J, 40, 30),
    (I.SQUARE2D, 6, I.PM_J, 7, 3),
])
def test_static_energies_match_batch_api(env, lattice, L, disorder, n_inst, nT):
    icmpt, ctx, torch = env
    N, Nb = icmpt.lattice_size(lattice, L)
    T = I.ladder(0.2, 2.0, nT)
    for call, seed in enumerate((101, 202)):                 # two calls in a row
        J = I.couplings(Nb, disorder, seed, range(n_inst))
        s = I.initial_spins(N, 2 * nT, seed, range(n_inst))
        Jd, sd = torch.from_numpy(J).cuda(), torch.from_numpy(s).cuda()
        out = torch.full((n_inst, 2 * nT), float("nan"), dtype=torch.float64, device="cuda")
        icmpt.energies_static(ctx, lattice, L, disorder, Jd, sd, out)
        got = out.cpu().numpy()
        b = icmpt.Batch(ctx, lattice, L, disorder, Jd, T, 1.0, seed, spins=sd)
        want = b.read_energies()
        b.close()
        if disorder == I.PM_J:
            assert np.array_equal(got, want), call
        else:
            tol = 1e-5 * np.abs(J.astype(np.float64)).sum(1, keepdims=True)
            assert np.all(np.abs(got - want) <= tol), call
        # and both equal H = -sum_b J_b s_i s_j evaluated here in float64
        from oracle import oracle as O
        g = O.Geometry(lattice, L)
        ref = -np.einsum("nb,nrb->nr", J.astype(np.float64),
                         (s[:, :, g.bi].astype(np.float64) * s[:, :, g.bj]))
        assert np.allclose(got, ref, rtol=0, atol=1e-4 * np.abs(J).sum() / n_inst + 1e-9)


def test_static_energies_reject_oversized_request(env):
    icmpt, ctx, torch = env
    N, Nb = icmpt.lattice_size(I.CUBIC3D, 8)
    n = 2000                                                  # about 33 MB of scratch: above the fixed 8 MiB
    J = torch.zeros((n, Nb), dtype=torch.float32, device="cuda")
    s = torch.ones((n, 48, N), dtype=torch.int8, device="cuda")
    out = torch.zeros((n, 48), dtype=torch.float64, device="cuda")
    with pytest.raises(icmpt.IcmError) as ei:
        icmpt.energies_static(ctx, I.CUBIC3D, 8, I.GAUSS, J, s, out)
    assert "scratch" in str(ei.value)
