"""Serving (continuous batching) and the thermalization criterion.

CPU: the per-instance test of icm_therm_update -- stability of the block means
of e and q_l over doubling windows, and delta = E(q_l) - e with Eq. 1's
E(q_l) = -(N_b/N)(1 - q_l)/T.
GPU: a slot replaced inside a running batch evolves exactly as the same
instance alone; every request that the server runs to thermalization reports
the same sweeps and window accumulators as the instance replayed alone
(random streams are keyed by seed and instance id, never by slot); the
batch-averaged delta of Eq. 2 equals its host computation.
"""
import numpy as np
import pytest

from paper_1501_05630_gb300 import inputs as I


@pytest.fixture(scope="module")
def lib():
    from paper_1501_05630_gb300 import build, icmpt
    build.build()
    return icmpt


def test_therm_update_stability_and_eq1(lib):
    icmpt = lib
    st, cr = icmpt.ThermState(), icmpt.ThermCriterion(0.01, 0.02, 2)
    seq = [(-1.50, 0.50), (-1.60, 0.60), (-1.605, 0.61), (-1.606, 0.605), (-1.40, 0.60), (-1.401, 0.601)]
    flags = [icmpt.therm_update(st, cr, e, q, 0.5, 3.0) for e, q in seq]
    # agreement with the previous window needed twice in a row; a jump resets it
    assert flags == [False, False, False, True, False, False]
    assert st.blocks == 6 and st.stable == 1
    assert st.delta == pytest.approx(-(3.0 / 0.5) * (1 - 0.601) - (-1.401))
    assert list(st.e)[:3] == [-1.401, -1.40, -1.606]
    with pytest.raises(icmpt.IcmError):
        icmpt.therm_update(st, cr, 0, 0, 0.0, 3.0)


def test_native_server_host_logic(lib):
    """Request validation, rejection by the memory budget and the queue, on
    the host (no class is created before the first step)."""
    icmpt = lib
    from paper_1501_05630_gb300.serve import Request, Server
    N, Nb = icmpt.lattice_size(I.SQUARE2D, 8)
    T = I.ladder(0.3, 1.5, 8)
    ok = Request(I.SQUARE2D, 8, I.PM_J, T, 1.0, 1, 7, I.couplings(Nb, I.PM_J, 1, [7])[0])
    srv = Server(slots_per_class=4, quantum=16, hbm_budget=8 << 20)
    t = srv.submit(ok)
    assert srv.poll(t) is None                              # pending
    assert srv.status() == (1, 0, 0)
    with pytest.raises(icmpt.IcmError) as e:                 # descending ladder
        srv.submit(Request(I.SQUARE2D, 8, I.PM_J, T[::-1].copy(), 1.0, 1, 8, ok.couplings))
    assert e.value.code == -1
    with pytest.raises(icmpt.IcmError) as e:                 # instance id beyond the RNG key
        srv.submit(Request(I.SQUARE2D, 8, I.PM_J, T, 1.0, 1, 1 << 24, ok.couplings))
    assert e.value.code == -1
    N2, Nb2 = icmpt.lattice_size(I.SQUARE2D, 128)
    big = Request(I.SQUARE2D, 128, I.PM_J, I.ladder(0.2, 1.5, 32), 1.0, 1, 9, np.ones(Nb2, np.int8))
    with pytest.raises(icmpt.IcmError) as e:                 # its class alone (21 MiB) exceeds 8 MiB
        srv.submit(big)
    assert e.value.code == -3
    with pytest.raises(icmpt.IcmError):
        srv.poll(12345)                                      # unknown ticket
    assert srv.status() == (1, 0, 0)
    t2 = srv.submit(Request(I.SQUARE2D, 8, I.PM_J, T, 1.0, 1, 8, ok.couplings))
    srv.cancel(t2)                                           # queued: dropped at once
    assert srv.poll(t2).status == "cancelled" and srv.poll(t2).sweeps == 0
    with pytest.raises(icmpt.IcmError) as e:
        srv.cancel(t2)
    assert e.value.code == -6
    assert srv.status() == (1, 0, 0) and srv.poll(t) is None
    srv.close()
    with pytest.raises(ValueError):
        Server(quantum=48)


@pytest.fixture(scope="module")
def gpu(lib):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA GPU")
    torch.cuda.set_device(0)
    ctx = lib.Context(0)
    yield lib, ctx
    ctx.close()


@pytest.mark.gpu
def test_slot_replacement_matches_instance_alone(gpu):
    icmpt, ctx = gpu
    T = I.ladder(0.3, 2.0, 10)
    g_N, g_Nb = icmpt.lattice_size(I.CUBIC3D, 4)
    J = I.couplings(g_Nb, I.PM_J, 3, range(6))
    s0 = I.initial_spins(g_N, 20, 3, range(6))
    b = icmpt.Batch(ctx, I.CUBIC3D, 4, I.PM_J, J[:4].copy(), T, 1.0, 3, spins=s0[:4].copy())
    b.set_active(-1, False)
    b.set_slot(2, J[4], s0[4], instance_id=4)
    b.start_window(2, 8)
    b.run(20)
    b.set_slot(0, J[5], s0[5], instance_id=5)       # admitted while slot 2 runs
    b.start_window(0, 0)
    b.run(13)
    spins, E, o, t = b.read_spins(), b.read_energies(), b.read_observables(), b.read_sweeps()
    for slot, inst, sweeps, t_meas in ((2, 4, 33, 8), (0, 5, 13, 0)):
        a = icmpt.Batch(ctx, I.CUBIC3D, 4, I.PM_J, J[inst:inst + 1].copy(), T, 1.0, 3,
                        spins=s0[inst:inst + 1].copy(), instance_ids=[inst])
        a.set_schedule(t_meas=t_meas)
        a.run(sweeps)
        oa = a.read_observables()
        assert t[slot] == sweeps
        assert np.array_equal(spins[slot], a.read_spins()[0])
        assert np.array_equal(E[slot], a.read_energies()[0])
        for f in ("accE", "acc_n", "acc_q2", "acc_pmin", "acc_d", "hist", "n_meas"):
            assert np.array_equal(getattr(o, f)[slot], getattr(oa, f)[0]), f
        a.close()
    # free slots were skipped
    assert t[1] == 0 and t[3] == 0


def _requests(icmpt, n, seed=77):
    rng = np.random.default_rng(seed)
    menu = [(I.SQUARE2D, 8, (0.3, 1.5), 1.0), (I.SQUARE2D, 16, (0.3, 1.5), 1.0), (I.CUBIC3D, 4, (0.4, 2.0), 1.0),
            (I.CHIMERA, 4, (0.3, 3.0), 1.5)]
    reqs = []
    for i in range(n):
        lat, L, (tl, th), ticm = menu[rng.integers(len(menu))]
        nT = int(rng.choice([8, 12]))
        N, Nb = icmpt.lattice_size(lat, L)
        from paper_1501_05630_gb300.serve import Request
        reqs.append(Request(lat, L, I.PM_J, I.ladder(tl, th, nT), ticm, 11, 1000 + i,
                            I.couplings(Nb, I.PM_J, 11, [1000 + i])[0], I.initial_spins(N, 2 * nT, 11, [1000 + i])[0]))
    return reqs


@pytest.mark.gpu
def test_server_results_equal_each_instance_alone(gpu):
    icmpt, ctx = gpu
    from paper_1501_05630_gb300.serve import Server
    reqs = _requests(icmpt, 24)
    srv = Server(slots_per_class=4, quantum=16, eps_e=0.02, eps_ql=0.05, need=2, max_sweeps=1024)
    tickets = [srv.submit(r) for r in reqs]
    srv.run_until_idle()
    res = [srv.poll(t) for t in tickets]
    assert all(r is not None for r in res)
    assert {r.status for r in res} <= {"thermalized", "not_thermalized"}
    assert sum(r.status == "thermalized" for r in res) > 0
    for r, q in zip(res, reqs):
        assert r.sweeps <= 1024 and r.sweeps % 16 == 0
        a = icmpt.Batch(ctx, q.lattice, q.L, q.disorder, q.couplings[None].copy(), q.T, q.T_icm, q.seed,
                        spins=q.spins[None].copy(), instance_ids=[q.instance_id])
        a.set_schedule(t_meas=r.sweeps // 2)          # the last doubling window [t/2, t)
        a.run(r.sweeps)
        oa = a.read_observables(hist=False)
        assert oa.accE[0, 0] == r.accE and oa.acc_d[0, 0] == r.acc_d and oa.n_meas[0] == r.n_meas
        a.close()
    srv.close()


@pytest.mark.gpu
def test_server_draws_couplings_when_none_given(gpu):
    """Requests without couplings get the disorder drawn from their seed and
    instance id: each result equals the instance replayed alone from a batch
    that draws the same couplings."""
    icmpt, ctx = gpu
    from paper_1501_05630_gb300.serve import Request, Server
    reqs = []
    for i in range(6):
        lat, L = (I.SQUARE2D, 8) if i % 2 else (I.CUBIC3D, 4)
        reqs.append(Request(lat, L, I.PM_J, I.ladder(0.3, 1.5, 8), 1.0, 13, 2000 + i, None, None))
    srv = Server(slots_per_class=2, quantum=16, eps_e=0.02, eps_ql=0.05, need=2, max_sweeps=256)
    tickets = [srv.submit(r) for r in reqs]
    srv.run_until_idle()
    for t, q in zip(tickets, reqs):
        r = srv.poll(t)
        a = icmpt.Batch(ctx, q.lattice, q.L, q.disorder, None, q.T, q.T_icm, q.seed, instance_ids=[q.instance_id])
        a.set_schedule(t_meas=r.sweeps // 2)
        a.run(r.sweeps)
        oa = a.read_observables(hist=False)
        assert oa.accE[0, 0] == r.accE and oa.acc_d[0, 0] == r.acc_d and oa.n_meas[0] == r.n_meas
        a.close()
    srv.close()


@pytest.mark.gpu
def test_batch_delta_matches_host(gpu):
    icmpt, ctx = gpu
    T = I.ladder(0.5, 2.0, 6)
    N, Nb = icmpt.lattice_size(I.CUBIC3D, 4)
    J = I.couplings(Nb, I.GAUSS, 5, range(32))
    b = icmpt.Batch(ctx, I.CUBIC3D, 4, I.GAUSS, J, T, 1.0, 5, spins=I.initial_spins(N, 12, 5, range(32)))
    b.set_schedule(t_meas=100)
    b.run(400)
    o = b.read_observables(hist=False)
    for k in (0, 3):
        m = o.n_meas.astype(np.float64)
        e = o.accE[:, k] / (2 * N * m)
        ql = 1 - 2 * o.acc_d[:, k] / (Nb * m)
        d = -(Nb / N) * (1 - ql) / T[k] - e
        mean, se, n = b.delta(k)
        assert n == 32 and mean == pytest.approx(d.mean(), rel=1e-12, abs=1e-12)
        assert se == pytest.approx(d.std() / np.sqrt(31), rel=1e-9)


@pytest.mark.gpu
def test_server_mixes_wide_and_shared_memory_classes(gpu):
    """2D L=128 requests (global-resident layout, one slow class) served
    beside small shared-memory classes: classes advance independently, and
    every result equals the instance replayed alone."""
    icmpt, ctx = gpu
    from paper_1501_05630_gb300.serve import Request, Server
    reqs = []
    for i, (L, nT) in enumerate([(128, 8), (8, 8), (8, 12), (128, 8), (16, 8), (8, 8)]):
        N, Nb = icmpt.lattice_size(I.SQUARE2D, L)
        inst = 3000 + i
        reqs.append(Request(I.SQUARE2D, L, I.PM_J, I.ladder(0.5, 1.5, nT), 1.0, 13, inst,
                            I.couplings(Nb, I.PM_J, 13, [inst])[0], I.initial_spins(N, 2 * nT, 13, [inst])[0]))
    srv = Server(slots_per_class=2, quantum=16, eps_e=0.02, eps_ql=0.05, need=2, max_sweeps=256)
    tickets = [srv.submit(r) for r in reqs]
    srv.run_until_idle()
    res = [srv.poll(t) for t in tickets]
    assert all(r is not None for r in res)
    info = srv.class_info()
    assert [c.L for c in info if c.threads > 128] == [128]     # the one wide class
    assert all(c.active == 0 for c in info)
    for r, q in zip(res, reqs):
        a = icmpt.Batch(ctx, q.lattice, q.L, q.disorder, q.couplings[None].copy(), q.T, q.T_icm, q.seed,
                        spins=q.spins[None].copy(), instance_ids=[q.instance_id])
        a.set_schedule(t_meas=r.sweeps // 2)
        a.run(r.sweeps)
        oa = a.read_observables(hist=False)
        assert oa.accE[0, 0] == r.accE and oa.acc_d[0, 0] == r.acc_d and oa.n_meas[0] == r.n_meas
        a.close()
    srv.close()


@pytest.mark.gpu
def test_server_cancel_running_request(gpu):
    icmpt, ctx = gpu
    from paper_1501_05630_gb300.serve import Request, Server
    T = I.ladder(0.3, 1.5, 8)
    N, Nb = icmpt.lattice_size(I.SQUARE2D, 8)
    reqs = [Request(I.SQUARE2D, 8, I.PM_J, T, 1.0, 3, 400 + i, I.couplings(Nb, I.PM_J, 3, [400 + i])[0])
            for i in range(3)]
    srv = Server(slots_per_class=4, quantum=16, eps_e=0.0, eps_ql=0.0, need=50, max_sweeps=4096)
    tk = [srv.submit(r) for r in reqs]
    for _ in range(20):
        srv.step()
    srv.cancel(tk[1])
    srv.run_until_idle()
    res = [srv.poll(t) for t in tk]
    assert res[1].status == "cancelled" and 0 < res[1].sweeps < 4096
    assert res[0].status == res[2].status == "not_thermalized" and res[0].sweeps == res[2].sweeps == 4096
    assert srv.status() == (0, 0, 1)
    srv.close()


@pytest.mark.gpu
def test_invalid_couplings_are_refused(gpu):
    icmpt, ctx = gpu
    T = I.ladder(0.3, 2.0, 6)
    N, Nb = icmpt.lattice_size(I.CUBIC3D, 4)
    J = I.couplings(Nb, I.PM_J, 1, range(3))
    bad = J.copy()
    bad[1, 5] = 2                                            # not a +-J value
    with pytest.raises(icmpt.IcmError) as e:
        icmpt.Batch(ctx, I.CUBIC3D, 4, I.PM_J, bad, T, 1.0, 1)
    assert e.value.code == -1
    Jg = I.couplings(Nb, I.GAUSS, 1, range(2))
    Jg[0, 3] = np.nan
    with pytest.raises(icmpt.IcmError):
        icmpt.Batch(ctx, I.CUBIC3D, 4, I.GAUSS, Jg, T, 1.0, 1)
    b = icmpt.Batch(ctx, I.CUBIC3D, 4, I.PM_J, J, T, 1.0, 1)
    b.run(3)
    with pytest.raises(icmpt.IcmError):                      # the slot is refused and freed
        b.set_slot(2, bad[1], None, instance_id=9)
    b.run(3)                                                 # the other slots keep running
    assert list(b.read_sweeps()) == [6, 6, 3]
    with pytest.raises(icmpt.IcmError):
        b.load(couplings=bad)
    with pytest.raises(icmpt.IcmError) as e:                 # refused until valid couplings are loaded
        b.run(1)
    assert e.value.code == -6
    b.load(couplings=J)
    b.run(1)
    b.close()
