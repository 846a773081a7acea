"""Reduced-scale thermalization experiments (Fig. 2 / Fig. 3 of the paper).

CPU: the automated thermalization time of a Delta(t) curve.
GPU: Delta(t) of Eq. 2 from the library for +-J couplings equals the value
computed from the oracle's accumulators of the same windows (exact
integers), for plain PT, PT+ICM and HCA; with Gaussian couplings PT+ICM
drives Delta to zero within errors on a small lattice."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1501_05630_gb300 import inputs as I


def test_thermalization_time_rule():
    from paper_1501_05630_gb300.experiments import DeltaCurve, thermalization_time
    t = np.array([16, 32, 64, 128, 256])
    c = DeltaCurve("x", t, np.array([-0.5, -0.1, 0.01, -0.2, 0.0]), np.array([0.05] * 5))
    assert thermalization_time(c) == 256                      # a later excursion resets it
    c2 = DeltaCurve("x", t, np.array([-0.5, -0.09, 0.01, 0.02, 0.0]), np.array([0.05] * 5))
    assert thermalization_time(c2) == 32
    c3 = DeltaCurve("x", t, np.array([-0.5, -0.3, -0.2, -0.2, -0.2]), np.array([0.01] * 5))
    assert thermalization_time(c3) is None
    assert thermalization_time(c3, floor=0.25) == 64


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA GPU")
    from paper_1501_05630_gb300 import build, icmpt
    build.build()
    torch.cuda.set_device(0)
    ctx = icmpt.Context(0)
    yield icmpt, ctx
    ctx.close()


@pytest.mark.gpu
@pytest.mark.parametrize("method", ["pt", "icm", "hca"])
def test_delta_curve_equals_oracle_windows(env, method):
    icmpt, ctx = env
    from paper_1501_05630_gb300.experiments import delta_curve, method_schedule
    g = O.Geometry(O.SQUARE2D, 8)
    T = I.ladder(0.3, 1.6, 8)
    n, seed = 8, 123
    J = I.couplings(g.Nb, I.PM_J, seed, range(n))
    s0 = I.initial_spins(g.N, 16, seed, range(n))
    c = delta_curve(ctx, O.SQUARE2D, 8, I.PM_J, J, s0, T, 1.0, seed, method, 3, 7)
    ticm, every, two_a = method_schedule(method, 1.0)
    for w, t_end in enumerate(c.t):
        d = []
        for a in range(n):
            r = O.Instance(g, J[a].astype(np.float64), T, s0[a], pm=True, T_icm=ticm, seed=seed, inst=a,
                           icm_every=every, enable_2a=bool(two_a), t_meas=t_end // 2)
            r.run(int(t_end))
            m = r.n_meas[0]
            e = r.accE[0] / (2 * g.N * m)
            ql = 1 - 2 * r.acc_d[0] / (g.Nb * m)
            d.append(-(g.Nb / g.N) * (1 - ql) / T[0] - e)
        d = np.array(d)
        assert c.delta[w] == pytest.approx(d.mean(), rel=1e-12, abs=1e-12)
        assert c.se[w] == pytest.approx(d.std() / np.sqrt(n - 1), rel=1e-9, abs=1e-12)


@pytest.mark.gpu
def test_icm_drives_delta_to_zero_gaussian(env):
    icmpt, ctx = env
    from paper_1501_05630_gb300.experiments import delta_curve, thermalization_time
    N, Nb = icmpt.lattice_size(I.SQUARE2D, 8)
    T = I.ladder(0.3, 1.6, 16)
    n = 256
    J = I.couplings(Nb, I.GAUSS, 9, range(n))
    s0 = I.initial_spins(N, 32, 9, range(n))
    c = delta_curve(ctx, I.SQUARE2D, 8, I.GAUSS, J, s0, T, 2.0, 9, "icm", 4, 13)
    assert c.delta[0] < -3 * c.se[0]                          # far from equilibrium at first
    assert abs(c.delta[-1]) <= 3 * c.se[-1]                   # Eq. 1 holds at the end
    assert thermalization_time(c, nsig=3.0) is not None


@pytest.mark.gpu
def test_icm_frequency_judged_on_time_to_criterion(env):
    """The frequency tuner: each candidate's thermalization time is that of a
    Delta(t) curve run with that frequency (the runs are deterministic), its
    cost is that time times the measured time per sweep, and the choice is the
    cheapest candidate that thermalized."""
    icmpt, ctx = env
    from paper_1501_05630_gb300.experiments import delta_curve, icm_frequency, thermalization_time
    N, Nb = icmpt.lattice_size(I.SQUARE2D, 8)
    T = I.ladder(0.3, 1.6, 16)
    n = 128
    J = I.couplings(Nb, I.GAUSS, 19, range(n))
    s0 = I.initial_spins(N, 32, 19, range(n))
    best, rows = icm_frequency(ctx, I.SQUARE2D, 8, I.GAUSS, J, s0, T, 2.0, 19, candidates=(1, 4), log2_max=12,
                               timing_sweeps=128)
    assert [r.icm_every for r in rows] == [1, 4]
    for r in rows:
        c = delta_curve(ctx, I.SQUARE2D, 8, I.GAUSS, J, s0, T, 2.0, 19, "icm", 4, 12, icm_every=r.icm_every)
        assert thermalization_time(c, nsig=2.0) == r.t_therm
        assert r.ms_per_sweep > 0
        assert r.cost_ms is None if r.t_therm is None else r.cost_ms == pytest.approx(r.t_therm * r.ms_per_sweep)
    done = [r for r in rows if r.cost_ms is not None]
    assert best == (min(done, key=lambda r: r.cost_ms).icm_every if done else None)


@pytest.mark.gpu
@pytest.mark.parametrize("icm", [False, True])
def test_annealing_equals_oracle(env, icm):
    """+-J annealing with a changing temperature: spins and energies of the
    library equal the oracle's run with the same temperatures, bit for bit."""
    icmpt, ctx = env
    from paper_1501_05630_gb300.experiments import anneal
    g = O.Geometry(O.SQUARE2D, 8)
    n, seed, steps, sw = 6, 55, 12, 5
    J = I.couplings(g.Nb, I.PM_J, seed, range(n))
    s0 = I.initial_spins(g.N, 2, seed, range(n))
    b = anneal(ctx, O.SQUARE2D, 8, I.PM_J, J, s0, 3.0, 0.1, steps, sw, icm, seed)
    spins, E = b.read_spins(), b.read_energies()
    ts = 3.0 * (0.1 / 3.0) ** (np.arange(steps) / (steps - 1))
    for a in range(n):
        r = O.Instance(g, J[a].astype(np.float64), ts[:1].copy(), s0[a], pm=True, T_icm=1e300 if icm else 0.0,
                       seed=seed, inst=a, icm_every=1 if icm else 0, swap_every=0, t_meas=1 << 62)
        for T in ts:
            r.T[0] = T
            r.run(sw)
        assert np.array_equal(spins[a], r.s)
        assert np.array_equal(E[a], r.E)
    b.close()


# ----------------------------------------------------------------------------- Fig. 1
def test_crossing_temperature_interpolates():
    from paper_1501_05630_gb300.experiments import FractionCurve, crossing_temperature
    c = FractionCurve(np.array([0.5, 1.0, 1.5, 2.0]), np.array([0.1, 0.2, 0.4, 0.45]), np.zeros(4))
    assert crossing_temperature(c, 0.3) == pytest.approx(1.25)
    assert crossing_temperature(c, 0.05) == 0.5
    assert crossing_temperature(c, 0.5) is None


@pytest.mark.gpu
def test_cluster_fraction_equals_oracle_and_stays_below_2d_threshold():
    """p(T) of a +-J batch equals the oracle's per-instance averages (bit-exact
    sums); for 2D the fraction never reaches p_c = 0.592 (Fig. 1, top panel)
    and approaches 1/2 at high T."""
    import torch
    from oracle import oracle as O
    from paper_1501_05630_gb300 import build, icmpt
    from paper_1501_05630_gb300.experiments import cluster_fraction
    build.build()
    torch.cuda.set_device(0)
    ctx = icmpt.Context(0)
    T = I.ladder(0.3, 4.0, 8)
    g = O.Geometry(O.SQUARE2D, 8)
    n, sweeps, t_meas = 6, 600, 200
    J = I.couplings(g.Nb, I.PM_J, 12, range(n))
    s0 = I.initial_spins(g.N, 16, 12, range(n))
    c = cluster_fraction(ctx, O.SQUARE2D, 8, I.PM_J, J, s0, T, 1.0, 12, sweeps, t_meas)
    per = []
    for a in range(n):
        r = O.Instance(g, J[a].astype(np.float64), T, s0[a], pm=True, T_icm=1.0, seed=12, inst=a, t_meas=t_meas)
        r.run(sweeps)
        per.append(r.observables()["p"])
    assert np.allclose(c.p, np.mean(per, axis=0), rtol=0, atol=1e-12)
    assert np.all(c.p < 0.592) and c.p[-1] > 0.4
    ctx.close()
