"""The three-standard-error test of statcheck on synthetic samples."""
import numpy as np
import statcheck
from scipy import stats


def test_one_component_is_the_three_standard_error_rule():
    rng = np.random.default_rng(1)
    x = rng.standard_normal(400)
    x -= x.mean()
    sd = x.std(ddof=1) / np.sqrt(len(x))
    t_crit = stats.t.isf(statcheck.P_3SIGMA / 2, len(x) - 1)      # about 3.0
    assert 2.9 < t_crit < 3.1
    assert statcheck.hotelling(x + 0.99 * t_crit * sd)["p"] > statcheck.P_3SIGMA
    assert statcheck.hotelling(x + 1.01 * t_crit * sd)["p"] < statcheck.P_3SIGMA


def test_false_alarm_rate_and_power():
    rng = np.random.default_rng(2)
    C = 0.6 ** np.abs(np.subtract.outer(np.arange(12), np.arange(12)))     # correlated components
    A = np.linalg.cholesky(C)
    p0 = [statcheck.hotelling(rng.standard_normal((200, 12)) @ A.T)["p"] for _ in range(400)]
    assert 0.02 < np.mean(np.array(p0) < 0.1) < 0.2                     # about 10% below 0.1
    shifted = rng.standard_normal((200, 12)) @ A.T + 0.4
    assert statcheck.hotelling(shifted)["p"] < 1e-6


def test_degenerate_components():
    rng = np.random.default_rng(3)
    x = rng.random((100, 4))
    x /= x.sum(1, keepdims=True)                                      # rows sum to one: rank 3
    d = x - x.mean(0)
    r = statcheck.hotelling(np.hstack([d, np.zeros((100, 2))]))       # zero columns are dropped
    assert r["K"] == 3 and r["p"] > 0.99
    assert statcheck.hotelling(np.hstack([d, np.full((100, 1), 1e-3)]))["p"] == 0.0   # constant offset


def test_pq_bins_symmetrise_and_normalise():
    h = np.zeros((2, 9))
    h[0, 0] = 10                     # n = 0: q = 1
    h[1, 4] = 3
    h[1, 8] = 1                      # n = 8: q = -1
    P = statcheck.pq_bins(h, 4)
    assert np.allclose(P.sum(1), 1.0)
    assert np.allclose(P[0], [0, 0, 0, 1]) and np.allclose(P[1], [0.75, 0, 0, 0.25])
