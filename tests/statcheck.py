"""Statistical agreement at the level of three standard errors.

Gaussian couplings give no bit-exact chain, so the tests compare averages:
the GPU against the oracle on the same instances (paired differences), or a
sampled average against an exact value.  A quantity measured at K
temperatures (or K bins) is one vector; testing each of its K components
at three standard errors would raise a false alarm with probability about
1 - (1 - 0.0027)^K, 6% at K = 24, and more over several observables.  So each
vector is tested once, by Hotelling's T^2 of its mean difference, at the
false-alarm probability of one three-standard-error test, 0.0027 (the
two-sided normal tail beyond 3).  For K = 1 this is the plain three-standard-
error rule (with Student's t in place of the normal).  Correlations between
the components (neighbouring temperatures of one parallel-tempering chain
are correlated) enter through the sample covariance, so no independence is
assumed.
"""
from __future__ import annotations

import math

import numpy as np

P_3SIGMA = math.erfc(3.0 / math.sqrt(2.0))      # 0.0026998: P(|z| > 3) of a standard normal


def hotelling(d, rel_eig: float = 1e-10):
    """Test of mean(d) = 0 for samples d [n][...] (flattened to [n][K]).

    Components that are zero in every sample carry no evidence and are
    dropped.  The covariance is taken on its principal subspace (eigenvalues
    above rel_eig times the largest), so linear dependencies (bins of a
    distribution summing to one) are handled; a mean along a direction
    without variance (a component constant but nonzero) is a deterministic
    difference and gives p = 0.
    Returns dict(p, T2, K, n, z) with z the per-component mean / standard error."""
    d = np.asarray(d, dtype=np.float64)
    n = d.shape[0]
    d = d.reshape(n, -1)
    mu = d.mean(0)
    sd = d.std(0, ddof=1) if n > 1 else np.zeros_like(mu)
    z = np.where(sd > 0, mu / np.maximum(sd, 1e-300) * math.sqrt(n), 0.0)
    keep = np.any(d != 0, axis=0)
    d, mu = d[:, keep], mu[keep]
    if d.shape[1] == 0:
        return dict(p=1.0, T2=0.0, K=0, n=n, z=z)
    S = np.cov(d, rowvar=False).reshape(d.shape[1], d.shape[1])
    w, V = np.linalg.eigh(S)
    sel = w > rel_eig * max(w.max(), 0.0)
    K = int(sel.sum())
    # a mean along a direction without variance is a deterministic difference
    perp = mu - V[:, sel] @ (V[:, sel].T @ mu)
    if K == 0 or np.linalg.norm(perp) > 1e-8 * (np.linalg.norm(mu) + math.sqrt(max(w.max(), 0.0))):
        return dict(p=0.0, T2=math.inf, K=max(K, 1), n=n, z=z)
    if K >= n:
        raise ValueError(f"{K} components need more than {n} samples")
    y = V[:, sel].T @ mu
    T2 = float(n * np.sum(y * y / w[sel]))
    from scipy.stats import f as fdist
    F = T2 * (n - K) / (K * (n - 1))
    return dict(p=float(fdist.sf(F, K, n - K)), T2=T2, K=K, n=n, z=z)


def agree(d, what: str = "") -> dict:
    """Assert that the samples d agree with mean 0 at the three-standard-error
    level (hotelling p >= P_3SIGMA); returns the test's figures."""
    r = hotelling(d)
    assert r["p"] >= P_3SIGMA, (what, "p", r["p"], "K", r["K"], "max |z|", float(np.max(np.abs(r["z"]))))
    return r


def pq_bins(hist, n_bins: int = 4):
    """Symmetrised overlap distribution of each sample, coarse-grained: hist
    [..][N + 1] counts of n = #(q_i = -1) per measurement -> [..][n_bins]
    probabilities of |q| = |1 - 2n/N| in equal bins of [0, 1]."""
    h = np.asarray(hist, dtype=np.float64)
    N = h.shape[-1] - 1
    P = h / np.maximum(h.sum(-1, keepdims=True), 1.0)
    P = 0.5 * (P + P[..., ::-1])
    aq = np.abs(1.0 - 2.0 * np.arange(N + 1) / N)
    idx = np.minimum((aq * n_bins).astype(int), n_bins - 1)
    out = np.zeros(h.shape[:-1] + (n_bins,))
    for b in range(n_bins):
        out[..., b] = P[..., idx == b].sum(-1)
    return out


def agree_distribution(P, target, m, what: str = "", min_expected: float = 5.0) -> dict:
    """Sampled distributions P [n][bins] (each row normalised over m[n]
    measurements) against the exact distribution target [bins].  Bins that
    the run is expected to visit at least min_expected times are tested
    together by hotelling on the per-sample differences; the rarely visited
    bins are pooled, and their total count must be a plausible Poisson count
    at the three-standard-error level (two-sided 0.0027): a chain cannot be
    asked to visit a state of probability 1e-8 in 10^5 measurements."""
    from scipy.stats import poisson
    P = np.asarray(P, dtype=np.float64)
    target = np.asarray(target, dtype=np.float64)
    m = np.broadcast_to(np.asarray(m, dtype=np.float64), P.shape[:1])
    M = float(m.sum())
    common = target * M >= min_expected
    r = agree(P[:, common] - target[common][None, :], what)
    lam = float(target[~common].sum() * M)
    c = int(round(float((P[:, ~common] * m[:, None]).sum())))
    lo = poisson.cdf(c, lam) if lam > 0 else 1.0
    hi = poisson.sf(c - 1, lam) if lam > 0 else (1.0 if c == 0 else 0.0)
    assert min(lo, hi) >= P_3SIGMA / 2, (what, "rare bins", c, lam)
    r.update(rare_count=c, rare_expected=lam)
    return r
