"""Pins for the oracle's lognormal transform and Poisson sampling
(section 3.1, eqs. (Lncov) and (sampling); CPU only).

* inverse CDF against scipy.stats.poisson.ppf (independent library), including
  the large-intensity path that starts at the mode;
* the decision margin: moving mu by more than the margin flips the count,
  by less does not;
* closed forms: E[1+delta] = 1, Var delta = e^{sigma^2} - 1,
  E[n] = nbar f, Var n = nbar f + (nbar f)^2 (e^{sigma^2} - 1);
* the paper's counts-in-cells mixture prediction (section 3.4) by
  Gauss-Hermite quadrature, with the paper's own parameters
  (sigma_A^2 = 0.13, nbar = 9.68, N = 0..41) and a survey mask.
"""
import math

import numpy as np
import pytest
from scipy import stats

from paper_1406_6072_gb300 import workloads as W


def test_icdf_matches_scipy(orc):
    rng = np.random.default_rng(3)
    mus = np.concatenate([[1e-6, 0.01, 0.5, 1, 2, 9.68, 40, 150, 699.9],
                          rng.uniform(0, 30, 60), [701, 800, 2500]])
    checked = 0
    for mu in mus:
        for U in np.concatenate([rng.random(40), [0.0, 1e-300, 0.5, 1 - 2**-53]]):
            n, _ = orc.poisson_icdf(U, mu)
            ref = stats.poisson.ppf(U, mu)
            # skip U sitting on a CDF step to binary64 resolution
            cdf_n = stats.poisson.cdf(n, mu)
            cdf_nm1 = stats.poisson.cdf(n - 1, mu) if n > 0 else 0.0
            if min(abs(cdf_n - U), abs(U - cdf_nm1)) < 1e-9:
                continue
            assert n == ref, (mu, U, n, ref)
            checked += 1
    assert checked > 2800


def test_icdf_zero_intensity(orc):
    for U in (0.0, 0.3, 1 - 2**-53):
        assert orc.poisson_icdf(U, 0.0)[0] == 0
        assert orc.poisson_icdf(U, -1.0)[0] == 0


def test_icdf_large_intensity(orc):
    """Up to 1e9 the walk from the mode still matches scipy; from 1e9 on (and
    for an infinite intensity, an overflowing exp) the count saturates at the
    int32 maximum instead of walking billions of terms."""
    for mu in (2e5, 3e7, 9.9e8):
        for U in (0.01, 0.5, 0.97):
            n, _ = orc.poisson_icdf(U, mu)
            assert abs(n - stats.poisson.ppf(U, mu)) <= 1, (mu, U, n)
    for mu in (1e9, 1e12, np.inf):
        assert orc.poisson_icdf(0.5, mu)[0] == 2**31 - 1


def test_margin_flips_decision(orc):
    rng = np.random.default_rng(4)
    for _ in range(400):
        mu = rng.uniform(0.05, 50)
        U = rng.random()
        n, m = orc.poisson_icdf(U, mu)
        if m > 0.2:
            continue
        lo = orc.poisson_icdf(U, mu * (1 - 0.5 * m))[0]
        hi = orc.poisson_icdf(U, mu * (1 + 0.5 * m))[0]
        assert lo == n and hi == n
        flip_lo = orc.poisson_icdf(U, mu * (1 - 2.0 * m))[0]
        flip_hi = orc.poisson_icdf(U, mu * (1 + 2.0 * m))[0]
        assert flip_lo != n or flip_hi != n


def test_lognormal_and_poisson_moments(orc):
    sigma2, nbar = 0.8, 2.0
    G = W.gaussian_field_values((8, 20000), seed=5, scale=math.sqrt(sigma2))
    f = np.full(20000, 0.75)
    delta, counts, _ = orc.lognormal_poisson(G, sigma2, nbar, f=f, seed=6, field0=10)
    n = delta.size
    var_d = math.exp(sigma2) - 1
    assert abs(delta.mean()) < 5 * math.sqrt(var_d / n)
    assert abs(delta.var() / var_d - 1) < 0.06  # heavy tail: loose band
    lam = nbar * 0.75
    mean_n = lam
    var_n = lam + lam**2 * var_d
    assert abs(counts.mean() - mean_n) < 5 * math.sqrt(var_n / n)
    assert abs(counts.var() / var_n - 1) < 0.06
    assert np.allclose(delta, np.exp(G - sigma2 / 2) - 1, rtol=1e-14, atol=1e-15)


def test_field_offsets_are_consistent(orc):
    G = W.gaussian_field_values((6, 50), seed=7)
    _, all_counts, _ = orc.lognormal_poisson(G, 1.0, 3.0, seed=8, field0=4)
    _, part, _ = orc.lognormal_poisson(G[3:], 1.0, 3.0, seed=8, field0=7)
    assert np.array_equal(all_counts[3:], part)
    _, other, _ = orc.lognormal_poisson(G, 1.0, 3.0, seed=9, field0=4)
    assert not np.array_equal(all_counts, other)


def test_masked_cells_have_zero_counts(orc):
    G = W.gaussian_field_values((2, 400), seed=10)
    f = W.survey_mask((20, 20), seed=11).ravel()
    _, counts, _ = orc.lognormal_poisson(G, 1.0, 5.0, f=f, seed=12)
    assert np.all(counts[:, f == 0] == 0)
    assert counts[:, f > 0].sum() > 0


def test_counts_in_cells_mixture_prediction(orc):
    """Section 3.4: <P(N)> = int dA N(A; -s^2/2, s^2) e^{NA}/N! sum_i nbar_i^N
    e^{-nbar_i e^A} over unmasked cells, with the paper's parameter values."""
    sigma2, nbar = 0.13, 9.68
    shape = (128, 128)
    f = W.survey_mask(shape, seed=13).ravel().astype(np.float64)
    nb = nbar * f[f > 0]
    R = 40
    G = W.gaussian_field_values((R, f.size), seed=14, scale=math.sqrt(sigma2))
    _, counts, _ = orc.lognormal_poisson(G, sigma2, nbar, f=f, seed=15)
    hist = np.stack([np.bincount(c[f > 0], minlength=60)[:42] for c in counts])
    pred = orc.cic_prediction(sigma2, nbar, f, 42)
    assert np.array_equal(orc.cic_histogram(counts, f, 42), hist)
    mean_hist = hist.mean(0)
    assert pred.sum() == pytest.approx(nb.size, rel=1e-3)  # all mass within N <= 41
    sig = np.sqrt(np.maximum(pred, 1.0) / R)
    z = (mean_hist - pred) / sig
    assert np.max(np.abs(z)) < 6.0, z


def test_log1p_input_gives_the_density_correlation(orc):
    """Section 3.1, eq. (Lncov): a Gaussian field whose covariance is
    ln(1 + xi_delta) gives delta = exp(G - sigma^2/2) - 1 with correlation
    function xi_delta (E[e^{G_i + G_j}] = e^{sigma^2 + c_ij}).  Checked on
    sampled fields against the input xi_delta, at several lags."""
    n = (8, 8)
    amp, scale = 0.6, 2.0
    e = orc.embed(list(n), W.XI_EXPONENTIAL, amp, scale, log1p=True)
    assert e["report"]["n_negative"] == 0
    c = e["c"]
    assert c[0, 0] == pytest.approx(math.log1p(amp), rel=1e-15)
    assert c[0, 3] == pytest.approx(math.log1p(amp * math.exp(-3 / scale)), rel=1e-14)
    R = 30000
    G = orc.sample(n, e["sqrt_lambda"], 21, 0, R, 0).reshape(2 * R, n[0], n[1])
    sigma2 = math.log1p(amp)
    delta = np.exp(G - sigma2 / 2) - 1
    for lag in [(0, 0), (0, 1), (1, 1), (0, 3), (2, 3)]:
        a = delta[:, : n[0] - lag[0], : n[1] - lag[1]]
        b = delta[:, lag[0]:, lag[1]:]
        prod = (a * b).reshape(2 * R, -1).mean(1)  # one value per field (cells correlated)
        est = prod.mean()
        err = prod.std() / math.sqrt(prod.size)
        expect = amp * math.exp(-math.hypot(*lag) / scale)
        assert abs(est - expect) < 5 * err, (lag, est, expect, err)


def test_cic_prediction_small_variance_limit(orc):
    """sigma_A^2 -> 0: the mixture reduces to a sum of Poisson laws with the
    cells' own intensities (scipy.stats.poisson)."""
    f = W.survey_mask((16, 16), seed=30).ravel()
    nbar = 3.5
    pred = orc.cic_prediction(1e-10, nbar, f, 30)
    nb = nbar * f[f > 0]
    direct = stats.poisson.pmf(np.arange(30)[:, None], nb[None, :]).sum(1)
    assert np.allclose(pred, direct, rtol=1e-6, atol=1e-12)
    big = orc.cic_prediction(0.3, nbar, f, 60)
    assert big.sum() == pytest.approx((f > 0).sum(), rel=1e-6)  # probability of all N


def test_cic_histogram_brute_force(orc):
    rng = np.random.default_rng(31)
    counts = rng.integers(0, 9, size=(3, 40))
    f = rng.choice([0.0, 0.5, 1.0], size=40)
    h = orc.cic_histogram(counts, f, 6)
    for r in range(3):
        for N in range(6):
            assert h[r, N] == sum(1 for i in range(40) if f[i] != 0 and counts[r, i] == N)


def test_astar_matches_lambert_w(orc):
    """Eq. (As) in closed form: A* = c - W(k e^c), c = s^2 (N - 1/2),
    k = nbar f s^2 (scipy's Lambert W), and A* -> ln(N / nbar) for large N."""
    from scipy.special import lambertw
    s2, nbar = 0.13, 9.68
    f = np.array([1.0, 0.7, 0.0, 0.25])
    N = np.arange(0, 60)[:, None] * np.ones((1, 4), dtype=int)
    a = orc.astar(N, f, nbar, s2)
    c = s2 * (N - 0.5)
    k = nbar * f * s2
    with np.errstate(divide="ignore"):
        ref = np.where(f > 0, c - np.real(lambertw(k * np.exp(c))), 0.0)
    assert np.max(np.abs(a - ref)) < 1e-12
    big = orc.astar(np.array([[4000]]), None, nbar, s2)[0, 0]
    assert abs(big - math.log(4000 / nbar)) < 0.02
