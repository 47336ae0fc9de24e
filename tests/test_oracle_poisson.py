"""Pins of the oracle's Poisson macro-event sampling and capping (Sec. II.D)."""
import numpy as np
from scipy import stats

from oracle.poisson import cap_lambda, poisson_count
from oracle.philox import philox4x32_10, uniform23


def test_inversion_matches_scipy_ppf():
    u = (np.arange(1, 2 ** 12) - 0.5) / 2 ** 12
    for lam in (1e-6, 1e-3, 0.1, 0.7, 1.0, 4.0, 17.3, 40.0, 64.0):
        k = poisson_count(u, np.full(u.shape, lam))
        ref = stats.poisson.ppf(u, lam)
        cdf = stats.poisson.cdf(ref, lam)
        safe = np.abs(cdf - u) > 1e-5     # not within binary32 reach of a CDF step
        assert np.array_equal(k[safe], ref[safe].astype(int)), lam


def test_zero_rate_gives_zero():
    assert np.all(poisson_count(np.array([1e-7, 0.5, 1 - 1e-7]), np.zeros(3)) == 0)


def test_pmf_chi_square():
    n = 200000
    ctr = np.zeros(((n + 3) // 4, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(len(ctr))
    u = uniform23(philox4x32_10(ctr, (3, 3)).reshape(-1)[:n])
    lam = 2.5
    k = poisson_count(u, np.full(n, lam))
    obs = np.bincount(k, minlength=12)[:12]
    exp = stats.poisson.pmf(np.arange(12), lam) * n
    obs = np.append(obs, n - obs.sum())
    exp = np.append(exp, n - exp.sum())
    assert stats.chisquare(obs, exp).pvalue > 1e-4
    assert abs(k.mean() - lam) < 5 * np.sqrt(lam / n)
    assert abs(k.var() - lam) < 0.05


def test_cap_and_rescale_is_unbiased():
    """E[K] w' = lambda_macro w_a (Sec. II.D.2)."""
    n = 100000
    ctr = np.zeros(((n + 3) // 4, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(len(ctr))
    u = uniform23(philox4x32_10(ctr, (9, 1)).reshape(-1)[:n])
    lam_macro = np.full(n, 7.5)
    lam_eff, fac, capped = cap_lambda(lam_macro, 0.5)
    assert np.all(capped) and np.all(lam_eff == 0.5) and np.allclose(fac, 15.0)
    k = poisson_count(u, lam_eff)
    w_a = 3.0
    assert abs((k * w_a * fac).mean() / (7.5 * w_a) - 1) < 0.02
    # hard ceiling of 64 always applies
    lam_eff, fac, capped = cap_lambda(np.array([100.0, 10.0]), 0.0)
    assert lam_eff[0] == 64.0 and capped[0] and not capped[1] and fac[1] == 1.0
