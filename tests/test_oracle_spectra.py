"""Pins of the oracle's energy-sampling kernels (Sec. II.G, II.H, App. B)."""
import math
import os

import numpy as np
from scipy import integrate, optimize, special, stats

from oracle import spectra
from oracle.philox import philox4x32_10, uniform23

TABLE2 = os.path.join(os.path.dirname(__file__), "golden", "table2.txt")


def table2():
    out = []
    for line in open(TABLE2):
        if line.startswith("#") or not line.strip():
            continue
        t = line.split()
        out.append(dict(process=t[0], T=float(t[1]), Epk_pic=float(t[2]), Epk_R=float(t[4]),
                        Q_pic=float(t[6]), Q_R=float(t[7])))
    return out


def _uniforms(n, seed=11):
    ctr = np.zeros(((n + 3) // 4, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(len(ctr))
    return uniform23(philox4x32_10(ctr, (seed, 0)).reshape(-1)[:n])


def test_bose_integral_against_quadrature():
    for n in (2, 4):
        for x in (1e-3, 0.2, 0.99, 1.0, 1.7, 6.0, 25.0):
            ref = integrate.quad(lambda t: t ** n / math.expm1(t), 0, x, epsabs=0, epsrel=1e-13)[0]
            got = spectra.bose_integral_lower(n, np.array([x]))[0]
            assert abs(got - ref) <= 1e-11 * ref


def test_compton_mean_closed_form():
    # <x> = 5 zeta(6)/zeta(5) for the number pdf x^4/(e^x-1)
    closed = 5 * special.zeta(6) / special.zeta(5)
    assert abs(closed - 4.905564) < 1e-6
    num = integrate.quad(lambda t: t ** 5 * math.exp(-t) / -math.expm1(-t), 0, 200)[0]
    den = integrate.quad(lambda t: t ** 4 * math.exp(-t) / -math.expm1(-t), 0, 200)[0]
    assert abs(num / den - closed) < 1e-9
    assert abs(spectra.compton_mean_x() - closed) < 1e-12
    u = (np.arange(4000) + 0.5) / 4000
    assert abs(spectra.compton_icdf(u).mean() - closed) < 2e-3


def test_icdf_inverts_cdf_and_ks():
    u = _uniforms(3000)
    x = spectra.compton_icdf(u)
    assert np.max(np.abs(spectra.compton_cdf(x) - u)) < 1e-12
    # the CDF itself is pinned against quadrature above
    assert stats.kstest(x, spectra.compton_cdf).pvalue > 1e-3
    xp = spectra.planck_icdf(u)
    assert stats.kstest(xp, lambda t: spectra.bose_cdf(2, t)).pvalue > 1e-3
    # Planck mean 3 zeta(4)/zeta(3)
    us = (np.arange(4000) + 0.5) / 4000
    assert abs(spectra.planck_icdf(us).mean() - 3 * special.zeta(4) / special.zeta(3)) < 2e-3


def test_gamma_kernels():
    a = 1.70
    xs = np.array([0.01, 0.5, 1.7, 4.0, 12.0])
    for x in xs:
        ref = integrate.quad(lambda t: t ** (a - 1) * math.exp(-t), 0, x)[0] / math.gamma(a)
        assert abs(spectra.gamma_cdf(a, x) - ref) < 1e-10
    u = (np.arange(4000) + 0.5) / 4000
    assert abs(spectra.brems_icdf(a, u).mean() - a) < 2e-3
    assert abs(spectra.mb_axion_icdf(u).mean() - 3.0) < 2e-3


def test_brems_power_peak_matches_table2():
    """The bremsstrahlung sampler's power spectrum x * pdf(x) peaks at x = a;
    Table II puts the peak at E_pk/T = 1.723, 1.680, 1.694."""
    a = 1.70
    res = optimize.minimize_scalar(lambda x: -x * spectra.brems_pdf(a, x), bounds=(0.1, 10),
                                   method="bounded", options={"xatol": 1e-10})
    for row in table2():
        if row["process"] != "brems":
            continue
        assert abs(res.x * row["T"] / row["Epk_R"] - 1.0) < 0.025


def test_compton_power_peak_bound():
    """The Compton power kernel E^5/(e^x-1) peaks at x = 4.965 (Wien-type root
    of 5(1-e^-x) = x)."""
    root = optimize.brentq(lambda x: 5 * (1 - math.exp(-x)) - x, 1, 10)
    res = optimize.minimize_scalar(lambda x: -x * spectra.compton_pdf(x), bounds=(1, 10),
                                   method="bounded", options={"xatol": 1e-10})
    assert abs(res.x - root) < 1e-6
    assert abs(root - 4.965114) < 1e-5
