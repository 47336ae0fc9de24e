"""Energy-sampling kernels of the thermal-bath channels and of the initial
particle populations, as functions of x = E/T.

Test infrastructure only (imported by tests/, smoke() and bench.py's CPU
baseline).

* Compton-like (Sec. II.G, Eq. compton_kernel): the power spectrum is
  proportional to E^5/(exp(E/T)-1), so the number pdf is x^4/(e^x-1)/(Gamma(5) zeta(5)).
* Bremsstrahlung (Sec. II.H): x = E/T is drawn from a Gamma(a) law, pdf
  x^(a-1) e^-x / Gamma(a), whose power spectrum x^a e^-x peaks at x = a.
* Planck photon bath at T_e (Sec. II.G, "local blackbody"): number pdf
  x^2/(e^x-1)/(2 zeta(3)).
* Maxwell-Boltzmann equilibrium axions (Sec. II.I, MB target): number pdf
  x^2 e^-x / 2, i.e. Gamma(3).

Inverse CDFs are exact to ~1e-13: Bose-type integrals are summed from two
convergent expansions (Bernoulli series below x = 1, an exponential series of
incomplete gamma functions above), then inverted by bisection; the Gamma laws
use scipy's regularized incomplete gamma and its inverse.

Pinned by: KS tests of sampled x against these CDFs, the closed-form means
5 zeta(6)/zeta(5) and a, scipy quadrature of the pdfs, and Table II's
bremsstrahlung peak energies E_pk/T = 1.723, 1.680, 1.694.
"""
import math
import numpy as np
from scipy import special

_BERN_TERMS = 24
_BERN = special.bernoulli(_BERN_TERMS)


def bose_integral_lower(n, x):
    """I_n(x) = integral_0^x t^n/(e^t-1) dt for integer n >= 1, vectorised."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    small = x < 1.0
    if np.any(small):
        xs = x[small]
        # t^n/(e^t-1) = t^(n-1) * sum_m B_m t^m / m!  (|t| < 2 pi)
        acc = np.zeros_like(xs)
        for m in range(_BERN_TERMS):
            bm = _BERN[m]
            if bm == 0.0:
                continue
            acc += bm / math.factorial(m) * xs ** (n + m) / (n + m)
        out[small] = acc
    big = ~small
    if np.any(big):
        xb = x[big]
        total = math.factorial(n) * special.zeta(n + 1.0)
        # integral_x^inf t^n e^{-k t} dt = n! k^-(n+1) Q(n+1, k x); terms with
        # k x > 80 are below 1e-28 of the total and are not summed
        kmax = int(min(400, math.ceil(80.0 / float(np.min(xb))) + 1))
        k = np.arange(1, kmax + 1, dtype=np.float64)
        q = special.gammaincc(n + 1.0, xb[:, None] * k[None, :])
        tail = math.factorial(n) * (q @ k ** (-(n + 1.0)))
        out[big] = total - tail
    return out


def bose_cdf(n, x):
    """CDF of the number pdf x^n/(e^x-1) normalised by n! zeta(n+1)."""
    return bose_integral_lower(n, x) / (math.factorial(n) * special.zeta(n + 1.0))


def bose_pdf(n, x):
    x = np.asarray(x, dtype=np.float64)
    return x ** n / np.expm1(x) / (math.factorial(n) * special.zeta(n + 1.0))


def bose_icdf(n, u):
    """Inverse of bose_cdf by bisection on log x (60 halvings of [1e-8, 80])."""
    u = np.asarray(u, dtype=np.float64)
    lo = np.full(u.shape, math.log(1e-8))
    hi = np.full(u.shape, math.log(80.0))
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        c = bose_cdf(n, np.exp(mid))
        below = c < u
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    return np.exp(0.5 * (lo + hi))


def bose_mean_x(n):
    """Mean of x under x^n/(e^x-1): (n+1)! zeta(n+2) / (n! zeta(n+1))."""
    return (n + 1) * special.zeta(n + 2.0) / special.zeta(n + 1.0)


# Compton-like: number pdf x^4/(e^x-1)
COMPTON_N = 4
# Planck photons: number pdf x^2/(e^x-1)
PLANCK_N = 2


def compton_pdf(x):
    return bose_pdf(COMPTON_N, x)


def compton_cdf(x):
    return bose_cdf(COMPTON_N, x)


def compton_icdf(u):
    return bose_icdf(COMPTON_N, u)


def compton_mean_x():
    return bose_mean_x(COMPTON_N)


def planck_icdf(u):
    return bose_icdf(PLANCK_N, u)


def gamma_pdf(a, x):
    x = np.asarray(x, dtype=np.float64)
    return np.exp((a - 1.0) * np.log(x) - x - special.gammaln(a))


def gamma_cdf(a, x):
    return special.gammainc(a, np.asarray(x, dtype=np.float64))


def gamma_icdf(a, u):
    return special.gammaincinv(a, np.asarray(u, dtype=np.float64))


def brems_pdf(a, x):
    return gamma_pdf(a, x)


def brems_icdf(a, u):
    return gamma_icdf(a, u)


def mb_axion_icdf(u):
    """Equilibrium MB axions: x ~ Gamma(3)."""
    return gamma_icdf(3.0, u)
