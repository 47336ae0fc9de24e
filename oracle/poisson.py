"""Poisson macro-event counts with Poisson-mean capping (Sec. II.D.1-II.D.2).

Test infrastructure only (imported by tests/, smoke() and bench.py's CPU
baseline).

lambda_eff = min(lambda_macro, lambda_cap) (Eq. lambda_eff) and
w' = w lambda_macro/lambda_eff (Eq. wa_rescaled). K ~ Poisson(lambda_eff)
(Eq. poisson_macro) is drawn by sequential-search inversion of one uniform:
K = min{k : u <= sum_{j<=k} e^-lambda lambda^j / j!}. The paper names no
sampling algorithm; this is the reading both sides implement.

The integer K is decided by floating point, so it is decided in binary32, the
precision of the CUDA kernels: lambda is rounded to binary32 and the running
pmf and CDF are binary32, p_k = p_{k-1} * (lambda / k), F_k = F_{k-1} + p_k.

Pinned by: scipy's Poisson CDF on a grid of (u, lambda) and a chi-square test
of sampled counts against the pmf.
"""
import numpy as np

from . import constants as K


def cap_lambda(lam_macro, lambda_cap):
    """Return (lambda_eff, weight factor lambda_macro/lambda_eff, capped flag)."""
    lam = np.asarray(lam_macro, dtype=np.float64)
    cap = K.LAMBDA_HARD_CAP
    if lambda_cap > 0:
        cap = min(cap, lambda_cap)
    capped = lam > cap
    lam_eff = np.where(capped, cap, lam)
    factor = np.where(capped, lam / np.where(capped, cap, 1.0), 1.0)
    return lam_eff, factor, capped


def poisson_count(u, lam_eff):
    """K = min{k: u <= F_k}, decided in binary32; u in (0,1) exact in binary32."""
    u32 = np.asarray(u, dtype=np.float64).astype(np.float32)
    lam32 = np.asarray(lam_eff, dtype=np.float64).astype(np.float32)
    p = np.exp(-lam32).astype(np.float32)
    F = p.copy()
    k = np.zeros(u32.shape, dtype=np.int64)
    active = u32 > F
    for kk in range(1, K.POISSON_KMAX + 1):
        if not np.any(active):
            break
        step = (lam32 / np.float32(kk)).astype(np.float32)
        p = np.where(active, (p * step).astype(np.float32), p)
        F = np.where(active, (F + p).astype(np.float32), F)
        k = np.where(active, kk, k)
        active = active & (u32 > F) & (p > np.float32(0.0))
    return k
