"""Spectrum reconstruction and closed-form reference spectra (App. B).

Test infrastructure only (imported by tests/, smoke() and bench.py's CPU
baseline).

* H_k = sum over newly emitted axions in bin k of |q_i| E_i (App. B);
  the bin index is decided in binary32 like the kernels:
  k = floor(E * float32(nbins / E_max)).
* normalised spectrum H_k / sum_j H_j dE_j and absolute
  dQ/dE = H_k / (V t_tot dE_k) x (1 keV in erg) (Eq. absolute_spectrum).
* relative L2 = ||h - h_ref||_2 / ||h_ref||_2 over the bins (the paper does
  not define it; this is the reading).
* closed forms used as references: Primakoff on a Planck photon bath,
  dQ/dE = E (P(E)/dt) dn_gamma/dE with dn_gamma/dE = E^2/(pi^2 (hbar c)^3 (e^x-1));
  Compton-like Q_C x^5/(e^x-1)/(T Gamma(6) zeta(6)); bremsstrahlung
  Q_B x^a e^-x/(T Gamma(a+1)).
"""
import math

import numpy as np
from scipy import special

from . import constants as K
from .plasma import CellState, Params, primakoff_F


def bin_index(E_keV, nbins, E_max_keV):
    E32 = np.asarray(E_keV, dtype=np.float64).astype(np.float32)
    inv = np.float32(nbins / E_max_keV)
    k = np.floor((E32 * inv).astype(np.float32)).astype(np.int64)
    return k


def histogram(E_keV, w, nbins, E_max_keV):
    """H_k = sum w E over bins k in [0, nbins); energies beyond E_max are dropped."""
    k = bin_index(E_keV, nbins, E_max_keV)
    ok = (k >= 0) & (k < nbins)
    return np.bincount(k[ok], weights=(np.asarray(w) * np.asarray(E_keV))[ok], minlength=nbins)


def normalised(H, dE):
    return H / np.sum(H * dE)


def absolute_dQdE(H, volume_cm3, t_tot_s, dE_keV):
    """erg cm^-3 s^-1 keV^-1."""
    return H * K.KEV_ERG / (volume_cm3 * t_tot_s * dE_keV)


def rel_l2(h, h_ref):
    return float(np.linalg.norm(np.asarray(h) - np.asarray(h_ref)) / np.linalg.norm(h_ref))


def photon_density_per_keV(T_keV, E_keV):
    E = np.asarray(E_keV, dtype=np.float64)
    return E ** 2 / (math.pi ** 2 * K.HBARC_KEV_CM ** 3) / np.expm1(E / T_keV)


def primakoff_dQdE(cs: CellState, p: Params, E_keV):
    """Primakoff on a Planck bath with P = 1 - exp(-Gamma dt) per step."""
    E = np.asarray(E_keV, dtype=np.float64)
    s = 4.0 * E ** 2 / cs.kappa_keV ** 2
    P = -np.expm1(-cs.Gamma0_P * primakoff_F(s) * p.dt_phys_s)
    return E * K.KEV_ERG * (P / p.dt_phys_s) * photon_density_per_keV(cs.T_keV, E)


def compton_dQdE(cs: CellState, E_keV):
    x = np.asarray(E_keV, dtype=np.float64) / cs.T_keV
    return cs.Q_C * x ** 5 / np.expm1(x) / (cs.T_keV * math.gamma(6.0) * special.zeta(6.0))


def brems_dQdE(cs: CellState, a, E_keV):
    x = np.asarray(E_keV, dtype=np.float64) / cs.T_keV
    return cs.Q_B * np.exp(a * np.log(x) - x - special.gammaln(a + 1.0)) / cs.T_keV


def bin_average(fn, edges, sub=64):
    """Average of fn over each bin (Gauss-Legendre, `sub` nodes per bin)."""
    xg, wg = np.polynomial.legendre.leggauss(sub)
    lo, hi = edges[:-1], edges[1:]
    mid = 0.5 * (lo + hi)
    half = 0.5 * (hi - lo)
    pts = mid[:, None] + half[:, None] * xg[None, :]
    return np.sum(fn(pts) * wg[None, :], axis=1) / 2.0
