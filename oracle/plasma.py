"""Local plasma state and per-particle rates (Sec. II.E-II.I of the paper).

Test infrastructure only (imported by tests/, smoke() and bench.py's CPU
baseline). Everything here is plain FP64 and follows the paper's equations in
the paper's order:

* Eq. rho_def, qn_def: rho = sum n_i A_i m_u, n_e = sum Z_i n_i; X_H is the
  mass fraction carried by Z = 1 species.
* Eq. kappa_debye: kappa^2 = 4 pi alpha n_eff / T_e, n_eff = n_e + sum Z_i^2 n_i
  (natural units, densities converted with (hbar c)^3), or a fixed kappa.
* Eqs. prim_xs, prim_F, prim_rate, prim_prob: sigma = alpha g^2 Z^2 F(s)(hbar c)^2/8,
  s = 4 omega^2/kappa^2, F(s) = (1+1/s) ln(1+s) - 1, Gamma = n_t sigma c with
  n_t Z^2 -> sum_i Z_i^2 n_i (ions), P = 1 - exp(-Gamma dt).
* Eqs. epsC, QC, GammaC: eps_C = 2.67e-2 (1+X_H) T7^6 (alpha_ae/1.6e-23) erg/g/s,
  Q_C = rho eps_C, Gamma_C = Q_C/(n_e <E>).
* Eqs. eps_eZ, eps_ee: 0.150 T7^2.5 rho2 (1+X_H)(alpha_ae/1.6e-23)[1-0.0698 eta]
  and the same times (1+X_H)/(2 sqrt 2) with [1-0.140 eta], eta = (3+X_H) rho2/T7^2;
  Gamma_B = rho (eps_eZ+eps_ee)/(n_e <E>).
* Eq. gamma_abs: Gamma_abs(E) = (d ndot/dE) / (d n_eq/dE), MB or BE target.

Readings where the paper is silent: <E> is the number mean of the channel's sampling kernel; the fit brackets
[1-0.0698 eta] and [1-0.140 eta] are clamped at zero; Primakoff targets are
the ions (option: all charges, n_eff).

Pins: the 'all'-targets Primakoff rate equals Raffelt's g^2 T kappa^2 F/(32 pi);
F(s) equals an angular quadrature of the screened Coulomb kernel; Table II's
Compton Q^R within 3 percent. The absolute bremsstrahlung emissivity is
parity unpinned (Table II's bremsstrahlung Q^R cannot be reproduced from the
printed fit); its spectral shape is pinned by Table II's peak energies.
"""
import math
from dataclasses import dataclass, field

import numpy as np

from . import constants as K
from . import spectra


@dataclass
class Params:
    """Operator options (Sec. II.D, II.E, II.I, II.J)."""
    g_agg_GeV_inv: float = 1e-10
    g_ae: float = 1e-13
    dt_phys_s: float = 1.0
    w_a: float = 1.0
    w_gamma_ref: float = 0.0          # <= 0: use w_a
    lambda_cap: float = 0.0           # <= 0: off (the hard ceiling still applies)
    kappa_mode: int = 0               # 0 Debye, 1 fixed
    kappa_fixed_keV: float = 0.0
    prim_targets: int = 0             # 0 ions, 1 all charges (n_eff)
    prim_inverse_mult: float = 1.0
    eq_stats: int = 0                 # 0 MB, 1 BE
    brems_ee: int = 1
    absorb_mode: int = 0              # 0 Bernoulli deletion, 1 weight reduction
    brems_gamma_shape: float = 1.70
    relax_r: float = 0.1
    T_floor_keV: float = 0.0
    T_ceil_keV: float = 1e30
    T_mode: int = 0                   # 0 fixed, 1 prescribed field, 2 evolved
    seed: int = 0
    axion_mass_keV: float = 0.0       # m_a c^2 (Sec. II.B); 0: massless

    @property
    def w_gref(self):
        return self.w_gamma_ref if self.w_gamma_ref > 0 else self.w_a


@dataclass
class CellState:
    T_keV: float
    rho: float
    X_H: float
    n_e: float
    n_eff: float
    S_Z: float            # Primakoff target sum (ions: sum Z^2 n; all: n_eff)
    kappa_keV: float
    T7: float
    rho2: float
    eta: float
    eps_C: float
    eps_eZ: float
    eps_ee: float
    Q_C: float
    Q_B: float
    Gamma_C: float        # per electron [1/s]
    Gamma_B: float
    Gamma0_P: float       # Primakoff rate without F(s) [1/s]
    extra: dict = field(default_factory=dict)


def primakoff_F(s):
    """F(s) = (1 + 1/s) ln(1+s) - 1 (Eq. prim_F); power series below s = 1e-3."""
    s = np.asarray(s, dtype=np.float64)
    out = np.empty_like(s)
    small = s < 1e-3
    ss = s[small]
    # (1+1/s) ln(1+s) - 1 = sum_{n>=1} (-1)^(n+1) s^n / (n (n+1))
    acc = np.zeros_like(ss)
    for n in range(1, 9):
        acc += (-1.0) ** (n + 1) * ss ** n / (n * (n + 1))
    out[small] = acc
    sb = s[~small]
    out[~small] = (1.0 + 1.0 / sb) * np.log1p(sb) - 1.0
    return out


def cell_state(T_keV, n_ion, Z, A, p: Params) -> CellState:
    """Cell parameters from the temperature and ion densities (cm^-3)."""
    n_ion = np.asarray(n_ion, dtype=np.float64)
    Z = np.asarray(Z, dtype=np.float64)
    A = np.asarray(A, dtype=np.float64)
    rho = float(np.sum(n_ion * A) * K.M_U_G)
    n_e = float(np.sum(Z * n_ion))
    zsq = float(np.sum(Z * Z * n_ion))
    n_eff = n_e + zsq
    m_H = float(np.sum(np.where(Z == 1.0, n_ion * A, 0.0)) * K.M_U_G)
    X_H = m_H / rho if rho > 0 else 0.0
    if p.kappa_mode == 0:
        kappa2 = K.FOUR_PI * K.ALPHA_EM * n_eff * K.HBARC_KEV_CM ** 3 / T_keV
        kappa = math.sqrt(kappa2)
    else:
        kappa = p.kappa_fixed_keV
    S_Z = zsq if p.prim_targets == 0 else n_eff
    T7 = T_keV / (K.K_B_KEV_PER_K * 1e7)
    rho2 = rho / 100.0
    eta = (3.0 + X_H) * rho2 / T7 ** 2
    alpha_ae = p.g_ae ** 2 / K.FOUR_PI
    afac = alpha_ae / 1.60e-23
    eps_C = 2.67e-2 * (1.0 + X_H) * T7 ** 6 * afac
    eps_eZ = 0.150 * T7 ** 2.5 * rho2 * (1.0 + X_H) * afac * max(0.0, 1.0 - 6.98e-2 * eta)
    eps_ee = 0.0
    if p.brems_ee:
        eps_ee = (0.150 * T7 ** 2.5 * rho2 * (1.0 + X_H) * (1.0 + X_H) / (2.0 * math.sqrt(2.0))
                  * afac * max(0.0, 1.0 - 0.140 * eta))
    Q_C = rho * eps_C
    Q_B = rho * (eps_eZ + eps_ee)
    mean_E_C = spectra.compton_mean_x() * T_keV * K.KEV_ERG       # erg
    mean_E_B = p.brems_gamma_shape * T_keV * K.KEV_ERG              # Gamma(a) mean = a
    Gamma_C = Q_C / (n_e * mean_E_C) if n_e > 0 else 0.0
    Gamma_B = Q_B / (n_e * mean_E_B) if n_e > 0 else 0.0
    g_cm = p.g_agg_GeV_inv * K.HBARC_GEV_CM
    Gamma0_P = K.ALPHA_EM * g_cm ** 2 / 8.0 * S_Z * K.C_CM_S
    return CellState(T_keV=T_keV, rho=rho, X_H=X_H, n_e=n_e, n_eff=n_eff, S_Z=S_Z,
                     kappa_keV=kappa, T7=T7, rho2=rho2, eta=eta, eps_C=eps_C,
                     eps_eZ=eps_eZ, eps_ee=eps_ee, Q_C=Q_C, Q_B=Q_B,
                     Gamma_C=Gamma_C, Gamma_B=Gamma_B, Gamma0_P=Gamma0_P)


def primakoff_rate(cs: CellState, omega_keV):
    """Gamma_{gamma->a}(omega) [1/s] (Eqs. prim_xs, prim_rate)."""
    omega = np.asarray(omega_keV, dtype=np.float64)
    s = 4.0 * omega ** 2 / cs.kappa_keV ** 2
    return cs.Gamma0_P * primakoff_F(s)


def emission_number_pdf_per_keV(cs: CellState, channel, E_keV, p: Params):
    """Normalised number pdf p_c(E) [1/keV] of channel c's sampling kernel."""
    x = np.asarray(E_keV, dtype=np.float64) / cs.T_keV
    if channel == "compton":
        return spectra.compton_pdf(x) / cs.T_keV
    if channel == "brems":
        return spectra.brems_pdf(p.brems_gamma_shape, x) / cs.T_keV
    raise ValueError(channel)


def differential_emission(cs: CellState, channel, E_keV, p: Params):
    """d ndot_a / dE = n_e Gamma_c p_c(E)  [cm^-3 s^-1 keV^-1]."""
    rate = cs.Gamma_C if channel == "compton" else cs.Gamma_B
    return cs.n_e * rate * emission_number_pdf_per_keV(cs, channel, E_keV, p)


def equilibrium_density_per_keV(cs: CellState, E_keV, p: Params):
    """d n_a^eq / dE [cm^-3 keV^-1], BE or MB (Sec. II.I)."""
    E = np.asarray(E_keV, dtype=np.float64)
    pre = E ** 2 / (2.0 * math.pi ** 2 * K.HBARC_KEV_CM ** 3)
    x = E / cs.T_keV
    if p.eq_stats == 1:
        return pre / np.expm1(x)
    return pre * np.exp(-x)


def absorption_rate(cs: CellState, channel, E_keV, p: Params):
    """Gamma_abs(E) = (d ndot/dE)/(d n_eq/dE) [1/s] (Eq. gamma_abs)."""
    return (differential_emission(cs, channel, E_keV, p)
            / equilibrium_density_per_keV(cs, E_keV, p))
