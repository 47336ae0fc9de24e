"""Pins of the oracle's plasma state and rates (Sec. II.E-II.H)."""
import math
import os

import numpy as np
from scipy import integrate, optimize

from oracle import constants as K
from oracle import plasma, tally
from oracle.plasma import Params, cell_state, primakoff_F

from test_oracle_spectra import table2

H = (np.array([1.0]), np.array([K.A_H]))


def _hydrogen(n_e):
    return np.array([n_e]), np.array([1.0]), np.array([K.A_H])


def test_F_equals_screened_coulomb_angular_integral():
    """sigma ~ int dOmega |k x k'|^2 / (q^2 (q^2 + kappa^2)); with omega = 1 and
    c = cos(theta) the angular integral reduces to
    F(s) = int_{-1}^{1} (1+c) / (2(1-c) + 4/s) dc  (Eq. prim_F)."""
    for s in (1e-6, 1e-4, 9.99e-4, 1e-3, 1.01e-3, 1e-2, 0.3, 1.0, 7.0, 100.0, 1e6):
        ref = integrate.quad(lambda c: (1 + c) / (2 * (1 - c) + 4 / s), -1, 1,
                             epsabs=0, epsrel=1e-12, limit=200)[0]
        got = primakoff_F(np.array([s]))[0]
        assert abs(got - ref) <= 2e-11 * ref, (s, got, ref)


def test_F_limits():
    s = np.array([1e-9, 1e-7])
    assert np.allclose(primakoff_F(s), s / 2, rtol=1e-6)
    s = np.array([1e8, 1e10])
    assert np.allclose(primakoff_F(s), np.log(s) - 1, rtol=1e-6)


def test_primakoff_all_targets_equals_raffelt_kappa_form():
    """With every charge as a target, n_t Z^2 -> n_eff and
    Gamma = alpha g^2 n_eff F (hbar c)^2 c / 8 must equal the textbook
    Gamma = g^2 T kappa^2 F / (32 pi) (natural units, divided by hbar)."""
    for T, n_e in ((1.3, 6e25), (3.0, 1e24), (5.0, 3e26)):
        p = Params(g_agg_GeV_inv=1e-10, prim_targets=1)
        cs = cell_state(T, *_hydrogen(n_e), p)
        omega = np.array([0.5, 3.0, 20.0])
        s = 4 * omega ** 2 / cs.kappa_keV ** 2
        raffelt = ((1e-10) ** 2 * (T * 1e-6) * (cs.kappa_keV * 1e-6) ** 2 * primakoff_F(s)
                   / (32 * math.pi) / K.HBAR_GEV_S)
        assert np.allclose(plasma.primakoff_rate(cs, omega), raffelt, rtol=1e-12)


def test_debye_kappa_numbers():
    # kappa^2 = 4 pi alpha n_eff / T; hydrogen n_e = 6e25 at 1.3 keV -> ~8.06 keV
    cs = cell_state(1.3, *_hydrogen(6e25), Params())
    nat = 2 * 6e25 * K.HBARC_KEV_CM ** 3
    assert abs(cs.kappa_keV - math.sqrt(4 * math.pi * K.ALPHA_EM * nat / 1.3)) < 1e-12
    assert 8.0 < cs.kappa_keV < 8.1


def test_composition_of_config_two():
    """Ions 90% Z=1 + 10% Z=2 by number with n_e = 6e25 cm^-3."""
    n = 6e25 / 1.1
    cs = cell_state(3.0, np.array([0.9 * n, 0.1 * n]), np.array([1.0, 2.0]),
                    np.array([K.A_H, K.A_HE]), Params())
    assert abs(cs.n_e - 6e25) < 1e12
    assert abs(cs.rho - 118.4) < 0.1
    assert abs(cs.X_H - 0.694) < 1e-3
    assert abs(cs.S_Z - (0.9 * n + 4 * 0.1 * n)) < 1e12
    assert abs(cs.n_eff - (6e25 + 0.9 * n + 0.4 * n)) < 1e12


def test_compton_emissivity_matches_table2():
    """Table II Compton Q^R (g_ae = 1e-13) is rho eps_C for solar-core
    hydrogen at n_e = 6e25 cm^-3 within 3 percent, and its T^6 ratios."""
    p = Params(g_ae=1e-13)
    rows = [r for r in table2() if r["process"] == "compton"]
    Q = []
    for r in rows:
        cs = cell_state(r["T"], *_hydrogen(6e25), p)
        assert abs(cs.Q_C / r["Q_R"] - 1.0) < 0.03
        Q.append(cs.Q_C)
    assert abs(Q[1] / Q[0] - (3.0 / 1.3) ** 6) < 1e-9 * Q[1] / Q[0]
    assert abs(Q[2] / Q[1] - (5.0 / 3.0) ** 6) < 1e-9 * Q[2] / Q[1]


def test_compton_rate_recovers_emissivity():
    """n_e Gamma_C <E> = Q_C, with <E> the sampler's number mean."""
    p = Params(g_ae=1e-13)
    cs = cell_state(3.0, *_hydrogen(6e25), p)
    mean_E = integrate.quad(lambda E: E * plasma.emission_number_pdf_per_keV(cs, "compton", E, p),
                            1e-6, 300)[0]
    assert abs(cs.n_e * cs.Gamma_C * mean_E * K.KEV_ERG / cs.Q_C - 1) < 1e-8
    ebar = integrate.quad(lambda E: E * plasma.emission_number_pdf_per_keV(cs, "brems", E, p),
                          1e-9, 300, limit=200)[0]
    assert abs(cs.n_e * cs.Gamma_B * ebar * K.KEV_ERG / cs.Q_B - 1) < 1e-7


def test_brems_fit_brackets_clamped():
    """In the cold dense corner both brackets are negative and are clamped."""
    p = Params(g_ae=1e-13)
    n = 1e26 / 2
    cs = cell_state(0.5, np.array([n]), np.array([2.0]), np.array([K.A_HE]), p)
    assert cs.eta > 1 / 0.0698
    assert cs.eps_eZ == 0.0 and cs.eps_ee == 0.0 and cs.Q_B == 0.0


def test_detailed_balance_identity_and_mb_form():
    """Gamma_abs dn_eq/dE = d ndot/dE; for MB the absorption rate is the
    forward density times e^{E/T} over E^2/(2 pi^2 (hbar c)^3)."""
    p = Params(g_ae=1e-13)
    cs = cell_state(3.0, *_hydrogen(6e25), p)
    E = np.linspace(0.3, 60, 50)
    for ch in ("compton", "brems"):
        ga = plasma.absorption_rate(cs, ch, E, p)
        fwd = plasma.differential_emission(cs, ch, E, p)
        assert np.allclose(ga * plasma.equilibrium_density_per_keV(cs, E, p), fwd, rtol=1e-12)
        mb = fwd * np.exp(E / 3.0) * 2 * math.pi ** 2 * K.HBARC_KEV_CM ** 3 / E ** 2
        assert np.allclose(ga, mb, rtol=1e-12)


def test_primakoff_power_peak_within_limits():
    """Primakoff on a Planck bath: dQ/dE ~ E^3 F(4E^2/kappa^2)/(e^x-1) peaks
    between the kappa -> inf (x^5, 4.965 T) and kappa -> 0 (x^3 ln x) limits;
    all Table II Primakoff peaks (4.68 T, 3.83 T, 3.37 T) lie inside."""
    p = Params(g_agg_GeV_inv=1e-13, kappa_mode=1, dt_phys_s=1.0)
    peaks = []
    for kT in (1e-3, 0.1, 1.0, 3.0, 10.0, 1e3):
        p.kappa_fixed_keV = kT
        cs = cell_state(1.0, *_hydrogen(6e25), p)
        r = optimize.minimize_scalar(lambda E: -tally.primakoff_dQdE(cs, p, np.array([E]))[0],
                                     bounds=(0.5, 8), method="bounded", options={"xatol": 1e-9})
        peaks.append(r.x)
    assert all(2.82 < x < 4.966 for x in peaks)
    assert all(np.diff(peaks) > 0)
    assert abs(peaks[-1] - 4.9651) < 2e-3
    for row in table2():
        if row["process"] == "primakoff":
            assert 2.82 < row["Epk_R"] / row["T"] < 4.966
