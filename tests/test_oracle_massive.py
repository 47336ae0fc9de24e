"""Pins of the oracle's massive-axion kinematics (Sec. II.B: E = sqrt(p^2 +
m_a^2); thresholds and phase-space factors in emission and absorption): the
detailed-balance plateau against the massive Maxwell-Boltzmann density
(closed form with the Bessel function K_2), the emission threshold and the
momenta of every product, and the reduction to the massless step."""
import math

import numpy as np
from scipy import integrate, special

from oracle import constants as K
from oracle import plasma, step as S
from oracle.plasma import Params, cell_state


def _hyd(n_e=6e25):
    return np.array([n_e]), np.array([1.0]), np.array([K.A_H])


def _cell(T, p, n_el=256, n_ph=64, n_ax=64, cell=0):
    return S.init_cell(p, cell, T, 6e25, 1e-12, n_el, n_ph, n_ax)


def test_massless_limit_is_the_massless_step():
    """axion_mass_keV = 0 leaves every particle of a full step as it is
    without the option."""
    T = 3.0
    base = dict(g_agg_GeV_inv=1e-10, g_ae=2e-12, dt_phys_s=2e12, w_a=3e9, seed=4)
    out = []
    for p in (Params(**base), Params(**base, axion_mass_keV=0.0)):
        parts = _cell(T, p)
        S.step_cell(S.CellInput(T, *_hyd()), parts, p, 1, 0, 7)
        out.append(parts)
    for k in "ega":
        for f in ("w", "px", "py", "pz", "x", "y", "z"):
            assert np.array_equal(getattr(out[0][k], f), getattr(out[1][k], f))


def test_emitted_axions_above_threshold_with_massive_momenta():
    """Thermal-bath emission with m_a = T: every emitted axion has E >= m_a
    and |p| = sqrt(E^2 - m_a^2) / m_e c^2; the kept fraction of events is the
    mean of beta = p/E over the massless spectrum (thinning); the electrons'
    exchange is minus the emitted total energy and momentum."""
    T = 3.0
    m = 3.0
    mu = m / K.ME_C2_KEV
    kept, drawn, beta_sum = 0, 0, 0.0
    for seed in range(8):
        p = Params(g_ae=1e-11, dt_phys_s=2e12, w_a=3e9, seed=seed, axion_mass_keV=m)
        p0 = Params(g_ae=1e-11, dt_phys_s=2e12, w_a=3e9, seed=seed)
        ci = S.CellInput(T, *_hyd())
        cs = cell_state(T, *_hyd(), p)
        parts = {"e": _cell(T, p, 512, 0, 0)["e"], "g": S.Species.empty(), "a": S.Species.empty()}
        parts0 = {k: v.copy() for k, v in parts.items()}
        t, t0 = S.StepTally(), S.StepTally()
        S.emit_cell(cs, parts, p, 0, 0, S.CH_COMPTON | S.CH_BREMS, t)
        S.emit_cell(cs, parts0, p0, 0, 0, S.CH_COMPTON | S.CH_BREMS, t0)
        a, a0 = parts["a"], parts0["a"]
        E = S.axion_energy_mc2(a, mu) * K.ME_C2_KEV
        assert np.all(E >= m * (1 - 1e-6))
        # the same draws: a kept axion is its massless twin's energy, thinned
        E0 = a0.pmag() * K.ME_C2_KEV
        assert set(np.round(E, 6)).issubset(set(np.round(E0, 6)))
        assert abs(t.dE + np.sum(a.w * E)) <= 1e-9 * np.sum(a.w * E)
        np.testing.assert_allclose(t.dP, -np.array([np.sum(a.w * a.px), np.sum(a.w * a.py), np.sum(a.w * a.pz)]),
                                   rtol=1e-9, atol=1e-30)
        kept += len(a)
        drawn += len(a0)
        x = E0 / K.ME_C2_KEV
        beta_sum += float(np.sum(np.sqrt(np.maximum(x * x - mu * mu, 0)) / x))
    assert drawn > 300
    assert abs(kept - beta_sum) < 4 * math.sqrt(beta_sum), (kept, beta_sum)


def test_primakoff_with_mass_threshold_and_momenta():
    """gamma -> a with m_a = 3 keV on photons of a 1.3 keV bath boosted so
    that conversions are frequent: only photons above m_a convert, every
    axion keeps the photon's energy and direction with |p| = beta |p_gamma|;
    a -> gamma of a massive axion gives a photon of energy E along p."""
    T, m = 1.3, 3.0
    mu = m / K.ME_C2_KEV
    p = Params(g_agg_GeV_inv=3e-10, dt_phys_s=2e12, w_a=1.0, seed=3, axion_mass_keV=m)
    cs = cell_state(T, *_hyd(), p)
    parts = _cell(T, p, 0, 4096, 0)
    p.w_a = float(parts["g"].w[0]) / 4
    g = parts["g"].copy()
    t = S.StepTally()
    S.emit_cell(cs, parts, p, 0, 0, S.CH_PRIMAKOFF, t)
    a = parts["a"]
    assert len(a) > 50
    E = S.axion_energy_mc2(a, mu)
    # each axion's momentum direction and energy against its parent photons'
    pg = g.pmag()
    pa = a.pmag()
    for i in range(len(a)):
        j = np.argmin(np.abs(pg - E[i]) + np.abs(g.px / pg - a.px[i] / pa[i]) + np.abs(g.py / pg - a.py[i] / pa[i]))
        # E = omega and |p| = beta |p_gamma| (beta in binary32: e^2 - mu^2
        # cancels near the threshold, a few 1e-7 relative)
        assert abs(pg[j] - E[i]) <= 2e-6 * E[i]
        assert abs(g.pz[j] / pg[j] - a.pz[i] / pa[i]) <= 1e-12
        assert abs(pa[i] - math.sqrt(pg[j] ** 2 - mu ** 2)) <= 2e-6 * pa[i]
    assert np.all(E * K.ME_C2_KEV > m)
    # a -> gamma: the photons carry the axions' total energy along p
    p2 = Params(g_agg_GeV_inv=3e-10, dt_phys_s=2e12, w_a=p.w_a, seed=5, axion_mass_keV=m)
    parts2 = {"e": S.Species.empty(), "g": S.Species.empty(), "a": a.copy()}
    t2 = S.StepTally()
    S.absorb_cell(cs, parts2, p2, 0, 0, S.CH_PRIMAKOFF, t2)
    ng = parts2["g"]
    assert len(ng) > 0
    Eg = ng.pmag()
    Ea = S.axion_energy_mc2(a, mu)
    for i in range(len(ng)):
        j = np.argmin(np.abs(a.px / a.pmag() - ng.px[i] / Eg[i]) + np.abs(a.py / a.pmag() - ng.py[i] / Eg[i]))
        assert abs(Eg[i] - Ea[j]) <= 1e-12 * Ea[j]


def _expected_massive_trajectory(cs, p, ch, V, ks, m):
    """N(k) after k absorb -> emit steps from an empty start with mass m: per
    total energy E > m, n_k(E) = S(E) beta(E) (1 - (1 - P(E))^k) / P(E), S the
    massless source d ndot/dE V dt, P = 1 - exp(-Gamma_abs(E) dt)."""
    def integrand(E, k):
        beta = math.sqrt(max(0.0, 1.0 - (m / E) ** 2))
        Pa = -np.expm1(-plasma.absorption_rate(cs, ch, np.array([E]), p)[0] * p.dt_phys_s)
        src = plasma.differential_emission(cs, ch, np.array([E]), p)[0] * V * p.dt_phys_s
        return src * beta * (1 - (1 - Pa) ** k) / Pa
    return np.array([integrate.quad(integrand, m, 40 * cs.T_keV, args=(k,), limit=400)[0] for k in ks])


def test_detailed_balance_plateau_of_massive_axions():
    """Compton-like emission and absorption (MB target) alone with m_a = T:
    the axion number follows the massive closed-form trajectory, whose
    plateau is the massive Maxwell-Boltzmann density n_eq(m) = T m^2
    K_2(m/T) / (2 pi^2 (hbar c)^3) (per volume, times the steady-state
    factor of the absorb -> emit order), i.e. (m/T)^2 K_2(m/T) / 2 of the
    massless plateau."""
    T, m, V = 3.0, 3.0, 1e-12
    p = Params(g_ae=1e-13, seed=8, eq_stats=0, axion_mass_keV=m)
    cs = cell_state(T, *_hyd(), p)
    ci = S.CellInput(T, *_hyd())
    p.dt_phys_s = 0.05 / plasma.absorption_rate(cs, "compton", np.array([3 * T]), p)[0]
    n_eq0 = T ** 3 / (math.pi ** 2 * K.HBARC_KEV_CM ** 3)
    p.w_a = n_eq0 * V / 3000
    e = S.init_cell(p, 0, T, 6e25, V, 256, 0, 0)["e"]
    parts = {"e": e, "g": S.Species.empty(), "a": S.Species.empty()}
    N = []
    for st in range(240):
        t = S.StepTally()
        S.absorb_cell(cs, parts, p, st, 0, S.CH_COMPTON, t)
        S.emit_cell(cs, parts, p, st, 0, S.CH_COMPTON, t, n_g0=t.n_g0)
        N.append(parts["a"].w.sum())
    ks = np.arange(120, 241, 10)
    Ne = _expected_massive_trajectory(cs, p, "compton", V, ks, m)
    Nmc = np.array([N[k - 1] for k in ks])
    assert abs(Nmc.mean() / Ne.mean() - 1) < 0.06, (Nmc.mean(), Ne.mean())
    # the plateau against the massive equilibrium density, and the ratio to
    # the massless one against the Bessel closed form
    n_eq_m = T * m * m * special.kv(2, m / T) / (2 * math.pi ** 2 * K.HBARC_KEV_CM ** 3)
    ratio = Ne[-1] / (n_eq_m * V)
    assert 0.8 < ratio < 1.2, ratio
    N0 = _expected_massive_trajectory(cs, p, "compton", V, ks[-1:], 1e-9)[0]
    assert abs((Ne[-1] / N0) / ((m / T) ** 2 * special.kv(2, m / T) / 2) - 1) < 0.05
    # every axion alive is above threshold
    a = parts["a"]
    assert np.all(S.axion_energy_mc2(a, m / K.ME_C2_KEV) * K.ME_C2_KEV >= m * (1 - 1e-6))
