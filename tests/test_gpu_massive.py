"""Massive axions (Sec. II.B: E = sqrt(p^2 + m_a^2), emission thresholds and
phase-space factors) through the C ABI against the oracle (needs a GB300):
full steps slot by slot, and the thermal-bath relaxation plateau against the
massive detailed-balance trajectory."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import constants as K
from oracle import plasma
from oracle import step as ostep
from oracle.plasma import Params as OParams
from parity_util import assert_species_close, oracle_step

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2604_24627_gb300 import AxionPlasma, _lib  # noqa: E402


@pytest.mark.parametrize("m", [0.0, 2.0, 6.0])
def test_massive_step_matches_oracle(m):
    """Hydrogen cells at 1.3-5 keV with 61 electrons, 37 photons and 13 axions
    (the sampler's momenta, read with the mass), all channels forward and
    inverse, couplings raised so that every channel fires (about 120
    Compton-like, 10 bremsstrahlung and 300-390 Primakoff events over the
    run, at most about 130 axions in a cell): two full steps,
    every axion and photon slot against the oracle's step with the same mass
    (thresholds, thinning of thermal-bath events, beta-scaled gamma->a
    momenta, a->gamma photons at the axion's total energy)."""
    T = np.linspace(1.3, 5.0, 16)
    prm = dict(g_agg_GeV_inv=1e-10, g_ae=1e-12, dt_phys_s=2e12, w_a=3.0e9, seed=0x3131, T_mode=2, relax_r=0.1,
               diag_enable=1, tally_enable=1, axion_mass_keV=m)
    pl = AxionPlasma(16, T, np.full((16, 1), 6e25), [1.0], [K.A_H], 1e-12, (64, 192, 512), prm)
    pl.sample(61, 37, 13)
    torch.cuda.synchronize()
    Tc = pl.temperatures().copy()
    events = {"compton": 0, "brems": 0, "prim": 0}
    for step in range(2):
        before = [pl.cell(c) for c in range(16)]
        res = pl.residuals()
        Tc = pl.temperatures().copy()
        pl.step(step, _lib.CH_ALL)
        diag = pl.cell_diag()
        for c in range(16):
            got = pl.cell(c)
            parts, tally, _ = oracle_step(before[c], Tc[c], np.array([6e25]), np.array([1.0]), np.array([K.A_H]),
                                          prm, step, c, _lib.CH_ALL, res=res[c])
            assert_species_close(got["a"], parts["a"], "m %g cell %d axions" % (m, c))
            assert_species_close(got["g"], parts["g"], "m %g cell %d photons" % (m, c))
            assert abs(diag[c][0] - tally.dE) <= 1e-5 * tally.gross_E + 1e-30
            for k in events:
                events[k] += tally.events[k]
            if m > 0:
                a = got["a"]
                E = np.sqrt(a["px"] ** 2 + a["py"] ** 2 + a["pz"] ** 2 + (m / K.ME_C2_KEV) ** 2) * K.ME_C2_KEV
                assert np.all(E >= m)
    assert events["compton"] > 50 and events["prim"] > 150, events
    pl.close()


def test_massive_relaxation_reaches_the_massive_plateau():
    """Compton-like emission and absorption alone (MB target) with m_a = T =
    3 keV, 256 cells of 256 electrons from an axion-free start: the alive
    axion number follows the massive closed-form trajectory within 3 %
    (its plateau, the massive equilibrium density T m^2 K_2(m/T) /
    (2 pi^2 (hbar c)^3) times the steady-state factor, is pinned in the
    oracle's tests)."""
    from scipy import integrate
    T, m, V, ncells = 3.0, 3.0, 1e-12, 256
    op = OParams(g_ae=1e-13, seed=8, eq_stats=0, axion_mass_keV=m)
    cs = plasma.cell_state(T, np.array([6e25]), np.array([1.0]), np.array([K.A_H]), op)
    op.dt_phys_s = 0.05 / plasma.absorption_rate(cs, "compton", np.array([3 * T]), op)[0]
    n_eq0 = T ** 3 / (math.pi ** 2 * K.HBARC_KEV_CM ** 3)
    op.w_a = float(np.float32(n_eq0 * V / 1500))
    prm = dict(g_ae=1e-13, seed=8, eq_stats=0, dt_phys_s=op.dt_phys_s, w_a=op.w_a, T_mode=0, tally_enable=1,
               axion_mass_keV=m)
    pl = AxionPlasma(ncells, T, np.full((ncells, 1), 6e25), [1.0], [K.A_H], V, (256, 4, 2048), prm)
    pl.sample(256, 0, 0)
    torch.cuda.synchronize()
    ks = np.arange(120, 241, 10)
    N = []
    k = 0
    for target in ks:
        while k < target:
            pl.absorb(k, 2)
            pl.emit(k, 2)
            k += 1
        _, tot = pl.tally()
        N.append(tot["n_axions"] / ncells)

    def integrand(E, kk):
        beta = math.sqrt(max(0.0, 1.0 - (m / E) ** 2))
        Pa = -np.expm1(-plasma.absorption_rate(cs, "compton", np.array([E]), op)[0] * op.dt_phys_s)
        src = plasma.differential_emission(cs, "compton", np.array([E]), op)[0] * V * op.dt_phys_s
        return src * beta * (1 - (1 - Pa) ** kk) / Pa
    Ne = np.array([integrate.quad(integrand, m, 40 * T, args=(kk,), limit=400)[0] for kk in ks])
    assert abs(np.mean(N) / Ne.mean() - 1) < 0.03, (np.mean(N), Ne.mean())
    pl.close()
