"""Spectral records of the table/surrogate rate models (no GPU): the record's
rates against the closed forms they stand for, the spline and the sampler."""
import math

import numpy as np
import pytest

from oracle import constants as K
from oracle import plasma, step as ostep, surrogate as S


def exact_record(T, ne, Z, g_agg=1e-10, g_ae=1e-13, dt=1e12):
    """A record whose grid values are the exact targets of the cell itself."""
    cs, _ = S.cell(T, ne, Z)
    rec = np.empty(S.SR_LEN)
    for c, ch in enumerate(S.CHANNELS):
        rec[32 * c:32 * c + 32] = np.log(S.emissivity(ch, S.X_GRID, T, ne, Z)) + S.X_GRID
        rec[96 + 31 * c:96 + 31 * c + 31] = S.quantiles(ch, T, ne, Z)
    hc3 = K.HBARC_KEV_CM ** 3
    rec[189] = math.log(g_agg ** 2 * dt * math.pi ** 2 * hc3 / K.KEV_ERG) - 4 * math.log(T)
    rec[190] = math.log(g_ae ** 2 * dt * 2 * math.pi ** 2 * hc3 / K.KEV_ERG) - 4 * math.log(T)
    rec[191] = T
    return rec


@pytest.mark.parametrize("T,ne,Z", [(3.0, 6e25, 1), (1.2, 1e26, 2), (8.0, 3e23, 1)])
def test_record_rates_equal_closed_forms(T, ne, Z):
    g_agg, g_ae, dt = 1e-10, 1e-13, 1e12
    rec = exact_record(T, ne, Z, g_agg, g_ae, dt)
    p = plasma.Params(g_agg_GeV_inv=g_agg, g_ae=g_ae, dt_phys_s=dt)
    A = K.A_H if Z == 1 else K.A_HE
    cs = plasma.cell_state(T, np.array([ne / Z]), np.array([float(Z)]), np.array([A]), p)
    x = np.exp(np.random.default_rng(0).uniform(math.log(0.05), math.log(20.0), 400))
    E = x * T
    # Primakoff: Gamma dt from the record against Gamma0 F(s) dt (Eq. prim_rate)
    want = cs.Gamma0_P * plasma.primakoff_F(4 * E * E / cs.kappa_keV ** 2) * dt
    got = S.rec_prim_gdt(rec, x)
    assert np.max(np.abs(got / want - 1)) < 5e-4
    # at the grid points the spline is exact: only rounding remains
    xg = S.X_GRID[1:31]   # the grid points inside [0.05, 20]
    gp = S.rec_prim_gdt(rec, xg)
    wp = cs.Gamma0_P * plasma.primakoff_F(4 * (xg * T) ** 2 / cs.kappa_keV ** 2) * dt
    assert np.max(np.abs(gp / wp - 1)) < 1e-10
    # absorption: Gamma_abs dt (Eq. gamma_abs, MB and BE targets)
    for eq in (0, 1):
        p.eq_stats = eq
        for c, ch in ((1, "compton"), (2, "brems")):
            w = plasma.absorption_rate(cs, ch, xg * T, p) * dt
            assert np.max(np.abs(S.rec_tau(rec, c, xg, eq) / w - 1)) < 1e-10, (ch, eq)
            wx = plasma.absorption_rate(cs, ch, E, p) * dt
            assert np.max(np.abs(S.rec_tau(rec, c, x, eq) / wx - 1)) < 5e-4, (ch, eq)


def test_spline_and_sampler():
    rec = np.zeros(S.SR_LEN)
    lx = np.log(S.X_GRID)
    rec[32:64] = 3.0 * lx - 1.0   # stored values linear in ln x: the spline reproduces them exactly
    x = np.exp(np.linspace(math.log(0.05), math.log(20.0), 777))
    np.testing.assert_allclose(S.rec_lnL(rec, 1, x) + x, 3.0 * np.log(x) - 1.0, rtol=0, atol=1e-11)
    q = np.sort(np.exp(np.random.default_rng(1).uniform(math.log(0.06), math.log(19.0), 31)))
    rec[96 + 31:96 + 62] = q
    u = np.arange(33) / 32.0
    xs = S.rec_sample_x(rec, 1, u[:-1])
    np.testing.assert_allclose(xs, np.concatenate([[0.05], q]), rtol=1e-15)
    assert abs(S.rec_sample_x(rec, 1, np.array([1 - 1e-12]))[0] - 20.0) < 1e-6
    uu = np.random.default_rng(2).uniform(0, 1, 1000)
    xx = S.rec_sample_x(rec, 1, np.sort(uu))
    assert np.all(np.diff(xx) >= 0)


def test_table_record_at_a_node_is_the_node():
    tab = S.build_table(3, 2)
    # node (i=1, j=1, Z=1): kappa/T at the middle of the ln range, n_e = 1e26
    kT = math.exp(math.log(S.KT_LO) + math.log(S.KT_HI / S.KT_LO) * 0.5)
    ne = 1e26
    T = S.temperature(kT, ne, 1)
    rec = S.table_record(tab, T, kT * T, ne, 1, 1e-10, 1e-13, 1e12)
    node = tab[0, 1, 1].astype(np.float64)
    np.testing.assert_allclose(rec[:64], node[:64], rtol=1e-12)
    np.testing.assert_allclose(rec[96:189], node[96:189], rtol=1e-12)
    # the bremsstrahlung row gets the brackets back: the exact targets (to the
    # table's binary32 rounding)
    want = np.log(S.emissivity("brems", S.X_GRID, T, ne, 1)) + S.X_GRID
    np.testing.assert_allclose(rec[64:96], want, rtol=0, atol=2e-5)


def test_table_brems_row_across_the_bracket_floor():
    """Cells between nodes on either side of the brackets' floor: with the
    brackets divided out of the table and restored per cell, the record's
    bremsstrahlung row stays within 1e-3 on this coarse 12 x 8 table, where
    interpolating the kinked ln Q_B itself is off by more than 1 in ln."""
    nkt, nne = 12, 8
    tab = S.build_table(nkt, nne)
    worst = 0.0
    for T in (0.55, 0.6, 0.7, 0.8):
        for lne in (25.6, 25.75, 25.9, 25.97):
            ne = 10 ** lne
            kT = S.kappa_over_T(T, ne, 1)
            rec = S.table_record(tab, T, kT * T, ne, 1, 1e-10, 1e-13, 1e12)
            want = np.log(S.emissivity("brems", S.X_GRID, T, ne, 1)) + S.X_GRID
            worst = max(worst, float(np.max(np.abs(rec[64:96] - want))))
    assert worst < 1e-3, worst


def test_oracle_step_with_exact_record_matches_closed_forms_statistically():
    """With a record of the cell's own exact values, the record-model step and
    the closed-form step draw from the same laws: their event counts over
    many seeds agree within sampling noise."""
    T, ne = 3.0, 6e25
    p = plasma.Params(g_agg_GeV_inv=1e-10, g_ae=2e-12, dt_phys_s=2e12, w_a=3e9)
    rec = exact_record(T, ne, 1, p.g_agg_GeV_inv, p.g_ae, p.dt_phys_s)
    ci = ostep.CellInput(T, np.array([ne]), np.array([1.0]), np.array([K.A_H]))
    ev = {False: 0, True: 0}
    for seed in range(6):
        p.seed = seed
        for use in (False, True):
            parts = ostep.init_cell(p, 0, T, ne, 1e-12, 61, 200, 60)
            tally, _ = ostep.step_cell(ci, parts, p, 0, 0, 7, rec=rec if use else None)
            ev[use] += sum(tally.events.values())
    assert ev[False] > 20
    assert abs(ev[True] - ev[False]) <= 4 * math.sqrt(ev[False]), ev
