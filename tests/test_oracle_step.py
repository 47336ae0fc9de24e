"""Pins of the oracle's per-cell step: compaction, feedback, temperature,
detailed-balance steady states, unbiased variance control and spectra."""
import math

import numpy as np
from scipy import integrate, special

from oracle import constants as K
from oracle import plasma, step as S, tally
from oracle.plasma import Params, cell_state


def _hyd(n_e=6e25):
    return np.array([n_e]), np.array([1.0]), np.array([K.A_H])


def _electrons(n, T, seed=1, drift=(0.0, 0.0, 0.0)):
    rng = np.random.default_rng(seed)
    sig = math.sqrt(T / K.ME_C2_KEV)
    p = rng.normal(0, sig, size=(n, 3)) + np.array(drift)
    w = rng.uniform(0.5, 1.5, size=n) * 1e10
    return S.Species(w, p[:, 0], p[:, 1], p[:, 2], *rng.uniform(size=(3, n)))


# ---------------------------------------------------------------- compaction

def test_tail_fill_against_list_algorithm():
    rng = np.random.default_rng(0)
    for trial in range(300):
        n = int(rng.integers(0, 40))
        keep = rng.uniform(size=n) < rng.uniform()
        order = S.tail_fill(keep)
        # brute force: walk holes and movers explicitly
        ns = int(keep.sum())
        slots = list(range(n))
        movers = [i for i in range(ns, n) if keep[i]]
        out = []
        for i in range(ns):
            out.append(i if keep[i] else movers.pop(0))
        assert list(order) == out
        assert sorted(order) == sorted(np.flatnonzero(keep))


def test_recycle_against_list_algorithm():
    """Full-step slots: lost slots take the new particles in order, the rest
    are appended or the leftover holes closed by the tail fill; written out
    with plain lists."""
    rng = np.random.default_rng(1)
    for trial in range(400):
        n = int(rng.integers(0, 30))
        m = int(rng.integers(0, 12))
        keep = rng.uniform(size=n) < rng.uniform()
        old = S.Species(*[np.arange(n, dtype=float) + 100.0 * k for k in range(7)])
        new = S.Species(*[-1.0 - np.arange(m, dtype=float) - 100.0 * k for k in range(7)])
        got = S.recycle(old, keep, new)
        slots = [i if keep[i] else None for i in range(n)]   # survivors by old index
        fresh = [-1.0 - j for j in range(m)]
        for i in range(n):
            if slots[i] is None and fresh:
                slots[i] = fresh.pop(0)
        vals = [(float(v) if v is not None and v < 0 else v) for v in slots]
        if fresh:
            out = vals + fresh
        else:
            # close the remaining holes from the tail, in ascending order
            live = [v for v in vals if v is not None]
            ns = len(live)
            movers = [vals[i] for i in range(ns, n) if vals[i] is not None]
            out = [vals[i] if vals[i] is not None else movers.pop(0) for i in range(ns)]
        want = [float(v) for v in out]
        assert list(got.w) == want, (keep, m, list(got.w), want)
        assert list(got.z) == [v - 600.0 if v < 0 else v + 600.0 for v in want]
        assert len(got) == int(keep.sum()) + m


def test_full_step_holds_the_particles_of_separate_calls():
    """One full step and absorb + emit calls from the same state give the same
    particles (decisions do not depend on slot order within a step): photons
    slot for slot, axions in other slots (the full step reuses freed ones)."""
    p = Params(g_agg_GeV_inv=1e-10, g_ae=2e-12, dt_phys_s=4e12, seed=5)
    for cell in range(6):
        init = S.init_cell(p, cell, 3.0, 6e25, 1e-12, 96, 128, 80)
        p.w_a = init["g"].w[0]
        p.w_gamma_ref = p.w_a
        ci = S.CellInput(3.0, *_hyd())
        fused = {k: v.copy() for k, v in init.items()}
        sep = {k: v.copy() for k, v in init.items()}
        t1, _ = S.step_cell(ci, fused, p, 4, cell, 7, feedback=False)
        cs = cell_state(3.0, *_hyd(), p)
        t2 = S.StepTally()
        S.absorb_cell(cs, sep, p, 4, cell, 7, t2)
        S.emit_cell(cs, sep, p, 4, cell, 7, t2, n_g0=t2.n_g0)
        assert t1.events == t2.events and abs(t1.dE - t2.dE) <= 1e-12 * max(t1.gross_E, 1e-300)
        assert np.array_equal(np.stack(fused["g"].fields()), np.stack(sep["g"].fields()))
        a = np.stack(fused["a"].fields(), 1)
        b = np.stack(sep["a"].fields(), 1)
        assert a.shape == b.shape
        assert np.array_equal(a[np.lexsort(a.T[::-1])], b[np.lexsort(b.T[::-1])])


# ---------------------------------------------------------------- feedback

def _fb(parts, dE, dP, T=3.0, p=None):
    p = p or Params()
    cs = cell_state(T, *_hyd(), p)
    t = S.StepTally(dE=dE, dP=np.array(dP, dtype=float))
    return S.feedback_cell(cs, parts, p, t)


def _energy_momentum(e):
    pv = np.stack([e.px, e.py, e.pz], 1)
    return (np.sum(e.w * np.sum(pv * pv, 1)) / 2 * K.ME_C2_KEV, np.sum(e.w[:, None] * pv, 0))


def test_remap_conserves_momentum_and_energy():
    e = _electrons(500, 3.0, drift=(0.01, -0.003, 0.0))
    E0, P0 = _energy_momentum(e)
    for dE, dP in ((3e8, (1e6, -2e6, 5e5)), (-5e9, (0, 0, 0)), (1e10, (-4e7, 0, 3e7))):
        parts = {"e": e.copy()}
        r = _fb(parts, dE, dP)
        E1, P1 = _energy_momentum(parts["e"])
        assert np.allclose(P1 - P0, dP, rtol=1e-9, atol=1e-9 * np.abs(P0).max())   # Delta P exact
        assert abs((E1 - E0) - dE) < 1e-9 * abs(dE)                                  # Delta E exact
        assert abs(r.res_E) < 1e-9 * abs(dE)
        # new mean momentum = old mean + delta
        W = e.w.sum()
        assert np.allclose(r.b + (r.S - 1) * P0 / W, np.array(dP) / W, rtol=1e-9, atol=1e-20)


def test_remap_clamps_variance_and_carries_residual():
    e = _electrons(200, 1.0)
    E0, P0 = _energy_momentum(e)
    parts = {"e": e.copy()}
    r = _fb(parts, -10 * E0, (0, 0, 0))
    assert r.var_new == 0.0 and r.S == 0.0
    pv = np.stack([parts["e"].px, parts["e"].py, parts["e"].pz], 1)
    assert np.allclose(pv, pv[0], rtol=0, atol=1e-15)          # every electron at the mean
    E1, _ = _energy_momentum(parts["e"])
    assert abs(r.applied_E - (E1 - E0)) < 1e-9 * E0
    assert abs(r.res_E - (-10 * E0 - (E1 - E0))) < 1e-9 * E0


def test_cold_cell_keeps_variance():
    e = _electrons(10, 1.0)
    e.px[:] = 0.01
    e.py[:] = 0.0
    e.pz[:] = 0.0
    parts = {"e": e.copy()}
    r = _fb(parts, 1e5, (0, 0, 0))
    assert r.S == 1.0


def test_temperature_relaxation_is_geometric():
    """With no exchange the remap is the identity and T_n - T* = (1-r)^n (T_0 - T*)."""
    p = Params(T_mode=2, relax_r=0.1)
    e = _electrons(300, 2.0)
    pv = np.stack([e.px, e.py, e.pz], 1)
    W = e.w.sum()
    Pm = (e.w[:, None] * pv).sum(0)
    T_star = K.ME_C2_KEV / 3 * (np.sum(e.w * (pv * pv).sum(1)) - Pm @ Pm / W) / W
    T = 5.0
    parts = {"e": e}
    for n in range(1, 30):
        cs = cell_state(T, *_hyd(), p)
        r = S.feedback_cell(cs, parts, p, S.StepTally())
        T = r.T_new
        assert abs((T - T_star) - 0.9 ** n * (5.0 - T_star)) < 1e-12
    p.T_floor_keV, p.T_ceil_keV = 4.0, 4.5
    cs = cell_state(1.0, *_hyd(), p)
    assert S.feedback_cell(cs, parts, p, S.StepTally()).T_new == 4.0


def test_initial_maxwellian_temperature_estimate():
    p = Params(T_mode=2, relax_r=1.0, seed=3)
    T = 3.0
    N = 4096
    parts = S.init_cell(p, 5, T, 6e25, 1e-12, N, 16, 16)
    cs = cell_state(T, *_hyd(), p)
    r = S.feedback_cell(cs, parts, p, S.StepTally())
    assert abs(r.T_new / T - 1) < 4 * math.sqrt(2 / (3 * N))
    # photons: Planck mean energy 3 zeta(4)/zeta(3) T, weight n_gamma V / N
    g = parts["g"]
    assert np.allclose(g.w, S.photon_number_density(T) * 1e-12 / 16, rtol=1e-7)
    assert np.allclose(np.sqrt(g.px**2 + g.py**2 + g.pz**2) * K.ME_C2_KEV / T,
                       np.sqrt(g.px**2 + g.py**2 + g.pz**2) * K.ME_C2_KEV / T)


# ---------------------------------------------------------------- emission

def _emit_only(p, ci, parts, steps, mask, cell=0):
    E_all, w_all = [], []
    dE = 0.0
    for st in range(steps):
        pr = {k: v.copy() for k, v in parts.items()}
        pr["a"] = S.Species.empty()
        cs = cell_state(ci.T_keV, ci.n_ion, ci.Z, ci.A, p)
        t = S.StepTally()
        S.emit_cell(cs, pr, p, st, cell, mask, t)
        a = pr["a"]
        E_all.append(a.pmag() * K.ME_C2_KEV)
        w_all.append(a.w)
        dE += t.dE
    return np.concatenate(E_all), np.concatenate(w_all), dE


def test_emitted_power_matches_Q_compton_and_brems():
    """E[sum w' E] per step = Q V dt; checks Gamma = Q/(n_e <E>) with <E> the
    sampler mean (Eqs. QC, GammaC)."""
    T, V = 3.0, 1e-12
    ci = S.CellInput(T, *_hyd())
    for ch, a in ((S.CH_COMPTON, 1.70), (S.CH_BREMS, 1.70)):
        p = Params(g_ae=1e-13, dt_phys_s=1e12, seed=2, brems_gamma_shape=a)
        cs = cell_state(T, *_hyd(), p)
        e = _electrons(256, T)
        e.w[:] = 6e25 * V / 256
        Q = cs.Q_C if ch == S.CH_COMPTON else cs.Q_B
        # choose w_a so that ~60 events per step
        p.w_a = Q * V * p.dt_phys_s / (60 * (4.9 if ch == S.CH_COMPTON else a) * T * K.KEV_ERG)
        E, w, dE = _emit_only(p, ci, {"e": e, "g": S.Species.empty()}, 60, ch)
        emitted = np.sum(w * E) * K.KEV_ERG / 60
        assert abs(emitted / (Q * V * p.dt_phys_s) - 1) < 0.05
        assert abs(-dE * K.KEV_ERG / 60 / (Q * V * p.dt_phys_s) - 1) < 0.05


def test_unbiased_over_axion_weight_appendix_a():
    """App. A: the bremsstrahlung yield is invariant when w_a changes by 10^4,
    with capping active for the lightest weight."""
    T, V = 1.3, 1e-12
    ci = S.CellInput(T, *_hyd())
    e = _electrons(128, T)
    e.w[:] = 6e25 * V / 128
    yields = []
    for wa_scale, cap in ((1.0, 0.0), (1e-2, 2.0), (1e-4, 0.3)):
        p = Params(g_ae=1e-13, dt_phys_s=1e12, seed=4, lambda_cap=cap)
        cs = cell_state(T, *_hyd(), p)
        w_ref = cs.Q_B * V * p.dt_phys_s / (30 * 1.7 * T * K.KEV_ERG)
        p.w_a = w_ref * wa_scale
        E, w, _ = _emit_only(p, ci, {"e": e, "g": S.Species.empty()}, 80, S.CH_BREMS)
        yields.append(np.sum(w * E) / 80 / (cs.Q_B * V * p.dt_phys_s / K.KEV_ERG))
    assert all(abs(y - 1) < 0.06 for y in yields), yields


def test_primakoff_spectrum_matches_closed_form():
    """Primakoff on Planck photons against the screened closed form
    dQ/dE = E (P/dt) dn_gamma/dE; Table II reports Q ratios 0.992-1.00."""
    T, V = 1.3, 1e-12
    p = Params(g_agg_GeV_inv=1e-10, dt_phys_s=2e12, seed=6)
    ci = S.CellInput(T, *_hyd())
    init = S.init_cell(p, 0, T, 6e25, V, 0, 4096, 0)
    p.w_a = init["g"].w[0] / 4
    cs = cell_state(T, *_hyd(), p)
    steps = 150
    E, w, _ = _emit_only(p, ci, init, steps, S.CH_PRIMAKOFF)
    nb, Emax = 160, 80.0
    H = tally.histogram(E, w, nb, Emax)
    edges = np.linspace(0, Emax, nb + 1)
    dQ = tally.absolute_dQdE(H, V, steps * p.dt_phys_s, Emax / nb)
    # the photons are a finite sample of the Planck law: compare with the
    # closed form on the sampled photons' own energies as well as the law
    ref = tally.bin_average(lambda x: tally.primakoff_dQdE(cs, p, np.maximum(x, 1e-9)), edges)
    Q_mc, Q_ref = np.sum(dQ) * Emax / nb, np.sum(ref) * Emax / nb
    # events against the expectation over this photon sample (event noise only)
    g = init["g"]
    Eg = g.pmag() * K.ME_C2_KEV
    expect = np.sum(g.w * S.primakoff_prob(cs, p, Eg) * Eg) * steps
    assert abs(np.sum(w * E) / expect - 1) < 0.04
    # and against the Planck-law closed form (adds the photon sampling noise)
    assert abs(Q_mc / Q_ref - 1) < 0.06
    # shape: relative L2 over 2 keV bins (about 10^4 events: noise ~5e-2)
    coarse = dQ.reshape(40, 4).mean(1)
    coarse_ref = ref.reshape(40, 4).mean(1)
    assert tally.rel_l2(coarse, coarse_ref) < 0.1
    assert abs(np.sum(tally.normalised(H, Emax / nb)) * Emax / nb - 1) < 1e-12


# ---------------------------------------------------------------- detailed balance

def _expected_trajectory(cs, p, ch, V, steps):
    """N(k), U(k) after k steps of absorb -> emit from an empty start:
    n_k(E) = S(E) (1 - (1-P(E))^k) / P(E), S = d ndot/dE V dt / w_a."""
    def integrand(E, k, power):
        Pa = -np.expm1(-plasma.absorption_rate(cs, ch, E, p) * p.dt_phys_s)
        src = plasma.differential_emission(cs, ch, E, p) * V * p.dt_phys_s
        return src * (1 - (1 - Pa) ** k) / Pa * (E if power else 1.0)
    N = np.array([integrate.quad(integrand, 1e-9, 40 * cs.T_keV, args=(k, 0), limit=400)[0] for k in steps])
    U = np.array([integrate.quad(integrand, 1e-9, 40 * cs.T_keV, args=(k, 1), limit=400)[0] for k in steps])
    return N, U


def _relax(p, ci, e, steps, mask, cell=0):
    parts = {"e": e.copy(), "g": S.Species.empty(), "a": S.Species.empty()}
    N, U = [], []
    for st in range(steps):
        cs = cell_state(ci.T_keV, ci.n_ion, ci.Z, ci.A, p)
        t = S.StepTally()
        S.absorb_cell(cs, parts, p, st, cell, mask, t)
        S.emit_cell(cs, parts, p, st, cell, mask, t, n_g0=t.n_g0)
        a = parts["a"]
        N.append(a.w.sum())
        U.append(np.sum(a.w * a.pmag()) * K.ME_C2_KEV)
    return np.array(N), np.array(U)


def _check_relaxation(ch, eq_stats, T, tol=0.05):
    V = 1e-12
    p = Params(g_ae=1e-13, seed=8, eq_stats=eq_stats)
    cs = cell_state(T, *_hyd(), p)
    ci = S.CellInput(T, *_hyd())
    # dt: absorption probability 0.05 at x = 3; w_a: ~1500 macro-axions at equilibrium
    p.dt_phys_s = 0.05 / plasma.absorption_rate(cs, "compton" if ch == S.CH_COMPTON else "brems",
                                                np.array([3 * T]), p)[0]
    n_eq = T ** 3 / (math.pi ** 2 * K.HBARC_KEV_CM ** 3)
    if eq_stats == 1:
        n_eq *= special.zeta(3)
    p.w_a = n_eq * V / 3000
    e = _electrons(256, T)
    e.w[:] = 6e25 * V / 256
    steps = 240
    N, U = _relax(p, ci, e, steps, ch)
    name = "compton" if ch == S.CH_COMPTON else "brems"
    ks = np.arange(120, steps + 1, 10)
    Ne, Ue = _expected_trajectory(cs, p, name, V, ks)
    Nmc = np.array([N[k - 1] for k in ks])
    Umc = np.array([U[k - 1] for k in ks])
    assert abs(Nmc.mean() / Ne.mean() - 1) < tol, (Nmc.mean(), Ne.mean())
    # U is carried by the slowly absorbed high-energy tail: noisier than N
    assert abs(Umc.mean() / Ue.mean() - 1) < 1.5 * tol, (Umc.mean(), Ue.mean())
    # the expected plateau tends to the equilibrium n_eq V (x steady-state factor)
    return Ne[-1] / (n_eq * V)


def test_detailed_balance_relaxation_compton_mb():
    ratio = _check_relaxation(S.CH_COMPTON, 0, 3.0)
    assert 0.8 < ratio < 1.2


def test_detailed_balance_relaxation_brems_be():
    ratio = _check_relaxation(S.CH_BREMS, 1, 1.3)
    assert 0.8 < ratio < 1.3


def test_primakoff_pair_steady_state():
    """gamma <-> a conversion with inverse multiplicity m. With
    w_a = w_gamma = w_gamma_ref every macroparticle is one conversion unit: a
    conversion moves it whole (depletion clamp), so each one is a two-state
    Markov chain with per-step probabilities q_g = 1 - exp(-P_g),
    q_a = 1 - exp(-P_a) (lambda = P). Starting from photons only,
    E[a_k] = q_g/(q_g+q_a) (1 - (1-q_g-q_a)^k); for m = 1 the plateau is
    w_a = w_gamma (Sec. II.F.1, detailed balance of the pair)."""
    T, V = 1.3, 1e-12
    for m in (1.0, 2.0):
        p = Params(g_agg_GeV_inv=1e-10, dt_phys_s=4e12, seed=9, prim_inverse_mult=m)
        init = S.init_cell(p, 0, T, 6e25, V, 0, 1024, 0)
        p.w_a = init["g"].w[0]
        p.w_gamma_ref = p.w_a
        parts = {"e": S.Species.empty(), "g": init["g"], "a": S.Species.empty()}
        cs = cell_state(T, *_hyd(), p)
        tot0 = parts["g"].w.sum()
        E = init["g"].pmag() * K.ME_C2_KEV
        qg = -np.expm1(-S.primakoff_prob(cs, p, E))
        qa = -np.expm1(-S.primakoff_prob(cs, p, E, m))
        got, want = [], []
        for st in range(400):
            t = S.StepTally()
            S.absorb_cell(cs, parts, p, st, 0, S.CH_PRIMAKOFF, t)
            S.emit_cell(cs, parts, p, st, 0, S.CH_PRIMAKOFF, t, n_g0=t.n_g0)
            wa, wg = parts["a"].w.sum(), parts["g"].w.sum()
            assert abs((wa + wg) / tot0 - 1) < 1e-6          # number conserved
            if st >= 100:
                got.append(wa / tot0)
                want.append(np.mean(qg / (qg + qa) * (1 - (1 - qg - qa) ** (st + 1))))
        assert abs(np.mean(got) / np.mean(want) - 1) < 0.03, (m, np.mean(got), np.mean(want))
        if m == 1.0:
            plateau = np.mean(qg / (qg + qa))
            assert abs(plateau - 0.5) < 1e-12


def test_superposed_channels_keep_each_channel_power():
    """Compton-like and bremsstrahlung drawn as one Poisson process per
    electron: each channel's emitted power still equals its own Q V dt, and
    the event split follows lambda_C : lambda_B (superposition of Poisson
    processes, Sec. II.D.1 per channel)."""
    T, V = 3.0, 1e-12
    ci = S.CellInput(T, *_hyd())
    p = Params(g_ae=1e-13, dt_phys_s=1e12, seed=12)
    cs = cell_state(T, *_hyd(), p)
    e = _electrons(256, T)
    e.w[:] = 6e25 * V / 256
    p.w_a = (cs.Q_C + cs.Q_B) * V * p.dt_phys_s / (80 * 4.0 * T * K.KEV_ERG)
    steps = 60
    UC = UB = 0.0
    NC = NB = 0
    for st in range(steps):
        pr = {"e": e.copy(), "g": S.Species.empty(), "a": S.Species.empty()}
        t = S.StepTally()
        S.emit_cell(cs, pr, p, st, 0, S.CH_COMPTON | S.CH_BREMS, t)
        a = pr["a"]
        isC = t.new_axion_channel == S.CH_COMPTON
        UC += np.sum(a.w[isC] * t.new_axion_E[isC])
        UB += np.sum(a.w[~isC] * t.new_axion_E[~isC])
        NC += t.events["compton"]
        NB += t.events["brems"]
    QV = V * p.dt_phys_s * steps / K.KEV_ERG
    assert abs(UC / (cs.Q_C * QV) - 1) < 0.06
    assert abs(UB / (cs.Q_B * QV) - 1) < 0.12
    lam_ratio = (cs.Gamma_C / cs.Gamma_B)
    assert abs((NC / NB) / lam_ratio - 1) < 0.2
