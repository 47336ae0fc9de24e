"""Parity of the CUDA path with the oracle, element by element on the same
seeded inputs, through the C ABI (needs a GB300 and the built library)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import plasma as oplasma, spectra, step as ostep, tally as otally
from oracle.plasma import cell_state
from parity_util import (assert_electron_remap_close, assert_species_close, oracle_params, oracle_step,
                         to_species)

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2604_24627_gb300 import AxionPlasma, _lib  # noqa: E402

A_H, A_HE = 1.00794, 4.002602
MIX_Z = np.array([1.0, 2.0])
MIX_A = np.array([A_H, A_HE])


def mix_density(n_e, ncells):
    n = n_e / 1.1
    return np.tile([[0.9 * n, 0.1 * n]], (ncells, 1))


def base_params(**kw):
    prm = dict(g_agg_GeV_inv=1e-10, g_ae=1e-12, dt_phys_s=2e12, w_a=3.0e9, seed=0x1234_0000_0042,
               T_mode=0, relax_r=0.1, diag_enable=1, tally_enable=1)
    prm.update(kw)
    return prm


def make(ncells, T, prm, caps=(64, 192, 512), n_e=6e25, counts=(61, 37, 13), cell_index_base=0):
    pl = AxionPlasma(ncells, T, mix_density(n_e, ncells), MIX_Z, MIX_A, 1e-12, caps, prm,
                     cell_index_base=cell_index_base)
    pl.sample(*counts)
    torch.cuda.synchronize()
    return pl


# ------------------------------------------------------------------ sampler

def test_sampler_matches_oracle():
    prm = base_params()
    ncells = 19
    T = np.linspace(1.0, 5.0, ncells)
    pl = make(ncells, T, prm, cell_index_base=1000)
    op = oracle_params(prm)
    for c in range(ncells):
        got = pl.cell(c)
        ref = ostep.init_cell(op, 1000 + c, T[c], 6e25, 1e-12, 61, 37, 13)
        for k in "ega":
            assert_species_close(got[k], ref[k], "cell %d %s" % (c, k))
    pl.close()


# ------------------------------------------------------------------ deterministic rates

@pytest.mark.parametrize("opts", [dict(), dict(kappa_mode=1, kappa_fixed_keV=3.0), dict(prim_targets=1),
                                  dict(brems_ee=0, brems_gamma_shape=1.4)])
def test_cell_parameters_match_oracle(opts):
    prm = base_params(**opts)
    T = np.array([0.5, 1.3, 3.0, 5.0, 10.0])
    n_e = np.array([1e23, 6e25, 6e25, 1e26, 1e24])
    ncells = len(T)
    n_ion = np.stack([mix_density(ne, 1)[0] for ne in n_e])
    pl = AxionPlasma(ncells, T, n_ion, MIX_Z, MIX_A, 1e-12, (4, 4, 4), prm)
    info = pl.cell_info()
    op = oracle_params(prm)
    for c in range(ncells):
        cs = cell_state(T[c], n_ion[c], MIX_Z, MIX_A, op)
        want = dict(rho=cs.rho, X_H=cs.X_H, n_e=cs.n_e, n_eff=cs.n_eff, S_Z=cs.S_Z, kappa=cs.kappa_keV,
                    Q_C=cs.Q_C, Q_B=cs.Q_B, Gamma_C=cs.Gamma_C, Gamma_B=cs.Gamma_B, Gamma0_P=cs.Gamma0_P,
                    eta=cs.eta)
        for i, name in enumerate(_lib.CELL_INFO_NAMES[:12]):
            w = want[name]
            assert abs(info[c, i] - w) <= 1e-5 * abs(w) + 1e-30, (c, name, info[c, i], w)
    pl.close()


@pytest.mark.parametrize("eq_stats", [0, 1])
def test_rates_match_oracle(eq_stats):
    prm = base_params(eq_stats=eq_stats)
    T = np.array([1.3, 3.0, 5.0])
    pl = AxionPlasma(3, T, mix_density(6e25, 3), MIX_Z, MIX_A, 1e-12, (4, 4, 4), prm)
    E = np.geomspace(0.02, 120.0, 4001)
    op = oracle_params(prm)
    for c in range(3):
        got = pl.eval_rates(c, E)
        cs = cell_state(T[c], mix_density(6e25, 1)[0], MIX_Z, MIX_A, op)
        E32 = E.astype(np.float32).astype(np.float64)
        want = np.stack([ostep.primakoff_prob(cs, op, E32),
                         ostep.primakoff_prob(cs, op, E32, op.prim_inverse_mult),
                         oplasma.absorption_rate(cs, "compton", E32, op) * op.dt_phys_s,
                         oplasma.absorption_rate(cs, "brems", E32, op) * op.dt_phys_s], axis=1)
        np.testing.assert_allclose(got, want, rtol=1e-5, atol=0)
    pl.close()


# ------------------------------------------------------------------ one step

STEP_CASES = {
    "all-mb": dict(),
    "be-weight-absorb": dict(eq_stats=1, absorb_mode=1),
    "capped": dict(lambda_cap=0.004, w_a=3e7),
    "evolved-T": dict(T_mode=2, relax_r=0.3, g_ae=2e-12),
    "inverse-x2-all-targets": dict(prim_inverse_mult=2.0, prim_targets=1, kappa_mode=1, kappa_fixed_keV=4.0),
    "no-ee": dict(brems_ee=0, brems_gamma_shape=2.2),
}


def _describe_mismatch(got, parts, tally):
    lines = []
    for k in "ga":
        g, o = got[k], parts[k]
        lines.append("%s: gpu %d oracle %d" % (k, len(g["w"]), len(o)))
        n = min(len(g["w"]), len(o))
        if n:
            dw = np.flatnonzero(np.abs(g["w"][:n] - o.w[:n]) > 1e-5 * np.abs(o.w[:n]))
            lines.append("  first differing slot %s" % (dw[:5],))
    lines.append("oracle events %s clamps %d caps %d" % (tally.events, tally.clamp_hits, tally.cap_hits))
    return "\n".join(lines)


def _compare_step(pl, before, T_before, prm, step, mask, res_before, label, allow_count_mismatch=0):
    op = oracle_params(prm)
    diag = pl.cell_diag()
    Tn = pl.temperatures()
    mismatched = []
    n_ion = pl.n_ion.reshape(pl.ncells, -1).cpu().numpy()
    for c in range(pl.ncells):
        got = pl.cell(c)
        parts, tally, fb = oracle_step(before[c], T_before[c], n_ion[c], MIX_Z, MIX_A, prm, step, c, mask,
                                       res=res_before[c])
        what = "%s cell %d" % (label, c)
        if len(got["a"]["w"]) != len(parts["a"]) or len(got["g"]["w"]) != len(parts["g"]):
            mismatched.append(what + "\n" + _describe_mismatch(got, parts, tally))
            continue
        assert_species_close(got["a"], parts["a"], what + " axions")
        assert_species_close(got["g"], parts["g"], what + " photons")
        d = diag[c]
        # (i) the exchange of this step: sums of opposite-signed events, so
        # the bound scales with the gross exchange
        assert abs(d[0] - tally.dE) <= 1e-5 * tally.gross_E + 1e-30, (what, d[0], tally.dE, tally.gross_E)
        assert np.all(np.abs(d[1:4] - tally.dP) <= 1e-5 * tally.gross_P + 1e-30), (what, d[1:4], tally.dP)
        # (ii) the feedback arithmetic, fed the GPU's own request
        e_parts = {"e": to_species(before[c]["e"])}
        cs = cell_state(T_before[c], n_ion[c], MIX_Z, MIX_A, op)
        req = ostep.StepTally(dE=d[0], dP=np.array(d[1:4]))
        fb2 = ostep.feedback_cell(cs, e_parts, op, req, res_before[c][0], np.array(res_before[c][1:4]))
        remapped = d[11] != 0.0 or d[4] != 0.0 or np.any(d[5:8] != 0.0)
        if remapped:
            assert_electron_remap_close(before[c]["e"], got["e"], e_parts["e"], what + " electrons")
            assert abs(d[4] - (fb2.S - 1)) <= 1e-4 * abs(fb2.S - 1) + 1e-12, (what, d[4], fb2.S - 1)
            # the applied energy the GPU reports is what its binary32 momenta
            # received (FP64 recomputation from the stored arrays)
            pe0 = np.stack([before[c]["e"][f] for f in ("px", "py", "pz")], 1)
            pe1 = np.stack([got["e"][f] for f in ("px", "py", "pz")], 1)
            dd = pe1 - pe0
            per = got["e"]["w"] * np.sum(dd * (2 * pe0 + dd), 1) / 2 * 510.99895
            assert abs(d[11] - per.sum()) <= 1e-5 * np.abs(per).sum() + 1e-30, (what, d[11], per.sum())
            # energy actually applied plus what is carried equals the request
            assert abs(d[11] + d[12] - (d[0] + res_before[c][0])) <= 1e-12 * abs(d[0]) + 1e-6
        if prm.get("T_mode", 0) == 2:
            assert abs(Tn[c] - fb2.T_new) <= 1e-5 * fb2.T_new, (what, Tn[c], fb2.T_new)
    # per-cell event counts agree exactly in at least 99.99 % of cells
    assert len(mismatched) <= allow_count_mismatch, "\n".join(mismatched)


@pytest.mark.parametrize("case", sorted(STEP_CASES))
def test_fused_step_matches_oracle(case):
    prm = base_params(**STEP_CASES[case])
    ncells = 24
    T = np.linspace(1.3, 5.0, ncells)
    pl = make(ncells, T, prm)
    for step in range(3):
        before = [pl.cell(c) for c in range(ncells)]
        T_before = pl.temperatures().copy()
        res_before = pl.residuals()
        pl.step(step, _lib.CH_ALL)
        _compare_step(pl, before, T_before, prm, step, _lib.CH_ALL, res_before, "%s step %d" % (case, step))
    H, tot = pl.tally()
    assert tot["events_p"] > 0 and tot["events_c"] > 0 and tot["events_b"] > 0, tot
    assert tot["dropped"] == 0
    pl.close()


@pytest.mark.parametrize("n_el", [256, 512])
def test_whole_electron_passes_match_oracle(n_el):
    """Cells whose electrons fill whole passes of 64 quads take the
    cell-by-cell electron decisions; every chunk here does."""
    prm = base_params()
    ncells = 12
    pl = make(ncells, np.linspace(1.5, 4.5, ncells), prm, caps=(n_el, 192, 512), counts=(n_el, 37, 13))
    for step in range(3):
        before = [pl.cell(c) for c in range(ncells)]
        T_before = pl.temperatures().copy()
        res_before = pl.residuals()
        pl.step(step, _lib.CH_ALL)
        _compare_step(pl, before, T_before, prm, step, _lib.CH_ALL, res_before, "%d e- step %d" % (n_el, step))
    _, tot = pl.tally()
    assert tot["events_c"] > 0 and tot["events_b"] > 0, tot
    pl.close()


def test_channel_masks_each_alone():
    prm = base_params()
    for mask in (1, 2, 4, 3, 6):
        pl = make(8, 3.0, prm)
        before = [pl.cell(c) for c in range(8)]
        res0 = pl.residuals()
        pl.step(5, mask)
        _compare_step(pl, before, np.full(8, 3.0), prm, 5, mask, res0, "mask %d" % mask)
        pl.close()


def test_separate_calls_hold_the_particles_of_a_full_step():
    """One full step and absorb + emit + feedback calls from the same state:
    electrons and photons slot for slot, axions as the same particles in
    other slots (the full step reuses the axion slots its absorb phase
    frees), T and carried exchange to FP64 rounding (the exchange sums may
    run in another order)."""
    prm = base_params(T_mode=2)
    a = make(16, 3.0, prm)
    b = make(16, 3.0, prm)
    for step in range(2):  # identical histories: full steps on both
        a.step(step, _lib.CH_ALL)
        b.step(step, _lib.CH_ALL)
    a.step(2, _lib.CH_ALL)
    b.absorb(2, _lib.CH_ALL)
    b.emit(2, _lib.CH_ALL)
    b.feedback(2)
    torch.cuda.synchronize()
    moved = 0
    for c in range(16):
        ca, cb = a.cell(c), b.cell(c)
        for k in "eg":
            for f in ca[k]:
                assert len(ca[k][f]) == len(cb[k][f]), (c, k, f)
                np.testing.assert_allclose(ca[k][f], cb[k][f], rtol=1e-6, atol=0, err_msg="%d %s %s" % (c, k, f))
        fa = np.stack([ca["a"][f] for f in ca["a"]], 1)
        fb = np.stack([cb["a"][f] for f in cb["a"]], 1)
        assert fa.shape == fb.shape, (c, fa.shape, fb.shape)
        assert np.array_equal(fa[np.lexsort(fa.T[::-1])], fb[np.lexsort(fb.T[::-1])]), c
        moved += int(not np.array_equal(fa, fb))
    assert moved > 0  # the two placements did differ somewhere
    np.testing.assert_allclose(a.temperatures(), b.temperatures(), rtol=1e-12)
    ra, rb = a.residuals(), b.residuals()
    np.testing.assert_allclose(ra, rb, rtol=1e-9, atol=1e-9 * np.abs(ra).max() + 1e-300)
    a.close()
    b.close()


def test_tally_matches_oracle_spectrum():
    """H_k = sum w'E per channel and bin (App. B) against the oracle's
    histogram of its own emitted axions; cumulative sums absorb the rare
    binary32 bin-edge flips."""
    prm = base_params(g_ae=2e-12)
    ncells = 12
    pl = make(ncells, 3.0, prm, counts=(61, 37, 0))
    before = [pl.cell(c) for c in range(ncells)]
    pl.step(0, _lib.CH_ALL)
    H, tot = pl.tally()
    Hw = np.zeros((3, pl.nbins))
    N = np.zeros(3)
    U = np.zeros(3)
    for c in range(ncells):
        parts, tally, fb = oracle_step(before[c], 3.0, mix_density(6e25, 1)[0], MIX_Z, MIX_A, prm, 0, c, 7)
        nn = len(tally.new_axion_E)
        w_new = parts["a"].w[len(parts["a"]) - nn:]
        for k, ch in enumerate((ostep.CH_PRIMAKOFF, ostep.CH_COMPTON, ostep.CH_BREMS)):
            sel = tally.new_axion_channel == ch
            Hw[k] += otally.histogram(tally.new_axion_E[sel], w_new[sel], pl.nbins, 80.0)
            N[k] += w_new[sel].sum()
            U[k] += np.sum(w_new[sel] * tally.new_axion_E[sel])
    for k, name in enumerate("pcb"):
        assert abs(tot["nemit_" + name] - N[k]) <= 1e-5 * N[k], (name, tot["nemit_" + name], N[k])
        assert abs(tot["uemit_" + name] - U[k]) <= 1e-5 * U[k], (name, tot["uemit_" + name], U[k])
        cg, cw = np.cumsum(H[k]), np.cumsum(Hw[k])
        assert np.all(np.abs(cg - cw) <= 1e-5 * cw[-1] + 1e-12), name
    assert N.min() > 0
    pl.close()


# ------------------------------------------------------------------ edge cases

def test_empty_and_full_cells():
    prm = base_params(g_ae=2e-12)
    pl = make(5, 3.0, prm, caps=(8, 8, 8), counts=(0, 0, 0))
    pl.step(0, _lib.CH_ALL)
    H, tot = pl.tally()
    assert tot["events_p"] == 0 and tot["macro_axions"] == 0
    pl.close()
    # an axion slab too small for the products latches AXPIC_E_CAPACITY
    prm = base_params(g_ae=1e-10, w_a=1e8)
    pl = make(4, 5.0, prm, caps=(64, 64, 4), counts=(61, 37, 0))
    pl.step(0, _lib.CH_ALL)
    with pytest.raises(_lib.AxpicError) as ei:
        pl.sync()
    assert ei.value.status == _lib.AXPIC_E_CAPACITY
    assert (pl.counts()["axions"] <= 4).all()
    pl.ctx = None


def test_non_finite_temperature_is_reported():
    """Host-side fault injection: a NaN temperature handed in by the caller
    is caught when the cell records are rebuilt (no step is run) and the next
    synchronising call returns AXPIC_E_NUMERIC; destroying the context
    reports it again."""
    pl = make(4, 3.0, base_params())
    pl.T[2] = float("nan")
    pl.update_cells()
    with pytest.raises(_lib.AxpicError) as e:
        pl.sync()
    assert e.value.status == _lib.AXPIC_E_NUMERIC
    with pytest.raises(_lib.AxpicError):
        pl.close()


def test_invalid_arguments_rejected():
    prm = base_params()
    with pytest.raises(_lib.AxpicError):
        AxionPlasma(4, 3.0, mix_density(6e25, 4), MIX_Z, MIX_A, 1e-12, (6, 8, 8), prm)   # capacity % 4
    pl = make(4, 3.0, prm)
    with pytest.raises(_lib.AxpicError):
        pl.step(-1, 7)
    with pytest.raises(_lib.AxpicError):
        pl.step(0, 8)
    with pytest.raises(_lib.AxpicError):
        pl.sample(1000, 0, 0)
    pl.close()
