"""Helpers that run the CUDA path and the oracle on the same seeded input and
compare them cell by cell (used by the -m gpu tests and smoke)."""
import numpy as np

from oracle import step as ostep
from oracle.plasma import Params as OParams, cell_state

FIELDS = ("w", "px", "py", "pz", "x", "y", "z")
ORACLE_KEYS = ("g_agg_GeV_inv", "g_ae", "dt_phys_s", "w_a", "w_gamma_ref", "lambda_cap", "kappa_mode",
               "kappa_fixed_keV", "prim_targets", "prim_inverse_mult", "eq_stats", "brems_ee", "absorb_mode",
               "brems_gamma_shape", "relax_r", "T_floor_keV", "T_ceil_keV", "T_mode", "seed", "axion_mass_keV")


def oracle_params(prm):
    return OParams(**{k: v for k, v in prm.items() if k in ORACLE_KEYS})


def to_species(d):
    return ostep.Species(*[np.asarray(d[f], dtype=np.float64) for f in FIELDS])


def oracle_step(cell_arrays, T, n_ion, Z, A, prm, step, gcell, mask, res=None, phases="step", rec=None, net=None):
    """Run the oracle's step on one cell's GPU arrays (rec: the oracle's own
    spectral record for the table rate model; net: the oracle network's
    constants and quantile record for a cell the surrogate is trusted for).
    Returns (parts, tally, fb)."""
    parts = {k: to_species(cell_arrays[k]) for k in "ega"}
    op = oracle_params(prm)
    ci = ostep.CellInput(T, np.asarray(n_ion), np.asarray(Z), np.asarray(A))
    res_E, res_P = (0.0, np.zeros(3)) if res is None else (res[0], np.asarray(res[1:4]))
    tally, fb = ostep.step_cell(ci, parts, op, step, gcell, mask, res_E, res_P, rec=rec, net=net)
    return parts, tally, fb


def assert_species_close(got, want, what, rtol=1e-5, rel_atol=1e-6):
    """got: dict of float arrays (GPU, binary32 values); want: oracle Species."""
    n = len(want)
    assert len(got["w"]) == n, "%s: count %d != oracle %d" % (what, len(got["w"]), n)
    if n == 0:
        return
    np.testing.assert_allclose(got["w"], want.w, rtol=rtol, atol=0, err_msg=what + " w")
    pmag = np.sqrt(want.px ** 2 + want.py ** 2 + want.pz ** 2)
    for f in ("px", "py", "pz"):
        diff = np.abs(got[f] - getattr(want, f))
        tol = rtol * np.abs(getattr(want, f)) + rel_atol * pmag + 1e-30
        bad = diff > tol
        assert not bad.any(), "%s %s: %d mismatches, worst %g vs tol %g" % (
            what, f, bad.sum(), diff[bad].max(), tol[bad][np.argmax(diff[bad])])
    for f in ("x", "y", "z"):
        np.testing.assert_allclose(got[f], getattr(want, f), rtol=1e-6, atol=1e-7, err_msg=what + " " + f)


def assert_electron_remap_close(before, got, want, what):
    """Electron momenta after the remap: compare the change p' - p, to the
    binary32 storage resolution of p plus 1e-5 of the change."""
    n = len(want)
    assert len(got["w"]) == n
    for f in ("px", "py", "pz"):
        p0 = np.asarray(before[f])
        dg = got[f] - p0
        dw = getattr(want, f) - p0
        ulp = np.spacing(np.maximum(np.abs(p0), np.abs(getattr(want, f))).astype(np.float32)).astype(np.float64)
        tol = 2.0 * ulp + 1e-5 * np.abs(dw) + 1e-6 * np.abs(dw).max()
        bad = np.abs(dg - dw) > tol
        assert not bad.any(), "%s %s: %d remap mismatches" % (what, f, bad.sum())
