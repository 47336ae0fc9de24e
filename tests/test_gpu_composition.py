"""Composition from the deposited electron density through the C ABI against
the composition oracle: ion densities of ragged cells (empty, one warp's
worth and more, full) with mass fractions and with each bound species; the
in-place deposit rebuilding the cell records; invalid arguments (needs a
GB300)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import composition as CO
from oracle import plasma as P

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2604_24627_gb300 import AxionPlasma, _lib  # noqa: E402

Z3, A3 = [1.0, 2.0, 6.0], [1.00794, 4.002602, 12.011]
V = 1e-12
PRM = dict(g_agg_GeV_inv=1e-10, g_ae=1e-13, dt_phys_s=1e12, w_a=1e9, seed=3, tally_enable=0)


def plasma_with_weights(cells_w, Z, A, cap):
    n = len(cells_w)
    pl = AxionPlasma(n, np.full(n, 2.0), np.full((n, len(Z)), 1e24), Z, A, V, (cap, 4, 4), PRM)
    e = pl.slabs["electrons"]
    for c, w in enumerate(cells_w):
        k = len(w)
        e.set_cell(c, {"w": w, "px": np.zeros(k), "py": np.zeros(k), "pz": np.zeros(k), "x": np.zeros(k),
                       "y": np.zeros(k), "z": np.zeros(k)})
    torch.cuda.synchronize()
    return pl


@pytest.mark.parametrize("cap,logw", [(128, False), (4096, True)])
def test_deposit_matches_oracle(cap, logw):
    """A lane sums its weights (count/32 of them) as a compensated binary32
    pair, within about (terms) 2^-48 of the exact sum, and the lanes' pairs
    combine the same way in five levels: the bound below is that, doubled,
    plus the FP64 steps.
    Weights uniform in [1e10, 9e11], or log-uniform over six decades."""
    rng = np.random.default_rng(11 + cap)
    counts = [0, 1, 31, 32, 33, cap - 1, cap] + [int(v) for v in rng.integers(0, cap + 1, 57)]
    if logw:
        cells = [np.exp(rng.uniform(np.log(1e6), np.log(1e12), k)).astype(np.float32) for k in counts]
    else:
        cells = [rng.uniform(1e10, 9e11, k).astype(np.float32) for k in counts]
    pl = plasma_with_weights(cells, Z3, A3, cap)
    out = torch.full((len(cells) * 3,), -1.0, dtype=torch.float64, device="cuda")
    X = [0.55, 0.3, 0.15]
    rtol = 2.0 * (cap / 32 + 10) * 2.0 ** -48 + 1e-14
    for bind in (-1, 0, 1, 2):
        got = pl.deposit_composition(X if bind < 0 else None, bind, out)
        torch.cuda.synchronize()
        got = got.view(-1, 3).cpu().numpy()
        want = CO.deposit(cells, V, Z3, A3, X=X, bind=bind)
        np.testing.assert_allclose(got, want, rtol=rtol, atol=0.0)
        assert np.all(got[0] == 0.0)
        if bind >= 0:
            assert np.all(np.delete(got, bind, axis=1) == 0.0)
    pl.close()


def test_deposit_into_the_context_rebuilds_the_records():
    """A hydrogen-helium plasma sampled at n_e = 6e25 whose given ion
    densities are wrong: depositing into its own n_ion with X_H recovers the
    cell parameters of the right composition."""
    n = 96
    XH = 0.9 * 1.00794 / (0.9 * 1.00794 + 0.1 * 4.002602)
    n_tot = 6e25 / 1.1
    right = np.tile([[0.9 * n_tot, 0.1 * n_tot]], (n, 1))
    T = np.linspace(1.0, 5.0, n)
    Z, A = [1.0, 2.0], [1.00794, 4.002602]
    ref = AxionPlasma(n, T, right, Z, A, V, (512, 4, 4), PRM)
    ref.sample(512, 0, 0)
    pl = AxionPlasma(n, T, np.full((n, 2), 1e23), Z, A, V, (512, 4, 4), PRM)
    for f in ref.slabs["electrons"].data:
        pl.slabs["electrons"].data[f].copy_(ref.slabs["electrons"].data[f])
    pl.slabs["electrons"].count.copy_(ref.slabs["electrons"].count)
    pl.update_cells()
    pl.deposit_composition([XH, 1 - XH])
    torch.cuda.synchronize()
    cells_w = [ref.slabs["electrons"].cell(c)["w"] for c in range(n)]
    want_n = CO.deposit(cells_w, V, Z, A, X=[XH, 1 - XH])
    np.testing.assert_allclose(pl.n_ion.view(n, 2).cpu().numpy(), want_n, rtol=1e-13)
    np.testing.assert_allclose(want_n, right, rtol=1e-6)      # the binary32 weights
    names = _lib.CELL_INFO_NAMES
    got, exp = pl.cell_info(), ref.cell_info()
    prm = P.Params(g_agg_GeV_inv=1e-10, g_ae=1e-13, dt_phys_s=1e12, w_a=1e9)
    for key in ("rho", "X_H", "n_e", "n_eff", "kappa", "Q_C", "Q_B"):
        k = names.index(key)
        np.testing.assert_allclose(got[:, k], exp[:, k], rtol=2e-6, err_msg=key)
    for c in (0, n // 2, n - 1):
        cs = P.cell_state(T[c], want_n[c], Z, A, prm)
        assert abs(got[c, names.index("X_H")] - cs.X_H) <= 1e-6
        assert abs(got[c, names.index("n_e")] - cs.n_e) <= 1e-6 * cs.n_e
    ref.close()
    pl.close()


def test_invalid_composition_arguments_write_nothing():
    pl = plasma_with_weights([np.ones(4, np.float32)] * 2, Z3, A3, 8)
    out = torch.full((6,), -1.0, dtype=torch.float64, device="cuda")
    for X, bind in ((None, -1), ([0.5, 0.5, 0.5], -1), ([1.2, -0.2, 0.0], -1), ([np.nan, 0.5, 0.5], -1),
                    (None, 3), (None, -2)):
        with pytest.raises(_lib.AxpicError):
            pl.deposit_composition(X, bind, out)
    torch.cuda.synchronize()
    assert torch.all(out == -1.0)
    pl.close()
