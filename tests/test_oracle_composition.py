"""The composition oracle against textbook relations and the cell-parameter
oracle (no GPU)."""
import numpy as np

from oracle import composition as CO
from oracle import plasma as P
from oracle.constants import M_U_G

A_H, A_HE = 1.00794, 4.002602


def test_hydrogen_helium_with_integer_masses_gives_textbook_n_e():
    """With A_H = 1 and A_He = 4 a fully ionised H-He plasma has
    n_e = (rho / m_u)(1 + X_H) / 2."""
    for XH in (0.0, 0.3, 0.7, 1.0):
        n = CO.from_mass_fractions(6e25, [1, 2], [1, 4], [XH, 1 - XH])
        rho_over_mu = n[0] * 1 + n[1] * 4
        assert abs(6e25 - rho_over_mu * (1 + XH) / 2) <= 1e-14 * 6e25


def test_round_trip_through_the_cell_parameters():
    """The composition put back into the cell-parameter oracle returns the
    deposited n_e and the given X_H, with rho = sum n_i A_i m_u."""
    prm = P.Params(g_agg_GeV_inv=1e-10, g_ae=1e-13, dt_phys_s=1e12, w_a=1.0)
    for XH in (0.25, 0.6938, 1.0):
        n = CO.from_mass_fractions(6e25, [1, 2], [A_H, A_HE], [XH, 1 - XH])
        cs = P.cell_state(3.0, n, [1, 2], [A_H, A_HE], prm)
        assert abs(cs.n_e - 6e25) <= 1e-14 * 6e25
        assert abs(cs.X_H - XH) <= 1e-14
        assert abs(cs.rho - (n[0] * A_H + n[1] * A_HE) * M_U_G) <= 1e-14 * cs.rho


def test_relaxation_plasma_is_recovered_from_its_electrons():
    """90 % hydrogen and 10 % helium by number with n_e = 6e25: 512 equal
    electron weights n_e V / 512 deposit n_e, and its mass fraction gives the
    number fractions back."""
    V = 1e-12
    n_tot = 6e25 / 1.1
    XH = 0.9 * A_H / (0.9 * A_H + 0.1 * A_HE)
    w = np.full(512, np.float32(6e25 * V / 512))
    n_e = CO.deposited_electron_density(w, V)
    assert abs(n_e - 6e25) <= 1e-6 * 6e25          # the binary32 weight
    n = CO.deposit([w], V, [1, 2], [A_H, A_HE], X=[XH, 1 - XH])[0]
    np.testing.assert_allclose(n / (n_e / 6e25), [0.9 * n_tot, 0.1 * n_tot], rtol=1e-13)


def test_bound_species_and_quasi_neutrality():
    """Every composition is quasi-neutral; a bound species carries it all."""
    Z, A = [1, 2, 6], [A_H, A_HE, 12.011]
    rng = np.random.default_rng(3)
    for _ in range(20):
        n_e = rng.uniform(1e22, 1e26)
        X = rng.dirichlet([1, 1, 1])
        n = CO.from_mass_fractions(n_e, Z, A, X)
        assert abs(np.dot(Z, n) - n_e) <= 1e-14 * n_e
        np.testing.assert_allclose(n * A / np.sum(n * A), X, rtol=1e-13, atol=1e-16)
        for k in range(3):
            b = CO.bound_to_species(n_e, Z, k)
            assert abs(np.dot(Z, b) - n_e) <= 1e-15 * n_e and np.count_nonzero(b) == 1


def test_deposit_sums_the_weights_of_each_cell():
    """n_e is the sum of the cell's weights over V; an empty cell deposits 0."""
    V = 2e-12
    cells = [np.array([], np.float32), np.array([2.0 ** 40, 3 * 2.0 ** 40], np.float32),
             np.full(7, 2.0 ** 39, np.float32)]
    n = CO.deposit(cells, V, [1], [A_H], bind=0)
    np.testing.assert_array_equal(n[:, 0], [0.0, 2.0 ** 42 / V, 7 * 2.0 ** 39 / V])
