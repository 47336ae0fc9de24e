"""Pins of the surrogate's target function and of the FP64 MLP (no GPU)."""
import math

import numpy as np
import pytest
from scipy import integrate, optimize, special

from oracle import constants as K
from oracle import plasma, surrogate as S


def test_temperature_map_is_debye():
    for T, ne, Z in [(0.5, 1e26, 2), (3.0, 6e25, 1), (10.0, 1e23, 1), (1.7, 3e24, 2)]:
        kT = S.kappa_over_T(T, ne, Z)
        assert abs(S.temperature(kT, ne, Z) - T) <= 1e-12 * T
        cs, _ = S.cell(T, ne, Z)
        assert abs(cs.kappa_keV / T - kT) <= 1e-12 * kT
        assert abs(cs.n_e - ne) <= 1e-12 * ne
    # the domain corners quoted for the surrogate
    assert 0.011 < S.kappa_over_T(10.0, 1e23, 1) < 0.013
    assert 40.0 < S.kappa_over_T(0.5, 1e26, 2) < 42.0


def _quantiles_by_quad(pdf, lo=S.X_LO, hi=S.X_HI):
    tot = integrate.quad(pdf, lo, hi, limit=200, epsabs=0, epsrel=1e-12)[0]
    out = []
    for u in S.U_KNOTS:
        f = lambda x: integrate.quad(pdf, lo, x, limit=200, epsabs=0, epsrel=1e-12)[0] / tot - u
        out.append(optimize.brentq(f, lo, hi, xtol=1e-13, rtol=1e-13))
    return np.array(out)


def test_compton_and_brems_quantiles_by_quadrature():
    q_c = S.quantiles("compton", 3.0, 6e25, 1)
    want = _quantiles_by_quad(lambda x: x ** 4 / math.expm1(x))
    np.testing.assert_allclose(q_c, want, rtol=1e-9)
    for a in (1.70, 1.4):
        q_b = S.quantiles("brems", 3.0, 6e25, 1, brems_shape=a)
        want = _quantiles_by_quad(lambda x: x ** (a - 1.0) * math.exp(-x))
        np.testing.assert_allclose(q_b, want, rtol=1e-9)


@pytest.mark.parametrize("T,ne,Z", [(3.0, 6e25, 1), (0.7, 1e26, 2), (9.0, 2e23, 1)])
def test_primakoff_quantiles_by_quadrature(T, ne, Z):
    cs, _ = S.cell(T, ne, Z)
    k = cs.kappa_keV / T

    def pdf(x):  # number spectrum: x^2 F(4 x^2 / (kappa/T)^2) / (e^x - 1), up to constants
        s = 4.0 * x * x / (k * k)
        F = (1.0 + 1.0 / s) * math.log1p(s) - 1.0 if s > 1e-4 else s / 2 - s * s / 6 + s ** 3 / 12
        return x * x * F / math.expm1(x)
    np.testing.assert_allclose(S.quantiles("primakoff", T, ne, Z), _quantiles_by_quad(pdf), rtol=2e-6)


def test_emissivity_integrals():
    T, ne, Z = 3.0, 6e25, 1
    cs, p = S.cell(T, ne, Z)
    for ch, Q in (("compton", cs.Q_C), ("brems", cs.Q_B)):
        tot = integrate.quad(lambda x: float(S.emissivity(ch, x, T, ne, Z)), 0.0, 80.0, limit=400,
                             epsabs=0, epsrel=1e-11)[0]
        assert abs(tot - Q) <= 1e-8 * Q, (ch, tot, Q)
    # unit couplings: the emissivities scale with g^2 (Eqs. epsC, prim_xs)
    p2 = plasma.Params(g_agg_GeV_inv=1e-10, g_ae=1e-13)
    cs2 = plasma.cell_state(T, np.array([ne]), np.array([1.0]), np.array([K.A_H]), p2)
    assert abs(cs2.Q_C / cs.Q_C - 1e-26) <= 1e-12 * 1e-26
    assert abs(cs2.Gamma0_P / cs.Gamma0_P - 1e-20) <= 1e-12 * 1e-20


def test_primakoff_emissivity_limits():
    """dQ_P/dx = E Gamma(E) n_gamma(E) T: at x << kappa/T, F -> s/2 (s = 4
    x^2 / (kappa/T)^2), at x >> kappa/T, F -> ln s - 1."""
    T, ne, Z = 3.0, 6e25, 1
    cs, _ = S.cell(T, ne, Z)
    k = cs.kappa_keV / T
    pre = cs.Gamma0_P * T ** 5 / (math.pi ** 2 * K.HBARC_KEV_CM ** 3) * K.KEV_ERG
    for x, Flim, tol in ((1e-3 * k, lambda s: s / 2, 1e-5), (300 * k, lambda s: math.log(s) - 1, 1e-4)):
        if not (S.X_LO <= x <= 60.0):
            continue
        s = 4 * x * x / (k * k)
        want = pre * x ** 3 / math.expm1(x) * Flim(s)
        got = float(S.emissivity("primakoff", x, T, ne, Z))
        assert abs(got - want) <= tol * want * 10, (x, got, want)


def test_targets_layout():
    y = S.targets(2.0, S.kappa_over_T(3.0, 6e25, 1), 6e25, 1)
    assert y.shape == (96,)
    for c in range(3):
        knots = y[32 * c + 1:32 * c + 32]
        assert np.all(np.diff(knots) > 0) and knots[0] > S.X_LO and knots[-1] < S.X_HI
        assert np.isfinite(y[32 * c])
    # Compton and brems knots do not depend on the plasma
    y2 = S.targets(0.3, S.kappa_over_T(1.0, 1e24, 2), 1e24, 2)
    np.testing.assert_allclose(y[33:96][np.r_[0:31, 32:63]], y2[33:96][np.r_[0:31, 32:63]], rtol=1e-12)


def _residual(ch, x, T, ne, Z):
    """ln-emissivity of a channel minus the model's fixed x-shape."""
    kT = S.kappa_over_T(T, ne, Z)
    X = S.features(x, kT, ne, Z)
    o = {"primakoff": 0, "compton": 32, "brems": 64}[ch]
    return np.log(S.emissivity(ch, x, T, ne, Z)) - S.shape(X)[:, o], X


def test_shapes_leave_cell_constants():
    """Each channel's x-shape is its spectrum's exact x-dependence: what it
    leaves is constant in x (for Primakoff over s = 4x^2/(kappa/T)^2 from
    below 1e-5 to above 1e6, both limits of F and its series branch). For
    Compton-like and Primakoff that constant is linear in the cell features
    (ln Q_C = ln n_e + 6 ln T + const; the Primakoff factor is n_i Z^2 T^4
    times constants; ln T is linear in ln n_e and ln(kappa/T), and Z takes two
    values), so the FP32 linear map carries both rates exactly."""
    x = np.geomspace(S.X_LO, S.X_HI, 400)
    rows, Yc, Yp = [], [], []
    for T, ne, Z in ((0.7, 2e23, 1), (3.0, 6e25, 1), (9.0, 1e24, 2), (1.5, 5e25, 2), (5.0, 3e23, 1),
                     (2.2, 8e24, 2), (6.5, 2e25, 1), (0.5, 1e26, 2), (10.0, 1e23, 1)):
        for ch in ("primakoff", "compton", "brems"):
            r, X = _residual(ch, x, T, ne, Z)
            assert np.ptp(r) < 1e-11 * max(1.0, np.abs(r).max()), (ch, T, ne, Z, np.ptp(r))
        rows.append(np.r_[1.0, S.cell_features(X[:1])[0, 1:]])
        Yc.append(_residual("compton", x[:1], T, ne, Z)[0][0])
        Yp.append(_residual("primakoff", x[:1], T, ne, Z)[0][0])
    A = np.array(rows)
    for Y in (Yc, Yp):
        c, *_ = np.linalg.lstsq(A, np.array(Y), rcond=None)
        assert np.abs(A @ c - np.array(Y)).max() < 1e-9


def test_primakoff_shape_spans_both_screening_limits():
    """The s range of the domain's rows reaches both limits of F: s/2 (weak
    screening) and ln s - 1 (strong), where a bound such as min(s/2, ln(1+s))
    would leave an x-dependent residual of up to ln 0.6."""
    X = S.features(np.array([S.X_LO, S.X_HI]), np.array([S.KT_HI, S.KT_LO]), 1e25, 1)
    x = S.X_LO * (S.X_HI / S.X_LO) ** (0.5 * (X[:, 0] + 1.0))
    kT = S.KT_LO * (S.KT_HI / S.KT_LO) ** (0.5 * (X[:, 1] + 1.0))
    s = 4 * x ** 2 / kT ** 2
    assert s[0] < 1e-5 and s[1] > 1e6
    F = plasma.primakoff_F(s)
    assert abs(F[0] / (s[0] / 2) - 1) < 1e-5 and abs(F[1] / (np.log(s[1]) - 1) - 1) < 1e-5


def test_model_output_depends_on_x_only_through_the_shape():
    """The learned part (mu + S f_c + sigma z) sees the cell features: rows of
    one cell at different x differ by the shapes alone, whatever S holds in
    its ln x column."""
    rng = np.random.default_rng(3)
    X = S.features(np.array([0.1, 2.0, 15.0]), 0.9, 3e24, 2)
    mu, sigma, skip = rng.normal(size=96), rng.uniform(0.5, 2, 96), rng.normal(size=(96, 4))
    P = S.init_params(rng)
    z, _ = S.forward(P, S.cell_features(X))
    assert np.ptp(z, axis=0).max() == 0.0
    y = S.model_output(z, X, mu, sigma, skip) - S.shape(X)
    assert np.ptp(y, axis=0).max() < 1e-12


def test_features_span_the_domain():
    f = S.features([S.X_LO, S.X_HI], [S.KT_LO, S.KT_HI], [S.NE_LO, S.NE_HI], [1, 2])
    np.testing.assert_allclose(f[:, :3], [[-1, -1, -1], [1, 1, 1]], atol=1e-12)
    assert list(f[:, 3]) == [-0.5, 0.5]


@pytest.mark.parametrize("bf", [False, True])
def test_mlp_gradients_by_finite_differences(bf):
    rng = np.random.default_rng(5)
    P = S.init_params(rng)
    for k in P:
        if k.startswith("b"):
            P[k] = rng.normal(0, 0.1, P[k].shape)
    X = rng.uniform(-1, 1, (7, 4))
    Zt = rng.normal(0, 1, (7, 96))
    G = S.backward(P, X, Zt)
    h = 1e-6
    for k in P:
        flat = P[k].reshape(-1)
        for i in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[i]
            flat[i] = old + h
            lp = S.loss(P, X, Zt)
            flat[i] = old - h
            lm = S.loss(P, X, Zt)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            g = G[k].reshape(-1)[i]
            assert abs(g - fd) <= 1e-6 * max(1.0, abs(fd)), (k, i, g, fd)
    if bf:
        # the bfloat16-operand forward stays within bfloat16 resolution
        z0, _ = S.forward(P, X)
        z1, _ = S.forward(P, X, bf16_mma=True)
        assert np.max(np.abs(z1 - z0)) <= 0.05 * max(1.0, np.max(np.abs(z0)))


def test_bf16_rounding():
    # ties to even and exact values
    assert S.bf16(1.0) == 1.0
    assert S.bf16(1.0 + 2 ** -8) == 1.0          # tie: rounds to even (1.0)
    assert S.bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6
    assert S.bf16(-3.0) == -3.0


def test_adam_first_step():
    """A first Adam step moves each parameter by lr * sign(g) (bias
    correction makes m_hat = g and v_hat = g^2)."""
    P = {"w": np.array([1.0, -2.0, 0.5])}
    G = {"w": np.array([0.3, -4.0, 1e-3])}
    M = {"w": np.zeros(3)}
    V = {"w": np.zeros(3)}
    S.adam(P, G, M, V, 1, 0.01)
    np.testing.assert_allclose(P["w"], [1.0 - 0.01, -2.0 + 0.01, 0.5 - 0.01], rtol=1e-6)


@pytest.mark.parametrize("T,ne,Z", [(3.0, 6e25, 1), (1.4, 2e24, 2), (8.0, 5e23, 1)])
def test_network_cell_state_with_exact_constants_is_the_closed_forms(T, ne, Z):
    """The surrogate model's rates where the network is trusted keep the
    closed functional forms with the network's per-cell constants as
    prefactors: given the exact constants (the targets' ln-emissivity minus
    the shape, the same at every x), network_cell_state gives back the
    closed-form Gamma_0 (Eq. prim_rate), Q_C, Q_B and Gamma_C, Gamma_B
    (Eqs. QC, GammaC and the text after eps_ee), for any coupling."""
    A = K.A_H if Z == 1 else K.A_HE
    p = plasma.Params(g_agg_GeV_inv=3e-10, g_ae=2e-13, dt_phys_s=1.0)
    cs = plasma.cell_state(T, np.array([ne / Z]), np.array([float(Z)]), np.array([A]), p)
    assert cs.eps_eZ > 0 and cs.eps_ee > 0  # brackets above their floors: the targets' floor is moot
    kT = cs.kappa_keV / T
    c = []
    for x in (0.3, 2.0, 7.0):
        X = S.features(x, kT, ne, Z)[None, :]
        y = S.targets(x, kT, ne, Z)
        c.append([y[o] - S.shape(X)[0, o] for o in (0, 32, 64)])
    c = np.array(c)
    np.testing.assert_allclose(c, np.broadcast_to(c[0], c.shape), rtol=0, atol=1e-10)
    net = S.network_cell_state(cs, c[0], p)
    for f in ("Gamma0_P", "Q_C", "Q_B", "Gamma_C", "Gamma_B"):
        assert abs(getattr(net, f) / getattr(cs, f) - 1) < 1e-10, f
    # and a constant off by d scales the channel's rate by e^d
    net2 = S.network_cell_state(cs, c[0] + np.array([0.0, 0.0, 1e-3]), p)
    assert abs(net2.Gamma_B / cs.Gamma_B - math.exp(1e-3)) < 1e-12
    assert net2.Gamma_C == net.Gamma_C and net2.Gamma0_P == net.Gamma0_P
