"""The spectral surrogate's target function and its MLP, in FP64.

Test infrastructure only (imported by tests/ and smoke()).

What is approximated. For a single-ion plasma of charge Z (n_i = n_e / Z; A
of hydrogen or helium-4), Debye screening, ions as Primakoff targets, and the
axion couplings set to 1 (g_agg = 1 GeV^-1, g_ae = 1: the coupling squared is
factored out), the state (T, n_e, Z) is fixed by (kappa/T, n_e, Z):
T^3 = 4 pi alpha (hbar c)^3 n_e (1 + Z) / (kappa/T)^2 (Sec. II.F, Debye kappa
with n_eff = n_e + Z^2 n_i). At x = omega / T the 96 outputs are, per channel
c in (Primakoff, Compton-like, bremsstrahlung):
* slot 0: ln(dQ_c/dx) in erg cm^-3 s^-1 per unit x, the energy emissivity
  spectrum:
  - Compton-like: Q_C x^5 / (e^x - 1) / (Gamma(6) zeta(6)) (Sec. II.G);
  - bremsstrahlung: Q_B x^a e^-x / Gamma(a + 1) (Sec. II.H), with the two
    [1 - c eta] brackets floored at 1e-3 (the paper's fit turns negative at
    high eta; cells there are outside the trusted region);
  - Primakoff: E Gamma(E) n_gamma(E) T with the screened rate of Eqs.
    prim_xs, prim_rate and the Planck photon density of Sec. II.G.
* slots 1..31: the quantiles x(u_j), u_j = j/32, of the channel's number
  spectrum dQ_c/dx / x restricted to [0.05, 20] (the end points x(0) = 0.05
  and x(1) = 20 are fixed and not outputs).

The model's output is y = shape(x, kappa/T) + mu + S f_c + sigma z
(model_output below). shape is each channel's exact x-dependence on the
ln-emissivity outputs, so the rest is a function of the cell alone: the
network (4 -> 64 -> 64 -> 96, tanh hidden layers) and the FP32 linear map S
(96 x 4) see the cell features f_c = (0, ln(kappa/T), log10 n_e, Z), the
normalised features of the row with the ln x column held at zero, and mu,
sigma are per-output constants.

Pinned by: the Compton-like and bremsstrahlung quantiles against the
closed-form inverse CDFs of the spectra module (Bose integrals, scipy's
incomplete gamma), the emissivity integrals int dQ/dx dx = Q_C, Q_B (scipy
quadrature), the Primakoff spectrum against a direct quadrature of
E Gamma n_gamma, the temperature map against the Debye formula of
plasma.cell_state, and the MLP gradients against central finite differences.
"""
import math

import numpy as np
from scipy import integrate, special

from . import constants as K
from . import plasma, spectra

X_LO, X_HI = 0.05, 20.0
KT_LO, KT_HI = 0.012, 41.0
NE_LO, NE_HI = 1e23, 1e26
T_LO, T_HI = 0.5, 10.0
N_KNOTS = 31
U_KNOTS = np.arange(1, 32) / 32.0
N_OUT = 96
CHANNELS = ("primakoff", "compton", "brems")
LAYERS = (4, 64, 64, 96)


# ------------------------------------------------------------------ domain

def temperature(kT, ne, Z):
    """T [keV] of a single-ion plasma with Debye kappa/T = kT."""
    return (K.FOUR_PI * K.ALPHA_EM * K.HBARC_KEV_CM ** 3 * ne * (1.0 + Z) / kT ** 2) ** (1.0 / 3.0)


def kappa_over_T(T, ne, Z):
    return math.sqrt(K.FOUR_PI * K.ALPHA_EM * K.HBARC_KEV_CM ** 3 * ne * (1.0 + Z) / T ** 3)


def cell(T, ne, Z, brems_shape=1.70):
    """plasma.cell_state of the single-ion plasma with unit couplings."""
    A = K.A_H if Z == 1 else K.A_HE
    p = plasma.Params(g_agg_GeV_inv=1.0, g_ae=1.0, brems_gamma_shape=brems_shape)
    return plasma.cell_state(T, np.array([ne / Z]), np.array([float(Z)]), np.array([A]), p), p


def features(x, kT, ne, Z):
    """Normalised network inputs, each in [-1, 1] on the domain."""
    x, kT, ne, Z = (np.asarray(v, dtype=np.float64) for v in (x, kT, ne, Z))
    f0 = np.log(x / X_LO) / math.log(X_HI / X_LO) * 2.0 - 1.0
    f1 = np.log(kT / KT_LO) / math.log(KT_HI / KT_LO) * 2.0 - 1.0
    f2 = (np.log10(ne) - 24.5) / 1.5
    f3 = Z - 1.5
    return np.stack(np.broadcast_arrays(f0, f1, f2, f3), axis=-1)


def cell_features(X):
    """The features the network and the linear map see: the rows' features
    with the ln x column held at zero."""
    X = np.array(np.atleast_2d(X), dtype=np.float64)
    X[:, 0] = 0.0
    return X


def shape(X, brems_shape=1.70):
    """The fixed part of the model's 96 outputs at feature rows X: on the
    ln-emissivity outputs the channel's x-dependence at fixed cell, in ln
    (Primakoff: x^3/(e^x - 1) F(s), s = 4 x^2/(kappa/T)^2, with the screening
    function F of Eq. prim_F; Compton-like x^5/(e^x - 1); bremsstrahlung
    x^a e^-x); zero on the quantiles. x and kappa/T are recovered from the
    features."""
    X = np.atleast_2d(np.asarray(X, dtype=np.float64))
    x = X_LO * (X_HI / X_LO) ** (0.5 * (X[:, 0] + 1.0))
    kT = KT_LO * (KT_HI / KT_LO) ** (0.5 * (X[:, 1] + 1.0))
    s = 4.0 * x ** 2 / kT ** 2
    out = np.zeros((len(X), N_OUT))
    out[:, 0] = 3.0 * np.log(x) - np.log(np.expm1(x)) + np.log(plasma.primakoff_F(s))
    out[:, 32] = 5.0 * np.log(x) - np.log(np.expm1(x))
    out[:, 64] = brems_shape * np.log(x) - x
    return out


def model_output(z, X, mu, sigma, skip, brems_shape=1.70):
    """y = shape + mu + S f_c + sigma z for normalised network outputs z (the
    network evaluated at cell_features(X)) at feature rows X."""
    X = np.atleast_2d(np.asarray(X, dtype=np.float64))
    return (shape(X, brems_shape) + np.asarray(mu, np.float64) + cell_features(X) @ np.asarray(skip, np.float64).T
            + np.asarray(sigma, np.float64) * z)


# ------------------------------------------------------------------ targets

def _brems_Q_floored(cs, a):
    """Q_B with the [1 - c eta] brackets floored at 1e-3."""
    T7, rho2, X = cs.T7, cs.rho2, cs.X_H
    afac = (1.0 / K.FOUR_PI) / 1.60e-23
    eZ = 0.150 * T7 ** 2.5 * rho2 * (1.0 + X) * afac * max(1e-3, 1.0 - 6.98e-2 * cs.eta)
    ee = 0.150 * T7 ** 2.5 * rho2 * (1.0 + X) ** 2 / (2.0 * math.sqrt(2.0)) * afac * max(1e-3, 1.0 - 0.140 * cs.eta)
    return cs.rho * (eZ + ee)


def emissivity(channel, x, T, ne, Z, brems_shape=1.70):
    """dQ_c/dx [erg cm^-3 s^-1 per unit x] at unit coupling."""
    x = np.asarray(x, dtype=np.float64)
    cs, p = cell(T, ne, Z, brems_shape)
    if channel == "compton":
        return cs.Q_C * x ** 5 / np.expm1(x) / (math.gamma(6.0) * special.zeta(6.0))
    if channel == "brems":
        a = brems_shape
        return _brems_Q_floored(cs, a) * np.exp(a * np.log(x) - x - special.gammaln(a + 1.0))
    if channel == "primakoff":
        E = x * T
        n_gamma = E ** 2 / (math.pi ** 2 * K.HBARC_KEV_CM ** 3) / np.expm1(x)     # per keV per cm^3
        return E * plasma.primakoff_rate(cs, E) * n_gamma * T * K.KEV_ERG
    raise ValueError(channel)


def _number_quantiles(pdf_fn, n_grid=40001):
    """Quantiles u_j of a number pdf on [X_LO, X_HI]: cumulative trapezoid
    sums on a fine grid in ln x (40001 points), then linear inversion of the
    monotone cumulative."""
    t = np.linspace(math.log(X_LO), math.log(X_HI), n_grid)
    x = np.exp(t)
    f = pdf_fn(x) * x                      # d(number)/d(ln x)
    h = t[1] - t[0]
    cum = np.concatenate([[0.0], np.cumsum((f[:-1] + f[1:]) * 0.5 * h)])
    cum /= cum[-1]
    return np.interp(U_KNOTS, cum, x)


def quantiles(channel, T, ne, Z, brems_shape=1.70):
    """x(u_j), j = 1..31, of channel c's number spectrum on [X_LO, X_HI]."""
    if channel == "compton":
        F = spectra.compton_cdf
        lo, hi = F(X_LO), F(X_HI)
        return spectra.compton_icdf(lo + U_KNOTS * (hi - lo))
    if channel == "brems":
        a = brems_shape
        lo, hi = spectra.gamma_cdf(a, X_LO), spectra.gamma_cdf(a, X_HI)
        return spectra.gamma_icdf(a, lo + U_KNOTS * (hi - lo))
    if channel == "primakoff":
        return _number_quantiles(lambda x: emissivity("primakoff", x, T, ne, Z) / x)
    raise ValueError(channel)


def targets(x, kT, ne, Z, brems_shape=1.70):
    """The 96 outputs at one (x, kappa/T, n_e, Z)."""
    T = temperature(kT, ne, Z)
    y = np.empty(N_OUT)
    for c, ch in enumerate(CHANNELS):
        y[32 * c] = math.log(float(emissivity(ch, x, T, ne, Z, brems_shape)))
        y[32 * c + 1:32 * c + 32] = quantiles(ch, T, ne, Z, brems_shape)
    return y


def universal_output(o):
    """Whether output o does not depend on the cell: the Compton-like and
    bremsstrahlung quantiles (their number spectra in x are the same in every
    cell), o = 33..63 and 65..95."""
    return o > 32 and o % 32 != 0


def cell_constants(z, X, mu, sigma, skip, brems_shape=1.70):
    """A cell's three ln-emissivity constants c_c = y_c - shape_c (c = Primakoff,
    Compton-like, bremsstrahlung; outputs 0, 32, 64 of model_output), x-
    independent by construction of the model."""
    y = model_output(z, X, mu, sigma, skip, brems_shape)
    sh = shape(X, brems_shape)
    return (y - sh)[:, [0, 32, 64]]


def network_cell_state(cs, c, p):
    """The cell's rate parameters under the surrogate rate model where the
    network is trusted: every channel keeps its closed functional form and the
    network's constants c = (c_P, c_C, c_B) (ln-emissivity at unit coupling
    minus the exact x-shape) set the prefactors:
    * Primakoff (Eq. prim_rate with Planck photons): dQ_P/dx = Gamma_0 T^4 keV
      x^3 F(s) / (pi^2 (hbar c)^3 (e^x - 1)), so Gamma_0 = g^2 e^c_P pi^2
      (hbar c)^3 / (T^4 keV);
    * Compton-like: dQ_C/dx = Q_C x^5 / (e^x - 1) / (Gamma(6) zeta(6)), so Q_C =
      g_ae^2 e^c_C Gamma(6) zeta(6);
    * bremsstrahlung: Q_B = g_ae^2 e^c_B Gamma(a + 1);
    and Gamma_C, Gamma_B = Q / (n_e <E>) as in Eqs. GammaC and the text after
    eps_ee (the absorption rates follow from them, Eq. gamma_abs)."""
    import copy
    out = copy.copy(cs)
    a = p.brems_gamma_shape
    T = cs.T_keV
    out.Gamma0_P = (p.g_agg_GeV_inv ** 2 * math.exp(c[0]) * math.pi ** 2 * K.HBARC_KEV_CM ** 3
                    / (T ** 4 * K.KEV_ERG))
    out.Q_C = p.g_ae ** 2 * math.exp(c[1]) * math.gamma(6.0) * special.zeta(6.0)
    out.Q_B = p.g_ae ** 2 * math.exp(c[2]) * math.gamma(a + 1.0)
    out.Gamma_C = out.Q_C / (cs.n_e * spectra.compton_mean_x() * T * K.KEV_ERG) if cs.n_e > 0 else 0.0
    out.Gamma_B = out.Q_B / (cs.n_e * a * T * K.KEV_ERG) if cs.n_e > 0 else 0.0
    return out


def in_domain(kT, ne, Z):
    T = temperature(kT, ne, Z)
    return T_LO <= T <= T_HI and NE_LO <= ne <= NE_HI


# ------------------------------------------------------------------ MLP

def init_params(rng):
    """Glorot-uniform weights, zero biases (FP64)."""
    P = {}
    for i, (a, b) in enumerate(zip(LAYERS[:-1], LAYERS[1:]), start=1):
        lim = math.sqrt(6.0 / (a + b))
        P["W%d" % i] = rng.uniform(-lim, lim, (a, b))
        P["b%d" % i] = np.zeros(b)
    return P


def bf16(a):
    """Round to bfloat16 (round to nearest, ties to even), returned as FP64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(P, X, bf16_mma=False):
    """Normalised outputs z and the cache for backward. With bf16_mma the
    operands of layers 2 and 3 are rounded to bfloat16 (the GPU's tensor-core
    inputs); accumulation stays FP64."""
    q = bf16 if bf16_mma else (lambda a: a)
    a1 = X @ P["W1"] + P["b1"]
    h1 = np.tanh(a1)
    a2 = q(h1) @ q(P["W2"]) + P["b2"]
    h2 = np.tanh(a2)
    z = q(h2) @ q(P["W3"]) + P["b3"]
    return z, (X, h1, h2)


def loss(P, X, Zt, bf16_mma=False):
    """Mean over samples of the summed squared error of the normalised
    outputs."""
    z, _ = forward(P, X, bf16_mma)
    return float(np.sum((z - Zt) ** 2) / len(X))


def backward(P, X, Zt, bf16_mma=False):
    """Gradients of loss() with respect to every parameter (the bfloat16
    rounding, when on, is treated as identity in the derivative, as the GPU's
    straight-through training does)."""
    q = bf16 if bf16_mma else (lambda a: a)
    z, (X, h1, h2) = forward(P, X, bf16_mma)
    n = len(X)
    dz = 2.0 * (z - Zt) / n
    G = {"W3": q(h2).T @ q(dz), "b3": dz.sum(0)}
    dh2 = q(dz) @ q(P["W3"]).T
    da2 = dh2 * (1.0 - h2 ** 2)
    G["W2"] = q(h1).T @ q(da2)
    G["b2"] = da2.sum(0)
    dh1 = q(da2) @ q(P["W2"]).T
    da1 = dh1 * (1.0 - h1 ** 2)
    G["W1"] = X.T @ da1
    G["b1"] = da1.sum(0)
    return G


def adam(P, G, M, V, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (bias-corrected moments) in place; t counts from 1."""
    for k in P:
        M[k] = b1 * M[k] + (1.0 - b1) * G[k]
        V[k] = b2 * V[k] + (1.0 - b2) * G[k] ** 2
        mh = M[k] / (1.0 - b1 ** t)
        vh = V[k] / (1.0 - b2 ** t)
        P[k] = P[k] - lr * mh / (np.sqrt(vh) + eps)


# ------------------------------------------------------------------ spectral records
# A cell's spectral record under the table rate model: ln(dQ_c/dx) + x at unit
# coupling (the Boltzmann factor taken out, so that the spline in ln x is
# accurate to ~1e-4 at large x) on x_k = 0.05 e^((k - 1) h), h = ln(400) / 29, k = 0..31 (c * 32 +
# k; x_1 = 0.05 and x_30 = 20, one point beyond each end so that the spline
# has real neighbours everywhere in [0.05, 20]), the quantiles (96 +
# c * 31 + j - 1), ln(g_agg^2 dt pi^2 (hbar c)^3 / (T^4 keV)),
# ln(g_ae^2 dt 2 pi^2 (hbar c)^3 / (T^4 keV)) and T. The table holds the
# targets at nodes uniform in ln(kappa/T) on [ln 0.012, ln 41] and in
# log10 n_e on [23, 26], for Z = 1 and 2, stored in binary32; a cell's record
# is bilinear in (ln kappa/T, log10 n_e) at its Z. The bremsstrahlung row is
# tabulated with the fit's brackets divided out (ln_brackets below) and a
# cell's record adds them back for its own eta: the brackets' 1e-3 floor puts
# a kink into ln Q_B, which bilinear interpolation across it would smear.

SR_LEN = 192
GRID_H = math.log(X_HI / X_LO) / 29.0
X_GRID = np.exp(np.log(X_LO) + GRID_H * (np.arange(32) - 1.0))


def ln_brackets(eta, Z):
    """ln of the bremsstrahlung fit's brackets (Eqs. eps_eZ, eps_ee), each
    floored at 1e-3 and weighted as in Q_B, normalised to 1 at eta = 0:
    ln((b_eZ + c b_ee) / (1 + c)), c = (1 + X_H) / (2 sqrt 2), X_H = 1 for
    hydrogen (Z = 1), 0 for helium."""
    XH = 1.0 if Z == 1 else 0.0
    c = (1.0 + XH) / (2.0 * math.sqrt(2.0))
    bz = max(1e-3, 1.0 - 6.98e-2 * eta)
    be = max(1e-3, 1.0 - 0.140 * eta)
    return math.log((bz + c * be) / (1.0 + c))


def build_table(nkt, nne, brems_shape=1.70):
    tab = np.empty((2, nne, nkt, 189), dtype=np.float32)
    for z in range(2):
        for j in range(nne):
            for i in range(nkt):
                kT = math.exp(math.log(KT_LO) + math.log(KT_HI / KT_LO) * i / (nkt - 1))
                ne = 10.0 ** (23.0 + 3.0 * j / (nne - 1))
                Z = z + 1
                T = temperature(kT, ne, Z)
                lnbr = ln_brackets(cell(T, ne, Z, brems_shape)[0].eta, Z)
                for c, ch in enumerate(CHANNELS):
                    tab[z, j, i, 32 * c:32 * c + 32] = (np.log(emissivity(ch, X_GRID, T, ne, Z, brems_shape)) + X_GRID
                                                        - (lnbr if ch == "brems" else 0.0))
                    tab[z, j, i, 96 + 31 * c:96 + 31 * c + 31] = quantiles(ch, T, ne, Z, brems_shape)
    return tab


def table_record(tab, T, kappa, ne, Z, g_agg, g_ae, dt):
    """The cell's record from the table (bilinear, clamped to the grid)."""
    nne, nkt = tab.shape[1], tab.shape[2]
    kT = kappa / T
    u = (math.log(kT) - math.log(KT_LO)) / math.log(KT_HI / KT_LO) * (nkt - 1)
    v = (math.log10(ne) - 23.0) / 3.0 * (nne - 1)
    u = min(max(u, 0.0), nkt - 1.0)
    v = min(max(v, 0.0), nne - 1.0)
    i, j = min(int(u), nkt - 2), min(int(v), nne - 2)
    fu, fv = u - i, v - j
    t = tab[int(Z) - 1].astype(np.float64)
    rec = np.empty(SR_LEN)
    rec[:189] = ((1 - fv) * ((1 - fu) * t[j, i] + fu * t[j, i + 1]) + fv * ((1 - fu) * t[j + 1, i] + fu * t[j + 1, i + 1]))
    rec[64:96] += ln_brackets(cell(T, ne, Z)[0].eta, Z)
    hc3 = K.HBARC_KEV_CM ** 3
    rec[189] = math.log(g_agg ** 2 * dt * math.pi ** 2 * hc3 / K.KEV_ERG) - 4.0 * math.log(T)
    rec[190] = math.log(g_ae ** 2 * dt * 2.0 * math.pi ** 2 * hc3 / K.KEV_ERG) - 4.0 * math.log(T)
    rec[191] = T
    return rec


def rec_lnL(rec, ch, x):
    """ln(dQ_c/dx) at x in [0.05, 20] (clamped there): Catmull-Rom in ln x
    through the record's 32 values of ln(dQ_c/dx) + x, minus x."""
    x = np.asarray(x, dtype=np.float64)
    u = (np.log(x) - math.log(X_LO)) / GRID_H + 1.0
    u = np.clip(u, 1.0, 30.0)
    k = np.minimum(u.astype(np.int64), 29)
    f = u - k
    g = rec[32 * ch:32 * ch + 32]
    p0, p1, p2, p3 = g[k - 1], g[k], g[k + 1], g[k + 2]
    s = p1 + 0.5 * f * (p2 - p0 + f * (2 * p0 - 5 * p1 + 4 * p2 - p3 + f * (3 * (p1 - p2) + p3 - p0)))
    return s - np.clip(x, X_LO, X_HI)


def rec_prim_gdt(rec, x):
    """Gamma_{gamma->a} dt (multiplicity 1) from the record: the Primakoff
    emissivity divided by E T n_gamma(E) (Eq. prim_rate with Planck photons)."""
    x = np.asarray(x, dtype=np.float64)
    return np.exp(rec_lnL(rec, 0, x) + rec[189] - 3 * np.log(x)) * np.expm1(x)


def rec_tau(rec, ch, x, eq_stats):
    """tau_c = Gamma_abs,c dt from the record (Eq. gamma_abs: the emission rate
    per energy over the equilibrium density)."""
    x = np.asarray(x, dtype=np.float64)
    b = np.exp(rec_lnL(rec, ch, x) + rec[190] - 3 * np.log(x))
    return b * (np.expm1(x) if eq_stats else np.exp(x))


def rec_sample_x(rec, ch, u):
    """x from the record's quantiles of channel ch, linear between quantiles
    with the end points 0.05 and 20."""
    u = np.asarray(u, dtype=np.float64)
    q = np.concatenate([[X_LO], rec[96 + 31 * ch:96 + 31 * ch + 31], [X_HI]])
    t = u * 32.0
    j = np.minimum(t.astype(np.int64), 31)
    return q[j] + (t - j) * (q[j + 1] - q[j])
