"""One time step of the axion Monte-Carlo operators on one cell, plain FP64.

Test infrastructure only (imported by tests/, smoke() and bench.py's CPU
baseline). Nothing here is blocked, fused or reordered: each operator is
applied to the cell's particle lists in the order the step defines.

Operators and the passages they follow:
* absorb_cell  - Primakoff a->gamma (Sec. II.F.1, last paragraph) and the
  detailed-balance absorption of the thermal-bath channels (Sec. II.I,
  Eq. gamma_abs, P_abs = 1 - exp(-Gamma_abs dt)).
* emit_cell    - Primakoff gamma->a on photons (Sec. II.F, Eqs. prim_rate,
  prim_prob, lambda_P, weight depletion) and Compton-like / bremsstrahlung
  emission on electrons (Sec. II.D.1 Eq. lambda_macro, II.D.2 Eqs. lambda_eff,
  wa_rescaled, II.G, II.H).
* feedback_cell - cell moments, affine remap and temperature relaxation
  (Sec. II.J, Eqs. cell_moments to b_def, Te_est, Te_relax).
* init_cell    - the synthetic initial plasma (NR Maxwellian electrons, Planck
  photons at T_e, optional MB-equilibrium axions).

Readings of the paper that both implementations share (the paper is silent on
each): step order absorb -> emit -> feedback; Philox4x32-10 counters
(step, cell, particle, stream<<24 | sub); decisions use one 32-bit word per
particle, word (i & 3) of block (i >> 2); event j of particle i uses block
(step, cell, i, stream<<24 | j) with words (cos theta, phi, energy); new axions
are made photon products first (photon order), then electron products
(electron order, then event order; an electron's two thermal-bath channels are
drawn as one superposed Poisson process and each event is attributed to a
channel by a further uniform); weights are binary32 quantities and depletion
is evaluated in binary32 because it decides whether the parent survives.

Slot order (the paper fixes none; both implementations share this one):
* a separate absorb or emit call (absorb_cell, emit_cell) appends its new
  particles after the survivors and closes its holes by the tail fill (holes
  below the survivor count take, in ascending order, the survivors found at or
  beyond it);
* a full step (step_cell) does the same for the photons (a->gamma products
  appended in the absorb phase, holes of the emit phase closed by the tail
  fill), while the axion slots freed in the absorb phase are reused by the
  axions made in the emit phase: the freed slots, in ascending order, take the
  new axions in the order they are made; new axions beyond them are appended
  after the old count, and freed slots left over are closed by the tail fill.
"""
import math
from dataclasses import dataclass, field

import numpy as np
from scipy import special

from . import constants as K
from . import spectra
from .philox import philox4x32_10, uniform23, split_seed
from .plasma import Params, CellState, primakoff_F, absorption_rate, cell_state
from . import surrogate
from .poisson import cap_lambda, poisson_count

CH_PRIMAKOFF = 1
CH_COMPTON = 2
CH_BREMS = 4

STREAM_PRIM_FWD = 0
STREAM_EMIT_E = 1      # thermal-bath emission decision of an electron (both channels)
STREAM_PRIM_INV = 3
STREAM_ABSORB = 4
STREAM_EV_E = 5        # thermal-bath emission event (direction, energy, channel)
STREAM_INIT_E = 8
STREAM_INIT_G = 9
STREAM_INIT_A = 10
INIT_STEP = 0xFFFFFFFF

F32 = np.float32


@dataclass
class Species:
    """One species' particles in a cell, in slot order; p in m_e c, positions in cell units."""
    w: np.ndarray
    px: np.ndarray
    py: np.ndarray
    pz: np.ndarray
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray

    @staticmethod
    def empty():
        e = np.zeros(0)
        return Species(e.copy(), e.copy(), e.copy(), e.copy(), e.copy(), e.copy(), e.copy())

    def __len__(self):
        return len(self.w)

    def fields(self):
        return [self.w, self.px, self.py, self.pz, self.x, self.y, self.z]

    def take(self, idx):
        return Species(*[f[idx] for f in self.fields()])

    def concat(self, other):
        return Species(*[np.concatenate([a, b]) for a, b in zip(self.fields(), other.fields())])

    def copy(self):
        return Species(*[f.copy() for f in self.fields()])

    def pmag(self):
        return np.sqrt(self.px ** 2 + self.py ** 2 + self.pz ** 2)


@dataclass
class StepTally:
    """Per-cell bookkeeping of one step (energies in keV, momenta in m_e c)."""
    dE: float = 0.0
    dP: np.ndarray = field(default_factory=lambda: np.zeros(3))
    gross_E: float = 0.0          # sum of |contributions| to dE (for error bounds)
    gross_P: float = 0.0          # sum of |contributions| to dP
    events: dict = field(default_factory=lambda: {"prim": 0, "compton": 0, "brems": 0, "prim_inv": 0})
    absorbed: dict = field(default_factory=lambda: {"compton": 0, "brems": 0})
    cap_hits: int = 0
    clamp_hits: int = 0
    n_g0: int = 0
    new_axion_channel: np.ndarray = field(default_factory=lambda: np.zeros(0, dtype=np.int64))
    new_axion_E: np.ndarray = field(default_factory=lambda: np.zeros(0))


def _key(p: Params):
    return split_seed(p.seed)


def decision_uniforms(p: Params, step, cell, stream, n):
    """u_i for particles i < n: word (i & 3) of block (step, cell, i >> 2, stream << 24)."""
    if n == 0:
        return np.zeros(0)
    nq = (n + 3) // 4
    ctr = np.zeros((nq, 4), dtype=np.uint32)
    ctr[:, 0] = np.uint32(step & 0xFFFFFFFF)
    ctr[:, 1] = np.uint32(cell)
    ctr[:, 2] = np.arange(nq, dtype=np.uint32)
    ctr[:, 3] = np.uint32(stream << 24)
    return uniform23(philox4x32_10(ctr, _key(p)).reshape(-1)[:n])


def event_uniforms(p: Params, step, cell, stream, idx, sub):
    """Four uniforms of block (step, cell, idx, stream << 24 | sub), shape (m, 4)."""
    idx = np.asarray(idx, dtype=np.int64)
    m = len(idx)
    ctr = np.zeros((m, 4), dtype=np.uint32)
    ctr[:, 0] = np.uint32(step & 0xFFFFFFFF)
    ctr[:, 1] = np.uint32(cell)
    ctr[:, 2] = idx.astype(np.uint32)
    ctr[:, 3] = (np.uint32(stream << 24) | np.asarray(sub, dtype=np.uint32))
    return uniform23(philox4x32_10(ctr, _key(p)))


def isotropic(u_cos, u_phi):
    """Unit vectors with cos(theta) = 2u - 1 and phi = 2 pi u."""
    ct = 2.0 * u_cos - 1.0
    st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
    ph = 2.0 * math.pi * u_phi
    return st * np.cos(ph), st * np.sin(ph), ct


def tail_fill(keep):
    """New slot -> old index after removing ~keep: holes below the survivor
    count take, in ascending order, the survivors found at or beyond it."""
    keep = np.asarray(keep, dtype=bool)
    ns = int(keep.sum())
    idx = np.arange(len(keep))
    order = np.arange(ns)
    holes = idx[:ns][~keep[:ns]]
    movers = idx[ns:][keep[ns:]]
    order[holes] = movers
    return order


def recycle(s: Species, keep, new: Species):
    """Axion slots after a full step: the slots freed earlier in the step
    (~keep, ascending) take the new particles in order; new particles beyond
    them are appended after the old count; freed slots left over are closed by
    the tail fill."""
    keep = np.asarray(keep, dtype=bool)
    holes = np.flatnonzero(~keep)
    k = min(len(holes), len(new))
    out = s.copy()
    for f_out, f_new in zip(out.fields(), new.fields()):
        f_out[holes[:k]] = f_new[:k]
    if len(new) >= len(holes):
        return out.concat(new.take(np.arange(k, len(new))))
    keep2 = keep.copy()
    keep2[holes[:k]] = True
    return out.take(tail_fill(keep2))


def f32(a):
    return np.asarray(a, dtype=np.float64).astype(F32)


def deplete(w_parent, K, w_prod):
    """Weight depletion of a parent by K products of weight w_prod (Sec. II.F.1).

    If K w_prod exceeds the parent weight the products share the parent weight
    equally (reading: number is conserved exactly). Evaluated in binary32.
    Returns (product weight, remaining parent weight, clamped flag)."""
    w32 = f32(w_parent)
    wp32 = f32(w_prod)
    k32 = np.asarray(K).astype(F32)
    conv = (k32 * wp32).astype(F32)
    over = (np.asarray(K) > 0) & (conv > w32)
    safe_k = np.where(np.asarray(K) > 0, k32, F32(1.0))
    wprod = np.where(over, (w32 / safe_k).astype(F32), wp32)
    wrem = np.where(over, F32(0.0), (w32 - conv).astype(F32))
    return wprod.astype(np.float64), wrem.astype(np.float64), over


def primakoff_prob(cs: CellState, p: Params, omega_keV, mult=1.0):
    """P = 1 - exp(-m Gamma(omega) dt) (Eqs. prim_rate, prim_prob)."""
    s = 4.0 * np.asarray(omega_keV) ** 2 / cs.kappa_keV ** 2
    return -np.expm1(-mult * cs.Gamma0_P * primakoff_F(s) * p.dt_phys_s)


def _repeat_products(parent: Species, K, wprod, pos_from: Species = None):
    """Products in parent order, K[i] copies of parent i with weight wprod[i]."""
    idx = np.repeat(np.arange(len(K)), K)
    src = parent if pos_from is None else pos_from
    return Species(np.asarray(wprod)[idx], parent.px[idx], parent.py[idx], parent.pz[idx],
                   src.x[idx], src.y[idx], src.z[idx])


def _in_records(x):
    return (x >= 0.05) & (x <= 20.0)


# ---------------------------------------------------------------- massive axions
# Sec. II.B: an axion of momentum p carries E = sqrt(p^2 + m_a^2); the paper
# implements finite-mass kinematics (modified emission thresholds and
# absorption coefficients) without printing them. The readings:
# * absorption and a->gamma act on an axion with the massless rates taken at
#   its total energy E (the emission density and the equilibrium density both
#   carry the axion phase-space factor beta = p/E, which cancels in
#   Gamma_abs = (d ndot/dE) / (d n_eq/dE), Eq. gamma_abs); the a->gamma photon
#   takes energy E along p;
# * emission needs E >= m_a and carries beta: the massive process is the
#   massless one thinned with acceptance beta(E). A thermal-bath event keeps
#   its energy when u' < beta(E), u' the event's channel uniform rescaled
#   inside the interval of its channel (uniform and independent of the
#   channel choice); gamma->a converts at the rate beta(omega) Gamma and the
#   axion takes E = omega and momentum beta p_gamma;
# * the thermal-bath feedback exchanges the total energy E and the momentum p.
# The thinning and the threshold are decided in binary32, as the kernel
# decides them. With m_a = 0 every factor is exactly one and nothing is
# thinned.

def axion_energy_mc2(a: Species, mu):
    """E / (m_e c^2) of axions, E = sqrt(p^2 + m_a^2); mu = m_a / m_e c^2."""
    return np.sqrt(a.px ** 2 + a.py ** 2 + a.pz ** 2 + mu * mu)


def beta32(e, mu):
    """The axion phase-space factor p/E at energy e (m_e c^2 units) for mass
    mu, in binary32: p = sqrt(max(e^2 - mu^2, 0)), 0 below threshold."""
    e32 = f32(e)
    m32 = F32(mu)
    pm = np.sqrt(np.maximum((e32 * e32).astype(F32) - F32(m32 * m32), F32(0.0)).astype(F32)).astype(F32)
    return (pm / np.where(e32 > 0, e32, F32(1.0))).astype(F32)


def _absorb(cs: CellState, parts, p: Params, step, cell, mask, tally: StepTally, rec=None):
    """Inverse operators on the axions present at the start of the step. With
    a spectral record (table or surrogate rate model) the Primakoff and
    absorption rates at x = E/T in [0.05, 20] come from it. Returns the axions
    with their new weights, which of them stay, and the photon products."""
    a = parts["a"]
    tally.n_g0 = len(parts["g"])
    n = len(a)
    new_g = Species.empty()
    if n == 0:
        return a, np.ones(0, dtype=bool), new_g
    mu = p.axion_mass_keV / K.ME_C2_KEV
    omega = axion_energy_mc2(a, mu) * K.ME_C2_KEV     # the total energy E
    w = a.w.copy()
    x = omega / cs.T_keV
    use = _in_records(x) if rec is not None else np.zeros(n, dtype=bool)
    if mask & CH_PRIMAKOFF:
        P = primakoff_prob(cs, p, omega, p.prim_inverse_mult)
        if use.any():
            P = np.where(use, -np.expm1(-p.prim_inverse_mult * surrogate.rec_prim_gdt(rec, np.where(use, x, 1.0))), P)
        lam = w * P / F32(p.w_gref).astype(np.float64)
        lam_eff, fac, capped = cap_lambda(lam, p.lambda_cap)
        u = decision_uniforms(p, step, cell, STREAM_PRIM_INV, n)
        Kc = poisson_count(u, lam_eff)
        wprod, w, over = deplete(w, Kc, F32(p.w_gref).astype(np.float64) * fac)
        tally.events["prim_inv"] += int(Kc.sum())
        tally.cap_hits += int(capped.sum())
        tally.clamp_hits += int(over.sum())
        if Kc.sum() > 0:
            new_g = _repeat_products(a, Kc, wprod)
            if mu > 0:  # the photon takes the energy E along p
                pm = np.repeat(a.pmag(), Kc)
                f = np.repeat(omega / K.ME_C2_KEV, Kc) / np.where(pm > 0, pm, 1.0)
                new_g.px, new_g.py, new_g.pz = new_g.px * f, new_g.py * f, new_g.pz * f
    keep = w > 0
    want_c = bool(mask & CH_COMPTON)
    want_b = bool(mask & CH_BREMS)
    if want_c or want_b:
        E = omega
        tau_c = absorption_rate(cs, "compton", E, p) * p.dt_phys_s if want_c else np.zeros(n)
        tau_b = absorption_rate(cs, "brems", E, p) * p.dt_phys_s if want_b else np.zeros(n)
        if use.any():
            xs = np.where(use, x, 1.0)
            if want_c:
                tau_c = np.where(use, surrogate.rec_tau(rec, 1, xs, p.eq_stats), tau_c)
            if want_b:
                tau_b = np.where(use, surrogate.rec_tau(rec, 2, xs, p.eq_stats), tau_b)
        tau = tau_c + tau_b
        if p.absorb_mode == 0:
            P_abs = -np.expm1(-tau)
            u = decision_uniforms(p, step, cell, STREAM_ABSORB, n)
            absorbed = keep & (f32(u) < f32(P_abs))
            tally.dE += float(np.sum(w[absorbed] * omega[absorbed]))
            tally.gross_E += float(np.sum(w[absorbed] * omega[absorbed]))
            tally.gross_P += float(np.sum(w[absorbed] * a.pmag()[absorbed]))
            tally.dP += np.array([np.sum(w[absorbed] * a.px[absorbed]),
                                  np.sum(w[absorbed] * a.py[absorbed]),
                                  np.sum(w[absorbed] * a.pz[absorbed])])
            frac_c = f32(np.where(tau > 0, tau_c / np.where(tau > 0, tau, 1.0), 0.0))
            safeP = np.where(P_abs > 0, P_abs, 1.0)
            is_c = (f32(u) / f32(safeP)).astype(F32) < frac_c
            tally.absorbed["compton"] += int(np.sum(absorbed & is_c))
            tally.absorbed["brems"] += int(np.sum(absorbed & ~is_c))
            keep = keep & ~absorbed
        else:
            w_new = (f32(w) * f32(np.exp(-tau))).astype(np.float64)
            lost = w - w_new
            tally.dE += float(np.sum(lost * omega))
            tally.gross_E += float(np.sum(np.abs(lost) * omega))
            tally.gross_P += float(np.sum(np.abs(lost) * a.pmag()))
            tally.dP += np.array([np.sum(lost * a.px), np.sum(lost * a.py), np.sum(lost * a.pz)])
            w = w_new
            keep = keep & (w > 0)
    a2 = a.copy()
    a2.w = w
    return a2, keep, new_g


def absorb_cell(cs: CellState, parts, p: Params, step, cell, mask, tally: StepTally, rec=None):
    """Absorb phase of a separate call: photon products appended, axion holes
    closed by the tail fill."""
    a2, keep, new_g = _absorb(cs, parts, p, step, cell, mask, tally, rec)
    parts["a"] = a2.take(tail_fill(keep))
    if len(new_g):
        parts["g"] = parts["g"].concat(new_g)


def _emit(cs: CellState, parts, p: Params, step, cell, mask, tally: StepTally, n_g0=None, rec=None, qrec=None):
    """Forward operators: Primakoff on photons present at step start, then
    thermal-bath emission on electrons. With a spectral record the Primakoff
    rate (x in [0.05, 20]) and the emitted energies come from it; qrec (a
    record whose quantiles the energies come from, when rec is None) serves
    the surrogate model's network cells. Returns the photons with their
    remaining weights, which of them stay, and the new axions."""
    if n_g0 is None:
        n_g0 = len(parts["g"])
    g = parts["g"]
    w_a = F32(p.w_a).astype(np.float64)
    new_blocks = []
    chan_blocks = []
    energy_blocks = []
    if (mask & CH_PRIMAKOFF) and n_g0 > 0:
        g0 = g.take(np.arange(n_g0))
        omega = g0.pmag() * K.ME_C2_KEV
        mu = p.axion_mass_keV / K.ME_C2_KEV
        beta = beta32(omega / K.ME_C2_KEV, mu).astype(np.float64) if mu > 0 else np.ones(n_g0)
        s = 4.0 * omega ** 2 / cs.kappa_keV ** 2
        gdt = cs.Gamma0_P * primakoff_F(s) * p.dt_phys_s
        if rec is not None:
            x = omega / cs.T_keV
            use = _in_records(x)
            if use.any():
                gdt = np.where(use, surrogate.rec_prim_gdt(rec, np.where(use, x, 1.0)), gdt)
        P = -np.expm1(-beta * gdt)
        lam = g0.w * P / w_a
        lam_eff, fac, capped = cap_lambda(lam, p.lambda_cap)
        u = decision_uniforms(p, step, cell, STREAM_PRIM_FWD, n_g0)
        Kc = poisson_count(u, lam_eff)
        wprod, wrem, over = deplete(g0.w, Kc, w_a * fac)
        tally.events["prim"] += int(Kc.sum())
        tally.cap_hits += int(capped.sum())
        tally.clamp_hits += int(over.sum())
        prods = _repeat_products(g0, Kc, wprod)
        if mu > 0:  # the axion takes E = omega and momentum beta p_gamma
            bk = np.repeat(beta, Kc)
            prods.px, prods.py, prods.pz = prods.px * bk, prods.py * bk, prods.pz * bk
        new_blocks.append(prods)
        chan_blocks.append(np.full(len(prods), CH_PRIMAKOFF))
        energy_blocks.append(np.repeat(omega, Kc))
        g = g.copy()
        g.w[:n_g0] = wrem
    keep_g = g.w > 0
    e = parts["e"]
    ne = len(e)
    if (mask & (CH_COMPTON | CH_BREMS)) and ne > 0:
        # The Compton-like and bremsstrahlung operators of one electron are
        # independent Poisson processes (Sec. II.D.1, per channel, each with
        # its own cap, Eqs. lambda_eff and wa_rescaled). They are sampled as
        # their superposition: K ~ Poisson(lambda_C,eff + lambda_B,eff), and
        # event j goes to channel C when u < lambda_C,eff / (sum) (word 3 of
        # the event's block), which has the same law as two separate draws.
        zero = np.zeros(ne)
        lam_c = e.w * cs.Gamma_C * p.dt_phys_s / w_a if mask & CH_COMPTON else zero
        lam_b = e.w * cs.Gamma_B * p.dt_phys_s / w_a if mask & CH_BREMS else zero
        le_c, fac_c, cap_c = cap_lambda(lam_c, p.lambda_cap)
        le_b, fac_b, cap_b = cap_lambda(lam_b, p.lambda_cap)
        tally.cap_hits += int(cap_c.sum()) + int(cap_b.sum())
        # the sum and the channel split are decided in binary32 like the kernel
        lc32, lb32 = f32(le_c), f32(le_b)
        lsum32 = (lc32 + lb32).astype(F32)
        frac_c = np.where(lsum32 > 0, (lc32 / np.where(lsum32 > 0, lsum32, F32(1))).astype(F32), F32(0))
        u = decision_uniforms(p, step, cell, STREAM_EMIT_E, ne)
        Kc = poisson_count(u, lsum32.astype(np.float64))
        if Kc.sum() > 0:
            parent = np.repeat(np.arange(ne), Kc)
            sub = np.concatenate([np.arange(k) for k in Kc])
            uu = event_uniforms(p, step, cell, STREAM_EV_E, parent, sub)
            is_c = f32(uu[:, 3]) < frac_c[parent]
            qr = rec if rec is not None else qrec
            if qr is None:
                xE = np.where(is_c, spectra.compton_icdf(uu[:, 2]),
                              spectra.brems_icdf(p.brems_gamma_shape, uu[:, 2]))
            else:
                xE = np.where(is_c, surrogate.rec_sample_x(qr, 1, uu[:, 2]), surrogate.rec_sample_x(qr, 2, uu[:, 2]))
            E = xE * cs.T_keV
            mu = p.axion_mass_keV / K.ME_C2_KEV
            if mu > 0:
                # thinning with acceptance beta(E): the channel uniform
                # rescaled inside its channel's interval, in binary32
                u3 = f32(uu[:, 3])
                fc = frac_c[parent]
                ut = np.where(is_c, (u3 / np.where(fc > 0, fc, F32(1))).astype(F32),
                              ((u3 - fc).astype(F32) / np.where(fc < 1, (F32(1) - fc).astype(F32), F32(1))).astype(F32))
                e32 = (f32(E) * F32(1.0 / K.ME_C2_KEV)).astype(F32)
                keep_ev = ut < beta32(e32, mu)
                parent, sub, is_c, E, uu = parent[keep_ev], sub[keep_ev], is_c[keep_ev], E[keep_ev], uu[keep_ev]
                pm = np.sqrt(np.maximum((E / K.ME_C2_KEV) ** 2 - mu * mu, 0.0))
            else:
                pm = E / K.ME_C2_KEV
            dx, dy, dz = isotropic(uu[:, 0], uu[:, 1])
            fac = np.where(is_c, fac_c[parent], fac_b[parent])
            wv = f32(w_a * fac).astype(np.float64)
            prods = Species(wv, pm * dx, pm * dy, pm * dz, e.x[parent], e.y[parent], e.z[parent])
            tally.dE -= float(np.sum(wv * E))
            tally.gross_E += float(np.sum(wv * E))
            tally.gross_P += float(np.sum(wv * pm))
            tally.dP -= np.array([np.sum(wv * prods.px), np.sum(wv * prods.py), np.sum(wv * prods.pz)])
            tally.events["compton"] += int(is_c.sum())
            tally.events["brems"] += int((~is_c).sum())
            new_blocks.append(prods)
            chan_blocks.append(np.where(is_c, CH_COMPTON, CH_BREMS))
            energy_blocks.append(E)
    new = Species.empty()
    for b in new_blocks:
        new = new.concat(b)
    if new_blocks:
        tally.new_axion_channel = np.concatenate(chan_blocks)
        tally.new_axion_E = np.concatenate(energy_blocks)
    return g, keep_g, new


def emit_cell(cs: CellState, parts, p: Params, step, cell, mask, tally: StepTally, n_g0=None, rec=None):
    """Emit phase of a separate call: photon holes closed by the tail fill,
    new axions appended."""
    g, keep_g, new_a = _emit(cs, parts, p, step, cell, mask, tally, n_g0, rec)
    parts["g"] = g.take(tail_fill(keep_g))
    if len(new_a):
        parts["a"] = parts["a"].concat(new_a)


@dataclass
class FeedbackResult:
    T_new: float
    res_E: float
    res_P: np.ndarray
    S: float
    b: np.ndarray
    var: float
    var_new: float
    applied_E: float
    applied_P: np.ndarray
    W: float


def feedback_cell(cs: CellState, parts, p: Params, tally: StepTally, res_E=0.0, res_P=None):
    """Affine remap of the electron momenta (Sec. II.J.1) and temperature
    relaxation (Sec. II.J.2). Energies in keV; mu = 1 (electrons)."""
    if res_P is None:
        res_P = np.zeros(3)
    dE_req = tally.dE + res_E
    dP_req = tally.dP + res_P
    e = parts["e"]
    T = cs.T_keV
    if len(e) == 0 or np.sum(e.w) <= 0:
        return FeedbackResult(T, dE_req, dP_req.copy(), 1.0, np.zeros(3), 0.0, 0.0, 0.0, np.zeros(3), 0.0)
    pv = np.stack([e.px, e.py, e.pz], axis=1)
    W = float(np.sum(e.w))                                   # Eq. cell_moments
    Pm = np.sum(e.w[:, None] * pv, axis=0)
    U2 = float(np.sum(e.w * np.sum(pv * pv, axis=1)))
    mu = 1.0
    dE = dE_req / K.ME_C2_KEV                                # m_e c^2 units
    delta = dP_req / W                                       # Eq. delta_def
    dE_bulk = (2.0 * np.dot(delta, Pm) + W * np.dot(delta, delta)) / (2.0 * mu)   # Eq. dE_bulk
    dE_th = dE - dE_bulk                                     # Eq. dE_th
    var = U2 - np.dot(Pm, Pm) / W                            # Eq. var_unnormalized
    if var > 0:
        var_new = max(0.0, var + 2.0 * mu * dE_th)           # Eq. var_new
        S = math.sqrt(var_new / var)                         # Eq. s_def
    else:
        var_new = var
        S = 1.0
    b = (1.0 - S) * Pm / W + delta                           # Eq. b_def
    pnew = S * pv + b                                        # Eq. affine_map
    d = pnew - pv
    applied_E = float(np.sum(e.w * np.sum(d * (2.0 * pv + d), axis=1)) / 2.0) * K.ME_C2_KEV
    applied_P = np.sum(e.w[:, None] * d, axis=0)
    e2 = e.copy()
    e2.px, e2.py, e2.pz = pnew[:, 0].copy(), pnew[:, 1].copy(), pnew[:, 2].copy()
    parts["e"] = e2
    T_new = T
    if p.T_mode == 2:
        T_est = K.ME_C2_KEV / 3.0 * var_new / W              # Eq. Te_est
        T_new = (1.0 - p.relax_r) * T + p.relax_r * T_est    # Eq. Te_relax
        T_new = min(max(T_new, p.T_floor_keV), p.T_ceil_keV)
    return FeedbackResult(T_new, dE_req - applied_E, dP_req - applied_P, S, b, var, var_new,
                          applied_E, applied_P, W)


@dataclass
class CellInput:
    T_keV: float
    n_ion: np.ndarray
    Z: np.ndarray
    A: np.ndarray


def step_cell(ci: CellInput, parts, p: Params, step, cell, mask, res_E=0.0, res_P=None, feedback=True, rec=None,
              net=None):
    """absorb -> emit -> feedback for one cell; returns (tally, feedback result).
    The axions made in the emit phase reuse the axion slots freed in the
    absorb phase (recycle). rec: the cell's spectral record (table rate model,
    or the surrogate model where the network is not trusted) or None. net:
    (c, qrec) for a cell the surrogate network is trusted for: its three
    ln-emissivity constants (surrogate.network_cell_state) and a record
    holding the network's quantiles the energies come from."""
    cs = cell_state(ci.T_keV, ci.n_ion, ci.Z, ci.A, p)
    qrec = None
    if net is not None:
        cs = surrogate.network_cell_state(cs, net[0], p)
        qrec = net[1]
    tally = StepTally()
    a2, keep_a, new_g = _absorb(cs, parts, p, step, cell, mask, tally, rec)
    if len(new_g):
        parts["g"] = parts["g"].concat(new_g)
    g2, keep_g, new_a = _emit(cs, parts, p, step, cell, mask, tally, n_g0=tally.n_g0, rec=rec, qrec=qrec)
    parts["g"] = g2.take(tail_fill(keep_g))
    parts["a"] = recycle(a2, keep_a, new_a)
    fb = None
    if feedback:
        fb = feedback_cell(cs, parts, p, tally, res_E, res_P)
    return tally, fb


def photon_number_density(T_keV):
    """Planck photon density 2 zeta(3) T^3 / (pi^2 (hbar c)^3) [cm^-3]."""
    return 2.0 * special.zeta(3.0) * T_keV ** 3 / (math.pi ** 2 * K.HBARC_KEV_CM ** 3)


def init_cell(p: Params, cell, T_keV, n_e, volume_cm3, n_el, n_ph, n_ax):
    """Synthetic initial state of one cell: n_el NR-Maxwellian electrons of
    weight n_e V/n_el, n_ph Planck photons of weight n_gamma V/n_ph, and n_ax
    MB-equilibrium axions of weight w_a; positions uniform in the cell."""
    out = {}
    key_streams = (("e", STREAM_INIT_E, n_el), ("g", STREAM_INIT_G, n_ph), ("a", STREAM_INIT_A, n_ax))
    for name, stream, n in key_streams:
        if n == 0:
            out[name] = Species.empty()
            continue
        idx = np.arange(n)
        b0 = event_uniforms(p, INIT_STEP, cell, stream, idx, np.zeros(n, dtype=np.int64))
        b1 = event_uniforms(p, INIT_STEP, cell, stream, idx, np.ones(n, dtype=np.int64))
        if name == "e":
            sigma = math.sqrt(T_keV / K.ME_C2_KEV)
            r1 = np.sqrt(-2.0 * np.log(b0[:, 0]))
            r2 = np.sqrt(-2.0 * np.log(b0[:, 2]))
            px = sigma * r1 * np.cos(2.0 * math.pi * b0[:, 1])
            py = sigma * r1 * np.sin(2.0 * math.pi * b0[:, 1])
            pz = sigma * r2 * np.cos(2.0 * math.pi * b0[:, 3])
            w = np.full(n, f32(n_e * volume_cm3 / n_el).astype(np.float64))
        else:
            if name == "g":
                xE = spectra.planck_icdf(b0[:, 0])
                w = np.full(n, f32(photon_number_density(T_keV) * volume_cm3 / n_ph).astype(np.float64))
            else:
                xE = spectra.mb_axion_icdf(b0[:, 0])
                w = np.full(n, F32(p.w_a).astype(np.float64))
            pm = xE * T_keV / K.ME_C2_KEV
            dx, dy, dz = isotropic(b0[:, 1], b0[:, 2])
            px, py, pz = pm * dx, pm * dy, pm * dz
        out[name] = Species(w, px, py, pz, b1[:, 0].copy(), b1[:, 1].copy(), b1[:, 2].copy())
    return out
