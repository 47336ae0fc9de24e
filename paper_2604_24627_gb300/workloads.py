"""Synthetic workloads: the uniform thermal plasmas the paper benchmarks on
(Sec. III.A: uniform, static, fixed T_e), sized as the five configurations this
library is measured on. Seeded input generation only: this module holds cell
fields and option values, none of the method's arithmetic, and serves both the
CUDA path and the oracle.

Constants chosen here (time steps, macroparticle weights) were derived once
from the paper's rates: each dt makes the total absorption depth of the
median Maxwell-Boltzmann equilibrium axion (x = E/T = 2.674) over one step
equal to 1e-2, so per-step probabilities stay small; the axion weight is
w_a_over_w_gamma times a Planck photon weight that the caller picks
(photon_weight below).
"""
from dataclasses import dataclass, field

import numpy as np

A_H = 1.00794
A_HE = 4.002602
VOLUME_1UM3 = 1e-12  # cm^3


@dataclass
class Workload:
    name: str
    ncells: int
    shape: tuple
    T_keV: np.ndarray            # [ncells]
    n_ion: np.ndarray            # [ncells, nspecies], cm^-3
    Z: np.ndarray
    A: np.ndarray
    volume_cm3: float
    n_el: int
    n_ph: int
    n_ax: int
    caps: tuple                  # slots per cell (electrons, photons, axions)
    params: dict = field(default_factory=dict)
    mask: int = 7
    steps: int = 1
    box_of_cell: np.ndarray = None
    w_a_over_w_gamma: float = 0.0   # > 0: w_a = this * photon weight at T (set by the caller)

    def particles_per_cell(self):
        return self.n_el + self.n_ph + self.n_ax


def _hydrogen(ncells, n_e):
    n = np.broadcast_to(np.asarray(n_e, dtype=np.float64), (ncells,)).reshape(ncells, 1)
    return n.copy(), np.array([1.0]), np.array([A_H])


def config1(ncells=64):
    """1-D uniform hydrogen, 64 cells, T = 1.3 keV, n_e = 6e25 cm^-3, Primakoff
    forward only, g_agg = 1e-10 GeV^-1, 128 Planck photons per cell,
    w_a = w_gamma / 4 and dt such that about 0.1 events per cell per step."""
    n_ion, Z, A = _hydrogen(ncells, 6e25)
    return Workload("c1-primakoff-1d-64", ncells, (ncells,), np.full(ncells, 1.3), n_ion, Z, A, VOLUME_1UM3,
                    0, 128, 0, (4, 128, 256),
                    params=dict(g_agg_GeV_inv=1e-10, g_ae=1e-13, dt_phys_s=9.02e10, T_mode=0),
                    mask=1, steps=200, w_a_over_w_gamma=0.25)


def config2(nx=256, ny=256):
    """2-D 256x256, T = 3 keV, ions 90% Z=1 + 10% Z=2 by number with
    n_e = 6e25 cm^-3, 512 Maxwellian electrons + 256 Planck photons per cell,
    all channels forward and inverse, w_a = w_gamma, T evolved (r = 0.1),
    dt = 8.763e11 s (median MB axion: sum Gamma_abs dt = 1e-2)."""
    ncells = nx * ny
    n_tot = 6e25 / 1.1
    n_ion = np.tile(np.array([[0.9 * n_tot, 0.1 * n_tot]]), (ncells, 1))
    return Workload("c2-2d-256x256-all-channels", ncells, (nx, ny), np.full(ncells, 3.0), n_ion,
                    np.array([1.0, 2.0]), np.array([A_H, A_HE]), VOLUME_1UM3, 512, 256, 0, (512, 384, 384),
                    params=dict(g_agg_GeV_inv=1e-10, g_ae=1e-13, dt_phys_s=8.763e11, T_mode=2, relax_r=0.1,
                                eq_stats=0, brems_ee=1),
                    mask=7, steps=1000, w_a_over_w_gamma=1.0)


def config3(n=512, sigma=64.0):
    """2-D 512x512 with a Gaussian temperature bump 1 -> 5 keV (sigma 64
    cells), hydrogen n_e = 6e25 cm^-3, 256 electrons + 128 photons per cell,
    prescribed temperature field, dt = 9.93e11 s. With one axion weight (the
    photon weight at 3 keV) the hot cells turn their heavier photons into
    axion-weight photons (up to 128 (5/3)^3 ~ 593 per cell) and hold up to
    ~250 axion macroparticles at equilibrium: slabs of 768 and 384 slots."""
    i = np.arange(n) + 0.5 - n / 2
    r2 = i[:, None] ** 2 + i[None, :] ** 2
    T = (1.0 + 4.0 * np.exp(-r2 / (2 * sigma ** 2))).reshape(-1)
    n_ion, Z, A = _hydrogen(n * n, 6e25)
    return Workload("c3-2d-512x512-T-bump", n * n, (n, n), T, n_ion, Z, A, VOLUME_1UM3, 256, 128, 0,
                    (256, 768, 384),
                    params=dict(g_agg_GeV_inv=1e-10, g_ae=1e-13, dt_phys_s=9.93e11, T_mode=1),
                    mask=7, steps=100, w_a_over_w_gamma=1.0)


def config4(nboxes=4096, seed=0):
    """4096 independent uniform hydrogen boxes; cell counts log-normal (median
    256, sigma_ln = ln(16)/3) resampled into [16, 4096]; T ~ U[1, 5] keV;
    n_e log-uniform in [1e24, 1e26]; 128 electrons + 64 photons per cell.
    The boxes share one axion weight (the photon weight at 3 keV). In hot
    boxes the photons are heavier than that weight: Primakoff exchange turns
    them into axion macroparticles (up to about 0.42 * 64 * (5/3)^3 ~ 123 per
    cell at equilibrium) and back into photons of the axion weight (up to
    64 * (5/3)^3 ~ 296 per cell): slabs of 384 photon and 192 axion slots."""
    rng = np.random.default_rng(seed)
    counts = np.empty(nboxes, dtype=np.int64)
    for b in range(nboxes):
        while True:
            c = int(round(np.exp(np.log(256.0) + rng.normal() * np.log(16.0) / 3.0)))
            if 16 <= c <= 4096:
                counts[b] = c
                break
    T_box = rng.uniform(1.0, 5.0, nboxes)
    ne_box = 10.0 ** rng.uniform(24.0, 26.0, nboxes)
    box = np.repeat(np.arange(nboxes), counts)
    ncells = int(counts.sum())
    n_ion = ne_box[box].reshape(ncells, 1)
    return Workload("c4-4096-boxes", ncells, (ncells,), T_box[box], n_ion, np.array([1.0]), np.array([A_H]),
                    VOLUME_1UM3, 128, 64, 0, (128, 384, 192),
                    params=dict(g_agg_GeV_inv=1e-10, g_ae=1e-13, dt_phys_s=9.93e11, T_mode=2, relax_r=0.1),
                    mask=7, steps=100, box_of_cell=box, w_a_over_w_gamma=1.0)


def config5(n=256):
    """3-D 256^3, T = 5 keV, hydrogen n_e = 6e25 cm^-3, 64 electrons + 32
    photons per cell, all channels, T evolved, dt = 5.448e11 s. With w_a =
    w_gamma the Primakoff exchange moves photons and axions between about 45
    macroparticles a cell (plus the thermal-bath axions): slabs of 64 photon
    and 64 axion slots keep the tails of 16.8 M cells."""
    ncells = n ** 3
    n_ion, Z, A = _hydrogen(ncells, 6e25)
    return Workload("c5-3d-%d^3" % n, ncells, (n, n, n), np.full(ncells, 5.0), n_ion, Z, A, VOLUME_1UM3, 64, 32,
                    0, (64, 64, 64),
                    params=dict(g_agg_GeV_inv=1e-10, g_ae=1e-13, dt_phys_s=5.448e11, T_mode=2, relax_r=0.1),
                    mask=7, steps=50, w_a_over_w_gamma=1.0)


def photon_weight(T_keV, volume_cm3, n_ph):
    """Planck photon macroparticle weight n_gamma V / n_ph used to set w_a
    (photon number density 2 zeta(3) T^3 / (pi^2 (hbar c)^3))."""
    zeta3 = 1.2020569031595942
    hbarc = 1.973269804e-8
    n_gamma = 2.0 * zeta3 * T_keV ** 3 / (np.pi ** 2 * hbarc ** 3)
    return n_gamma * volume_cm3 / n_ph


def subset(w: Workload, cells):
    """The same workload restricted to a list of cells (keeps global indices
    through cell_index_base only when the list is contiguous)."""
    cells = np.asarray(cells)
    out = Workload(**{k: getattr(w, k) for k in w.__dataclass_fields__})
    out.ncells = len(cells)
    out.shape = (len(cells),)
    out.T_keV = w.T_keV[cells]
    out.n_ion = w.n_ion[cells]
    if w.box_of_cell is not None:
        out.box_of_cell = w.box_of_cell[cells]
    return out
