"""Composition from the deposited electron density, plain CPU, FP64.

Test infrastructure only (imported by tests/).

What it computes (Sec. II.E, Eqs. rho_def and qn_def). The rate models are
parameterised by the local electron density n_e and mass density
rho = sum_i n_i A_i m_u. The method can infer both from the deposited
charge density, given the hydrogen mass fraction X_H, under quasi-neutrality
n_e = sum_i Z_i n_i, or bind the whole density to one chosen ion species.

Readings (the paper gives the relations, not the deposit):
* The deposited density of a cell is that of its own electron
  macroparticles: n_e = sum_j w_j / V, with w_j the physical electrons a
  macroparticle carries and V the cell volume (the macroparticles are
  binned by cell, so the deposit is nearest-grid-point).
* Mass fractions X_i (X_H and 1 - X_H for hydrogen and helium) with
  quasi-neutrality: n_i = X_i rho / (A_i m_u), so
  n_e = (rho / m_u) sum_i Z_i X_i / A_i, which fixes rho / m_u.
* Bound to species k: n_k = n_e / Z_k, every other species 0.
"""
import numpy as np


def deposited_electron_density(weights, volume_cm3):
    """n_e [cm^-3] of one cell from its electron weights."""
    return float(np.sum(np.asarray(weights, dtype=np.float64))) / volume_cm3


def from_mass_fractions(n_e, Z, A, X):
    """Ion densities [cm^-3] from n_e and mass fractions X (summing to 1)."""
    Z, A, X = (np.asarray(v, dtype=np.float64) for v in (Z, A, X))
    rho_over_mu = n_e / float(np.sum(Z * X / A))
    return X * rho_over_mu / A


def bound_to_species(n_e, Z, k):
    """Ion densities [cm^-3] with the whole density on species k."""
    Z = np.asarray(Z, dtype=np.float64)
    n = np.zeros(len(Z))
    n[k] = n_e / Z[k]
    return n


def deposit(cells_w, volume_cm3, Z, A, X=None, bind=-1):
    """[ncells, nspecies] ion densities from each cell's electron weights."""
    out = []
    for w in cells_w:
        n_e = deposited_electron_density(w, volume_cm3)
        out.append(bound_to_species(n_e, Z, bind) if bind >= 0 else from_mass_fractions(n_e, Z, A, X))
    return np.array(out).reshape(len(cells_w), len(Z))
