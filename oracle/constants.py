"""Physical constants used by the oracle (CODATA 2018 exact or recommended values).

Test infrastructure only (imported by tests/, smoke() and bench.py's CPU
baseline). The paper rounds m_e c^2 to 511 keV (Eq. Ek_keV), 1 keV to
1.602e-9 erg (App. B) and alpha to 1/137 (Sec. II.E); the oracle uses the
CODATA values, which differ from those roundings by less than 2e-3 relative.
"""
import math

ME_C2_KEV = 510.99895000            # electron rest energy [keV]
HBARC_KEV_CM = 1.973269804e-8       # hbar*c [keV cm]
HBARC_GEV_CM = 1.973269804e-14      # hbar*c [GeV cm]
HBAR_GEV_S = 6.582119569e-25        # hbar [GeV s]
ALPHA_EM = 1.0 / 137.035999084      # fine-structure constant
M_U_G = 1.66053906660e-24           # atomic mass unit [g]
C_CM_S = 2.99792458e10              # speed of light [cm/s]
K_B_KEV_PER_K = 8.617333262e-8      # Boltzmann constant [keV/K]
KEV_ERG = 1.602176634e-9            # 1 keV in erg
A_H = 1.00794                       # hydrogen atomic mass number (standard atomic weight)
A_HE = 4.002602                     # helium-4 atomic mass number
LAMBDA_HARD_CAP = 64.0              # ceiling on the sampled Poisson mean (always applied)
POISSON_KMAX = 255                  # bound of the Poisson inversion loop
FOUR_PI = 4.0 * math.pi
