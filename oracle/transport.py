"""Axion free streaming and cell migration, plain CPU.

Test infrastructure only (imported by tests/). Nothing here is blocked or
fused: each axion is moved, then every cell's slots are rebuilt from the
moved axions in the order defined below.

What it computes. Axions move along their momentum at v = p / E c with
E = sqrt(p^2 + m_a^2) (Sec. II.B: massless axions at c, v = p / |p|;
massive ones sub-luminal): x += (p / E) c dt, the free-streaming transport
of the axion macroparticles between the emission and absorption steps.
Positions are fractions of the cell in [0, 1).

Readings of the paper (it is silent on each):
* The grid is regular: nx x ny x nz cubic cells of edge h [cm], cell index
  (k ny + j) nx + i.
* A step moves an axion at most one cell per dimension (c dt <= h).
* A dimension of one cell is not streamed: its position component is kept.
  A 2-D run moves axions in its plane only.
* Boundaries are periodic (leaving one side enters the other) or open (an
  axion leaving the box is removed and counted).
* The position update is binary32, since it decides the destination cell:
  E = sqrt(((px px + py py) + pz pz) + mu mu), each operation rounded, with
  mu = binary32(m_a c^2 / m_e c^2) (momenta are in m_e c);
  d = (kappa / E) p_dim with kappa = binary32(c dt / h);
  t = x + d; s = floor(t) in {-1, 0, 1}; t = t - s, and t = the largest
  binary32 below 1 where that rounds up to 1. E = 0 does not move.
* The energy counted for an axion leaving an open box is its total energy
  sqrt(p^2 + m_a^2) (in keV, times its weight).
* Re-binning: the arrivals of a cell are ordered by the position of their
  source cell relative to it, (dz, dy, dx) in ascending lexicographic order
  over {-1, 0, 1}^3, then by source slot. They take the slots the cell's
  leaving axions freed, in ascending order; arrivals beyond those are
  appended after the old count, and freed slots left over are closed by the
  tail fill (step.recycle, the slot rule of a full step's axions). Staying
  axions keep their slots unless the tail fill moves them. Axions beyond the
  slab capacity are dropped and counted.
"""
import numpy as np

from . import constants as K
from .step import Species, recycle

C_CM_S = 2.99792458e10
_ONE_BELOW = np.nextafter(np.float32(1.0), np.float32(0.0))


def offsets():
    """The 26 relative positions (dz, dy, dx), ascending lexicographic."""
    return [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
            if (dz, dy, dx) != (0, 0, 0)]


def stream(cells, dims, h_cm, dt_s, periodic, cap, mass_keV=0.0):
    """cells: list of Species (axions, slot order) indexed (k ny + j) nx + i;
    mass_keV: the axion mass m_a c^2. Returns (new cells, escaped [number,
    weight, weight x energy keV], dropped number)."""
    nx, ny, nz = dims
    assert len(cells) == nx * ny * nz
    f = np.float32
    kappa = f(C_CM_S * dt_s / h_cm)
    assert kappa <= 1.0, "a step may move an axion at most one cell"
    mu = f(mass_keV / K.ME_C2_KEV)
    n_dim = (nx, ny, nz)
    moved = []  # per source cell: (Species with new positions, shift per axion [n, 3] as (sx, sy, sz))
    for s in cells:
        px, py, pz = (np.asarray(v, dtype=np.float32) for v in (s.px, s.py, s.pz))
        en = np.sqrt(((px * px + py * py) + pz * pz) + mu * mu)
        newpos, shifts = [], []
        for dim, (pc, q) in enumerate(zip((px, py, pz), (s.x, s.y, s.z))):
            q = np.asarray(q, dtype=np.float32)
            if n_dim[dim] == 1:
                newpos.append(q.copy())
                shifts.append(np.zeros(len(q), dtype=np.int64))
                continue
            with np.errstate(divide="ignore", invalid="ignore"):
                d = np.where(en > 0, (kappa / en) * pc, f(0.0)).astype(np.float32)
            t = (q + d).astype(np.float32)
            sh = np.floor(t).astype(np.float32)
            t = (t - sh).astype(np.float32)
            t = np.where(t >= f(1.0), _ONE_BELOW, t).astype(np.float32)
            newpos.append(t)
            shifts.append(sh.astype(np.int64))
        m = Species(np.asarray(s.w, dtype=np.float32), px, py, pz, newpos[0], newpos[1], newpos[2])
        moved.append((m, np.stack(shifts, axis=1) if len(s) else np.zeros((0, 3), dtype=np.int64)))

    escaped = np.zeros(3)
    dest = []  # per source cell: destination cell per axion (-1: escaped)
    for c, (m, sh) in enumerate(moved):
        i, j, k = c % nx, (c // nx) % ny, c // (nx * ny)
        out = np.empty(len(m), dtype=np.int64)
        for a in range(len(m)):
            ii, jj, kk = i + sh[a, 0], j + sh[a, 1], k + sh[a, 2]
            if periodic:
                ii, jj, kk = ii % nx, jj % ny, kk % nz
            elif not (0 <= ii < nx and 0 <= jj < ny and 0 <= kk < nz):
                out[a] = -1
                E = float(np.sqrt(float(m.px[a]) ** 2 + float(m.py[a]) ** 2 + float(m.pz[a]) ** 2
                                  + float(mu) ** 2)) * K.ME_C2_KEV
                escaped += (1.0, float(m.w[a]), float(m.w[a]) * E)
                continue
            out[a] = (kk * ny + jj) * nx + ii
        dest.append(out)

    new_cells, dropped = [], 0
    for d in range(len(cells)):
        i, j, k = d % nx, (d // nx) % ny, d // (nx * ny)
        m, sh = moved[d]
        stay = (dest[d] == d) & np.all(sh == 0, axis=1)
        parts = []
        for dz, dy, dx in offsets():
            si, sj, sk = i + dx, j + dy, k + dz
            if periodic:
                si, sj, sk = si % nx, sj % ny, sk % nz
            elif not (0 <= si < nx and 0 <= sj < ny and 0 <= sk < nz):
                continue
            if (dx and nx == 1) or (dy and ny == 1) or (dz and nz == 1):
                continue
            src = (sk * ny + sj) * nx + si
            ms, shs = moved[src]
            # the axions of src that moved by (-dx, -dy, -dz) into d
            sel = np.flatnonzero((dest[src] == d) & (shs[:, 0] == -dx) & (shs[:, 1] == -dy) & (shs[:, 2] == -dz))
            parts.append(ms.take(sel))
        arrivals = Species.empty()
        for p in parts:
            arrivals = arrivals.concat(p)
        cell = recycle(m, stay, arrivals)
        if len(cell) > cap:
            dropped += len(cell) - cap
            cell = cell.take(np.arange(cap))
        new_cells.append(cell)
    return new_cells, escaped, dropped
