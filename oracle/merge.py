"""Axion macroparticle merging for population control, plain CPU.

Test infrastructure only (imported by tests/). Each cell is handled on its
own, its groups one after the other, in slot order.

What it computes. The method advances, merges and deletes axions as a
particle species of the PIC code (Sec. II.A) and names no merging
algorithm. This follows the merging of N macroparticles into two of
Vranic et al., Comput. Phys. Commun. 191, 65 (2015), for massless
particles: a group of weights w_i and momenta p_i (m_e c) with
  W = sum w_i,  P = sum w_i p_i,  E = sum w_i |p_i|
becomes two particles of weight W / 2 and momentum magnitude E / W at the
angle theta, cos theta = |P| / E, on either side of P, so that W, P and E are
unchanged.

Readings (the paper is silent on each):
* Only a cell holding more than n_target axions is merged, in one pass; it
  may stay above n_target.
* Groups: the octant of p (the signs of px, py, pz, zero counting as
  positive) and the |p|^2 bin, the number of the caller's ascending binary32
  thresholds at or below |p|^2 = (px px + py py) + pz pz in binary32 (so the
  group is decided by comparisons alone). A group of three or more axions is
  merged.
* Arithmetic in binary32, each operation rounded: the sums over a group
  run in slot order with Kahan compensation (y = v - c; t = s + y;
  c = (t - s) - y; s = t), of w_i, w_i p_i, w_i |p_i| with
  |p_i| = sqrt((px px + py py) + pz pz), and w_i x_i; the position is the
  weighted mean sum w_i x_i / W. The merged axions are binary32 anyway, and
  the compensation keeps the sums' error near one rounding whatever the
  group's size.
* Directions: e_P = P / |P| (e_z when P = 0); the perpendicular e_perp is
  e_P x e_a, normalised, with e_a the axis of e_P's smallest |component|
  (the lowest index on ties); p_a = (E/W)(cos theta e_P + sin theta e_perp)
  and p_b = (E/W)(cos theta e_P - sin theta e_perp), sin theta =
  sqrt(1 - cos^2 theta), cos theta clamped to 1.
* The two new axions take the group's first two slots (p_a the first); the
  group's other slots are freed and closed by the tail fill (step.tail_fill).
"""
import numpy as np

from .step import Species, tail_fill


def group_of(px, py, pz, edges_p2):
    """Group index per axion: |p|^2 bin * 8 + octant."""
    f = np.float32
    px, py, pz = (np.asarray(v, dtype=f) for v in (px, py, pz))
    p2 = (px * px + py * py) + pz * pz
    e = np.zeros(len(p2), dtype=np.int64)
    for t in np.asarray(edges_p2, dtype=f):
        e += (p2 >= t).astype(np.int64)
    octant = (px < 0).astype(np.int64) | ((py < 0).astype(np.int64) << 1) | ((pz < 0).astype(np.int64) << 2)
    return e * 8 + octant


def _kahan(values):
    """Compensated binary32 sum in the order given."""
    f = np.float32
    s = f(0.0)
    c = f(0.0)
    for v in values:
        y = f(v) - c
        t = s + y
        c = (t - s) - y
        s = t
    return s


def merge_group(w, px, py, pz, x, y, z):
    """The two axions that replace one group (binary32, each step rounded as
    written): ((w, px, py, pz, x, y, z) of a, of b)."""
    f = np.float32
    w, px, py, pz, x, y, z = (np.asarray(v, dtype=f) for v in (w, px, py, pz, x, y, z))
    pn = [np.sqrt((px[i] * px[i] + py[i] * py[i]) + pz[i] * pz[i]) for i in range(len(w))]
    W = _kahan(w)
    Px = _kahan([w[i] * px[i] for i in range(len(w))])
    Py = _kahan([w[i] * py[i] for i in range(len(w))])
    Pz = _kahan([w[i] * pz[i] for i in range(len(w))])
    E = _kahan([w[i] * pn[i] for i in range(len(w))])
    X = _kahan([w[i] * x[i] for i in range(len(w))])
    Y = _kahan([w[i] * y[i] for i in range(len(w))])
    Zs = _kahan([w[i] * z[i] for i in range(len(w))])
    pm = E / W
    Pn = np.sqrt((Px * Px + Py * Py) + Pz * Pz)
    if Pn > f(0.0):
        e = (Px / Pn, Py / Pn, Pz / Pn)
        ct = min(Pn / E, f(1.0))
    else:
        e = (f(0.0), f(0.0), f(1.0))
        ct = f(0.0)
    st = np.sqrt(f(1.0) - ct * ct)
    ae = [abs(v) for v in e]
    k = 0
    for j in (1, 2):
        if ae[j] < ae[k]:
            k = j
    ax = [f(0.0), f(0.0), f(0.0)]
    ax[k] = f(1.0)
    u = (e[1] * ax[2] - e[2] * ax[1], e[2] * ax[0] - e[0] * ax[2], e[0] * ax[1] - e[1] * ax[0])
    un = np.sqrt((u[0] * u[0] + u[1] * u[1]) + u[2] * u[2])
    q = (u[0] / un, u[1] / un, u[2] / un)
    wh = W * f(0.5)
    pos = (X / W, Y / W, Zs / W)
    pa = tuple(pm * (ct * e[j] + st * q[j]) for j in range(3))
    pb = tuple(pm * (ct * e[j] - st * q[j]) for j in range(3))
    return tuple(f(v) for v in (wh,) + pa + pos), tuple(f(v) for v in (wh,) + pb + pos)


def merge_cell(s: Species, n_target, edges_p2):
    """One cell's axions after merging (a copy when it holds at most n_target)."""
    n = len(s)
    if n <= n_target:
        return s.copy(), 0
    g = group_of(s.px, s.py, s.pz, edges_p2)
    out = Species(*[np.asarray(v, dtype=np.float32).copy() for v in s.fields()])
    keep = np.ones(n, dtype=bool)
    for grp in np.unique(g):
        idx = np.flatnonzero(g == grp)
        if len(idx) < 3:
            continue
        a, b = merge_group(*[np.asarray(v)[idx] for v in s.fields()])
        for fld, va, vb in zip(out.fields(), a, b):
            fld[idx[0]] = va
            fld[idx[1]] = vb
        keep[idx[2:]] = False
    return out.take(tail_fill(keep)), int(n - keep.sum())


def merge(cells, n_target, edges_p2):
    """All cells: (new cells, axions removed)."""
    new, removed = [], 0
    for s in cells:
        c, r = merge_cell(s, n_target, edges_p2)
        new.append(c)
        removed += r
    return new, removed
