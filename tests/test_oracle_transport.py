"""The streaming oracle (axion free streaming and cell migration) against
closed forms, a brute-force global-coordinate computation and invariants
(no GPU)."""
import math

import numpy as np
import pytest

from oracle import transport as TR
from oracle.step import Species

C = TR.C_CM_S


def axions(rng, n, spread=True):
    """n random axions: weights, isotropic momenta of random size, positions in [0, 1)."""
    u = rng.uniform(-1, 1, n)
    phi = rng.uniform(0, 2 * math.pi, n)
    s = np.sqrt(1 - u * u)
    pm = rng.uniform(0.5, 20, n) / 511.0
    f = np.float32
    return Species(rng.uniform(1, 2, n).astype(f), (pm * s * np.cos(phi)).astype(f), (pm * s * np.sin(phi)).astype(f),
                   (pm * u).astype(f), rng.uniform(0, 1, n).astype(f), rng.uniform(0, 1, n).astype(f),
                   rng.uniform(0, 1, n).astype(f))


def grid_cells(rng, dims, per_cell):
    return [axions(rng, int(rng.integers(0, per_cell + 1))) for _ in range(int(np.prod(dims)))]


def test_straight_line_closed_form():
    """One axion along +x: after n steps of kappa = c dt / h it sits at
    x0 + n kappa cells from its start, wrapped around the periodic box."""
    dims = (7, 1, 1)
    h = 1e-4
    kappa = 0.3
    dt = kappa * h / C
    f = np.float32
    cells = [Species.empty() for _ in range(7)]
    cells[2] = Species(np.array([1.5], f), np.array([3e-3], f), np.zeros(1, f), np.zeros(1, f),
                       np.array([0.25], f), np.array([0.5], f), np.array([0.5], f))
    for n in range(1, 41):
        cells, esc, dropped = TR.stream(cells, dims, h, dt, True, 8)
        where = [c for c in range(7) if len(cells[c])]
        assert len(where) == 1 and dropped == 0 and esc[0] == 0
        X = (2 + 0.25 + n * kappa) % 7
        assert where[0] == int(X)
        assert abs(float(cells[where[0]].x[0]) - (X - int(X))) < 2e-5
        assert float(cells[where[0]].y[0]) == 0.5 and float(cells[where[0]].w[0]) == f(1.5)


def test_massive_axion_moves_at_p_over_E():
    """A massive axion along +x moves kappa p / sqrt(p^2 + m^2) cells a step
    (sub-luminal); a massless one with the same momentum moves kappa."""
    dims = (11, 1, 1)
    h, kappa = 1e-4, 0.5
    dt = kappa * h / C
    f = np.float32
    p = 4.0 / 511.0
    m_keV = 3.0
    beta = p / math.sqrt(p * p + (m_keV / 510.99895) ** 2)
    cells = [Species.empty() for _ in range(11)]
    cells[0] = Species(np.array([1.0], f), np.array([p], f), np.zeros(1, f), np.zeros(1, f), np.array([0.0], f),
                       np.array([0.5], f), np.array([0.5], f))
    for n in range(1, 31):
        cells, _, _ = TR.stream(cells, dims, h, dt, True, 8, mass_keV=m_keV)
        where = [c for c in range(11) if len(cells[c])]
        X = (n * kappa * beta) % 11
        assert where == [int(X)] and abs(float(cells[where[0]].x[0]) - (X - int(X))) < 2e-5
    assert 0.7 < beta < 0.9


@pytest.mark.parametrize("mass", [0.0, 5.0])
@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("dims", [(5, 4, 3), (6, 5, 1)])
def test_brute_force_global_coordinates(periodic, dims, mass):
    """Every axion's new cell and fraction from its global coordinate
    X = i + x + kappa p_x / |p| in FP64 (per dimension), wrapped or dropped at
    the box; a dimension of one cell is not moved. The oracle's binary32
    result agrees to 1e-6 in X, and on the cell wherever X is not within 1e-6
    of a cell face."""
    rng = np.random.default_rng(5)
    nx, ny, nz = dims
    h, kappa = 1e-4, 0.8
    dt = kappa * h / C
    cells = grid_cells(rng, dims, 12)
    new, esc, dropped = TR.stream(cells, dims, h, dt, periodic, 64, mass_keV=mass)
    assert dropped == 0
    want, n_esc = {}, 0
    mu = mass / 510.99895
    for c, s in enumerate(cells):
        i, j, k = c % nx, (c // nx) % ny, c // (nx * ny)
        for a in range(len(s)):
            p = np.array([s.px[a], s.py[a], s.pz[a]], dtype=np.float64)
            X = np.array([i + s.x[a], j + s.y[a], k + s.z[a]], dtype=np.float64)
            for d, n in enumerate(dims):
                if n > 1:
                    X[d] += kappa * p[d] / math.sqrt(float(p @ p) + mu * mu)
            if periodic:
                X = np.mod(X, dims)
            elif np.any(X < 0) or np.any(X >= dims):
                n_esc += 1
                continue
            want[(float(s.w[a]), float(s.px[a]), float(s.pz[a]))] = X
    assert esc[0] == n_esc
    got = 0
    for c, s in enumerate(new):
        i, j, k = c % nx, (c // nx) % ny, c // (nx * ny)
        for a in range(len(s)):
            X = want[(float(s.w[a]), float(s.px[a]), float(s.pz[a]))]
            G = np.array([i + s.x[a], j + s.y[a], k + s.z[a]], dtype=np.float64)
            dG = np.abs(G - X)
            if periodic:
                dG = np.minimum(dG, np.abs(dG - np.array(dims)))
            assert dG.max() < 1e-6, (X, G)
            got += 1
    assert got == len(want)


def test_periodic_conserves_the_axions():
    """Periodic boundaries: every axion survives with its weight and momentum,
    whatever the number of steps."""
    rng = np.random.default_rng(6)
    dims = (4, 3, 2)
    cells = grid_cells(rng, dims, 10)
    before = sorted((float(s.w[a]), float(s.px[a]), float(s.py[a]), float(s.pz[a])) for s in cells
                    for a in range(len(s)))
    for _ in range(9):
        cells, esc, dropped = TR.stream(cells, dims, 1e-4, 0.9e-4 / C, True, 256)
        assert esc[0] == 0 and dropped == 0
    after = sorted((float(s.w[a]), float(s.px[a]), float(s.py[a]), float(s.pz[a])) for s in cells
                   for a in range(len(s)))
    assert before == after
    for s in cells:
        for q in (s.x, s.y, s.z):
            assert np.all((q >= 0) & (q < 1))


def test_open_box_escapes_count_weight_and_energy():
    rng = np.random.default_rng(7)
    dims = (3, 3, 3)
    cells = grid_cells(rng, dims, 8)
    new, esc, _ = TR.stream(cells, dims, 1e-4, 1e-4 / C, False, 256)
    n0 = sum(len(s) for s in cells)
    n1 = sum(len(s) for s in new)
    assert esc[0] == n0 - n1 > 0
    w0 = sum(float(np.sum(s.w, dtype=np.float64)) for s in cells)
    w1 = sum(float(np.sum(s.w, dtype=np.float64)) for s in new)
    assert abs(esc[1] - (w0 - w1)) < 1e-9 * w0
    E = lambda s: float(np.sum(s.w.astype(np.float64) * np.sqrt(s.px.astype(np.float64) ** 2 + s.py.astype(
        np.float64) ** 2 + s.pz.astype(np.float64) ** 2))) * 510.99895
    assert abs(esc[2] - (sum(E(s) for s in cells) - sum(E(s) for s in new))) < 1e-9 * sum(E(s) for s in cells)


def test_arrival_order():
    """Arrivals are ordered by the (dz, dy, dx) of their source relative to
    the cell, ascending, then by source slot (here all appended after the
    cell's stayers, which keep their slots)."""
    f = np.float32
    dims = (3, 3, 1)
    h = 1e-4
    dt = 0.5 * h / C
    cells = [Species.empty() for _ in range(9)]

    def put(c, w, px, py, x, y):
        cells[c] = cells[c].concat(Species(np.array([w], f), np.array([px], f), np.array([py], f),
                                           np.zeros(1, f), np.array([x], f), np.array([y], f), np.array([0.5], f)))

    centre = 4  # (i, j) = (1, 1)
    put(centre, 1.0, 1e-3, 0.0, 0.1, 0.5)   # stays (x 0.1 -> 0.6)
    put(5, 2.0, -1e-3, 0.0, 0.2, 0.5)       # from (2, 1): rel (0, 0, +1), moves -x
    put(centre, 3.0, 0.0, 0.0, 0.7, 0.7)    # stays (p = 0)
    put(1, 4.0, 0.0, 1e-3, 0.5, 0.8)        # from (1, 0): rel (0, -1, 0), moves +y
    put(3, 5.0, 1e-3, 0.0, 0.9, 0.5)        # from (0, 1): rel (0, 0, -1), moves +x
    put(1, 6.0, 0.0, 1e-3, 0.5, 0.9)        # second from (1, 0), later slot
    new, _, _ = TR.stream(cells, dims, h, dt, True, 16)
    assert [float(v) for v in new[centre].w] == [1.0, 3.0, 4.0, 6.0, 5.0, 2.0]


def test_arrivals_fill_the_freed_slots():
    """Arrivals take the slots of the cell's leavers in ascending order,
    extras are appended; with fewer arrivals than freed slots the tail fill
    closes the rest (survivors at or beyond the new count move down, in
    order)."""
    f = np.float32
    dims = (3, 1, 1)
    h = 1e-4
    dt = 0.5 * h / C

    def sp(ws, pxs, xs):
        n = len(ws)
        return Species(np.array(ws, f), np.array(pxs, f), np.zeros(n, f), np.zeros(n, f), np.array(xs, f),
                       np.full(n, 0.5, f), np.full(n, 0.5, f))

    # cell 1: slots 0 and 2 leave (+x), 1 and 3 stay; cell 0 sends one arrival
    cells = [sp([10.0], [1e-3], [0.8]), sp([1.0, 2.0, 3.0, 4.0], [1e-3, 0.0, 1e-3, 0.0], [0.7, 0.5, 0.9, 0.5]),
             Species.empty()]
    new, _, _ = TR.stream(cells, dims, h, dt, False, 8)
    # slot 0 takes the arrival (w 10); slot 2 is left over: the survivor count
    # is 3, so slot 2 stays a hole below it and takes slot 3 (w 4)
    assert [float(v) for v in new[1].w] == [10.0, 2.0, 4.0]
    # cell 2: no freed slots, two arrivals appended in source-slot order
    assert [float(v) for v in new[2].w] == [1.0, 3.0]
    # more arrivals than freed slots
    cells = [sp([10.0, 11.0], [1e-3, 1e-3], [0.8, 0.9]), sp([1.0, 2.0], [1e-3, 0.0], [0.7, 0.5]),
             Species.empty()]
    new, _, _ = TR.stream(cells, dims, h, dt, False, 8)
    assert [float(v) for v in new[1].w] == [10.0, 2.0, 11.0]


def test_one_cell_dimension_is_not_streamed():
    rng = np.random.default_rng(8)
    dims = (4, 4, 1)
    cells = grid_cells(rng, dims, 6)
    new, esc, _ = TR.stream(cells, dims, 1e-4, 1e-4 / C, False, 64)
    zs = sorted(float(v) for s in cells for v in s.z)
    zn = sorted(float(v) for s in new for v in s.z)
    assert set(zn) <= set(zs)


def test_capacity_drops_the_last_arrivals():
    f = np.float32
    dims = (2, 1, 1)
    cells = [Species(np.array([1, 2, 3], f), np.array([1e-3] * 3, f), np.zeros(3, f), np.zeros(3, f),
                     np.array([0.9, 0.95, 0.1], f), np.full(3, 0.5, f), np.full(3, 0.5, f)),
             Species(np.array([7], f), np.zeros(1, f), np.zeros(1, f), np.zeros(1, f), np.array([0.5], f),
                     np.full(1, 0.5, f), np.full(1, 0.5, f))]
    new, _, dropped = TR.stream(cells, dims, 1e-4, 0.5e-4 / C, True, 2)
    # cell 1 keeps its stayer (w 7) and takes the first arrival (w 1); w 2 is dropped
    assert [float(v) for v in new[1].w] == [7.0, 1.0] and dropped == 1
    assert [float(v) for v in new[0].w] == [3.0]
