"""The merging oracle against closed forms and the conservation it promises
(no GPU)."""
import math

import numpy as np

from oracle import merge as MG
from oracle.step import Species

f = np.float32
EDGES = np.array([1e-8, 1e-6, 1e-5, 1e-4], dtype=np.float32)


def sp(rows):
    """rows of (w, px, py, pz, x, y, z)."""
    a = np.array(rows, dtype=np.float64).T
    return Species(*[a[k].astype(f) for k in range(7)])


def test_collinear_group_closed_form():
    """Three axions along +z: W = 4, P = E = 9e-3 (m_e c), so both products
    carry weight 2 and p = (0, 0, 9e-3 / 4) at the weighted mean position."""
    s = sp([(1, 0, 0, 1e-3, 0.1, 0.2, 0.3), (1, 0, 0, 2e-3, 0.3, 0.2, 0.3), (2, 0, 0, 3e-3, 0.5, 0.5, 0.5)])
    a, b = MG.merge_group(*s.fields())
    for p in (a, b):
        assert p[0] == f(2.0)
        assert p[1] == 0 and p[2] == 0 and abs(float(p[3]) - 2.25e-3) < 1e-9
        assert abs(float(p[4]) - 0.35) < 1e-7 and abs(float(p[6]) - 0.4) < 1e-7


def test_two_products_at_the_angle_cos_theta_P_over_E():
    """A non-collinear group: both products have |p| = E/W, sum to P / (W/2),
    and make the angle theta with P, cos theta = |P| / E."""
    s = sp([(1.0, 1e-3, 0, 1e-3, .5, .5, .5), (2.0, 2e-3, 1e-3, 0, .5, .5, .5), (1.5, 0, 2e-3, 3e-3, .5, .5, .5)])
    w = s.w.astype(float)
    p = np.stack([s.px, s.py, s.pz], 1).astype(float)
    W, P = w.sum(), (w[:, None] * p).sum(0)
    E = float((w * np.linalg.norm(p, axis=1)).sum())
    a, b = MG.merge_group(*s.fields())
    pa, pb = np.array(a[1:4], float), np.array(b[1:4], float)
    for q in (pa, pb):
        assert abs(np.linalg.norm(q) - E / W) < 1e-6 * E / W
        assert abs(q @ P / (np.linalg.norm(q) * np.linalg.norm(P)) - np.linalg.norm(P) / E) < 1e-6
    np.testing.assert_allclose((pa + pb) * W / 2, P, rtol=1e-6)


def test_conservation_on_random_cells():
    """Per cell: weight, momentum and energy unchanged to binary32 rounding;
    the count falls by the members beyond two of every merged group."""
    rng = np.random.default_rng(2)
    for _ in range(20):
        n = int(rng.integers(5, 120))
        u = rng.uniform(-1, 1, n)
        phi = rng.uniform(0, 2 * math.pi, n)
        pm = rng.uniform(1e-4, 1.5e-2, n)
        st = np.sqrt(1 - u * u)
        s = Species(rng.uniform(1, 3, n).astype(f), (pm * st * np.cos(phi)).astype(f),
                    (pm * st * np.sin(phi)).astype(f), (pm * u).astype(f), rng.uniform(0, 1, n).astype(f),
                    rng.uniform(0, 1, n).astype(f), rng.uniform(0, 1, n).astype(f))
        new, removed = MG.merge_cell(s, 4, EDGES)

        def moments(c):
            w = c.w.astype(float)
            p = np.stack([c.px, c.py, c.pz], 1).astype(float)
            return w.sum(), (w[:, None] * p).sum(0), float((w * np.linalg.norm(p, axis=1)).sum())

        W0, P0, E0 = moments(s)
        W1, P1, E1 = moments(new)
        assert abs(W1 - W0) <= 2e-6 * W0 and abs(E1 - E0) <= 2e-6 * E0
        assert np.abs(P1 - P0).max() <= 2e-6 * E0
        g = MG.group_of(s.px, s.py, s.pz, EDGES)
        want = sum(max(0, int((g == k).sum()) - 2) for k in np.unique(g) if (g == k).sum() >= 3)
        assert removed == want and len(new) == n - want


def test_small_cells_and_small_groups_are_untouched():
    s = sp([(1, 1e-3, 1e-3, 1e-3, .1, .1, .1), (1, 2e-3, 1e-3, 1e-3, .2, .2, .2), (1, -1e-3, 1e-3, 1e-3, .3, .3, .3)])
    new, removed = MG.merge_cell(s, 3, EDGES)
    assert removed == 0 and all(np.array_equal(a, b) for a, b in zip(new.fields(), s.fields()))
    new, removed = MG.merge_cell(s, 2, EDGES)   # above n_target, but no group of three
    assert removed == 0 and all(np.array_equal(a, b) for a, b in zip(new.fields(), s.fields()))


def test_group_thresholds_are_inclusive_and_slots_follow_the_rule():
    """|p|^2 equal to a threshold goes to the upper bin; the products take
    the group's first two slots, the freed ones are closed by the tail fill."""
    t = f(np.sqrt(f(1e-6)))
    assert MG.group_of([t], [0], [0], EDGES)[0] // 8 == int((EDGES <= f(t) * f(t)).sum())
    rows = [(1, 1e-3, 0, 0, .5, .5, .5), (9, -1e-3, 0, 0, .5, .5, .5), (1, 1.1e-3, 0, 0, .5, .5, .5),
            (1, 1.2e-3, 0, 0, .5, .5, .5), (8, -2e-3, 0, 0, .5, .5, .5), (1, 1.3e-3, 0, 0, .5, .5, .5)]
    new, removed = MG.merge_cell(sp(rows), 2, EDGES)
    # the +x group (slots 0, 2, 3, 5) merges into slots 0 and 2; slots 3 and 5 are freed;
    # the survivor count is 4, so slot 3 takes slot 4 (w 8)
    assert removed == 2
    assert [float(v) for v in new.w] == [2.0, 9.0, 2.0, 8.0]


def test_degenerate_groups():
    """Zero momenta: P = 0, so e_P = e_z, cos theta = 0 and both products
    carry p = 0. Identical axions: |P| = E up to rounding, so cos theta is 1
    within a few binary32 roundings and sin theta = sqrt(1 - cos^2 theta) at
    most about sqrt(2 * 4 * 2^-24) ~ 1e-3: the products sit symmetrically
    about p, with |p| and the doubled-up weight."""
    a, b = MG.merge_group(*sp([(1, 0, 0, 0, .1, .2, .3)] * 4).fields())
    assert a == b and a[:4] == (f(2.0), f(0.0), f(0.0), f(0.0))
    row = (1.5, 1e-3, 2e-3, -3e-3, .25, .5, .75)
    a, b = MG.merge_group(*sp([row] * 5).fields())
    want = np.array(row, dtype=f).astype(float)
    pa, pb = np.array(a[1:4], float), np.array(b[1:4], float)
    pn = np.linalg.norm(want[1:4])
    assert a[0] == b[0] == f(3.75)
    np.testing.assert_allclose((pa + pb) / 2, want[1:4], rtol=0, atol=1e-6 * pn)
    for q in (pa, pb):
        assert abs(np.linalg.norm(q) - pn) <= 1e-6 * pn
        assert np.linalg.norm(q - want[1:4]) <= 1e-3 * pn
    np.testing.assert_allclose(np.array(a[4:], float), want[4:], rtol=1e-6)
