"""Axion free streaming and cell migration through the C ABI against the
streaming oracle: every field of every slot bit for bit (the position update
is binary32 on both sides), several steps, periodic and open boxes, 3-D and
2-D grids, ragged and empty cells, a full slab; and at the size of the
256 x 256 relaxation plasma, sampled cells against the oracle run on their
neighbourhoods plus the invariants of a periodic box (needs a GB300)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import transport as TR
from oracle.step import Species

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2604_24627_gb300 import AxionPlasma, _lib, workloads  # noqa: E402

FIELDS = ("w", "px", "py", "pz", "x", "y", "z")
C = TR.C_CM_S


def random_axions(rng, n):
    u = rng.uniform(-1, 1, n)
    phi = rng.uniform(0, 2 * math.pi, n)
    s = np.sqrt(1 - u * u)
    pm = rng.uniform(0.5, 20, n) / 511.0
    # a few at rest and a few along an axis
    pm[rng.uniform(size=n) < 0.05] = 0.0
    f = np.float32
    sp = Species(rng.uniform(1, 2, n).astype(f), (pm * s * np.cos(phi)).astype(f), (pm * s * np.sin(phi)).astype(f),
                 (pm * u).astype(f), rng.uniform(0, 1, n).astype(f), rng.uniform(0, 1, n).astype(f),
                 rng.uniform(0, 1, n).astype(f))
    ax = rng.uniform(size=n) < 0.05
    sp.py[ax] = 0.0
    sp.pz[ax] = 0.0
    return sp


def make(ncells, acap):
    prm = dict(g_agg_GeV_inv=1e-10, g_ae=1e-12, dt_phys_s=2e12, w_a=3.0e9, seed=7, tally_enable=0)
    n = 6e25
    return AxionPlasma(ncells, np.full(ncells, 2.0), np.full((ncells, 1), n), [1.0], [1.00794], 1e-12,
                       (4, 4, acap), prm)


def load(pl, cells):
    for c, sp in enumerate(cells):
        pl.slabs["axions"].set_cell(c, {f: getattr(sp, f) for f in FIELDS})
    torch.cuda.synchronize()


def gpu_cells(pl, n):
    out = []
    for c in range(n):
        d = pl.slabs["axions"].cell(c)
        out.append(Species(*[d[f].astype(np.float32) for f in FIELDS]))
    return out


def assert_cells_equal(got, want):
    assert len(got) == len(want)
    for c, (g, w) in enumerate(zip(got, want)):
        assert len(g) == len(w), (c, len(g), len(w))
        for f in FIELDS:
            assert np.array_equal(getattr(g, f), np.asarray(getattr(w, f), dtype=np.float32)), (c, f)


@pytest.mark.parametrize("dims,periodic,mass", [((5, 4, 3), True, 0.0), ((5, 4, 3), False, 0.0),
                                                ((9, 7, 1), True, 0.0), ((9, 7, 1), False, 0.0),
                                                ((33, 1, 1), True, 0.0), ((5, 4, 3), False, 4.0),
                                                ((9, 7, 1), True, 12.0)])
def test_streaming_matches_oracle(dims, periodic, mass):
    rng = np.random.default_rng(hash((dims, periodic, mass)) % 2 ** 32)
    n = int(np.prod(dims))
    cap = 96
    cells = [random_axions(rng, int(rng.integers(0, 40))) if rng.uniform() > 0.1 else random_axions(rng, 0)
             for _ in range(n)]
    pl = make(n, cap)
    load(pl, cells)
    h, kappa = 1e-4, 0.7
    dt = kappa * h / C
    esc_total = np.zeros(3)
    for _ in range(5):
        pl.stream_axions(dims, h, dt, periodic, mass_keV=mass)
        cells, esc, dropped = TR.stream(cells, dims, h, dt, periodic, cap, mass_keV=mass)
        esc_total += esc
        assert dropped == 0
    torch.cuda.synchronize()
    assert_cells_equal(gpu_cells(pl, n), cells)
    st = pl.stream_stats()
    assert st[0] == esc_total[0] and st[3] == 0
    assert abs(st[1] - esc_total[1]) <= 1e-9 * max(1.0, esc_total[1])
    assert abs(st[2] - esc_total[2]) <= 1e-9 * max(1.0, esc_total[2])
    pl.close()


def test_full_slab_drops_the_last_arrivals():
    rng = np.random.default_rng(11)
    dims = (4, 4, 1)
    n = 16
    cap = 24
    cells = [random_axions(rng, 22) for _ in range(n)]
    pl = make(n, cap)
    load(pl, cells)
    h, dt = 1e-4, 0.9e-4 / C
    pl.stream_axions(dims, h, dt, True)
    want, _, dropped = TR.stream(cells, dims, h, dt, True, cap)
    assert dropped > 0
    torch.cuda.synchronize()
    assert_cells_equal(gpu_cells(pl, n), want)
    assert pl.stream_stats()[3] == dropped
    with pytest.raises(_lib.AxpicError):  # the drop latched AXPIC_E_CAPACITY; destroy reports it
        pl.close()


def test_invalid_grid_or_step_launches_nothing():
    pl = make(12, 8)
    with pytest.raises(_lib.AxpicError):
        pl.stream_axions((3, 3, 1), 1e-4, 1e-15, True)   # 9 cells for 12
    with pytest.raises(_lib.AxpicError):
        pl.stream_axions((4, 3, 1), 1e-4, 1e-4 / C, True)  # c dt = h
    with pytest.raises(_lib.AxpicError):
        pl.stream_axions((4, 3, 1), -1.0, 1e-15, True)
    with pytest.raises(_lib.AxpicError):
        pl.stream_axions((4, 3, 1), 1e-4, 1e-15, True, mass_keV=-1.0)
    assert list(pl.stream_stats()) == [0, 0, 0, 0]
    pl.close()


def test_relaxation_size_sampled_cells_and_invariants():
    """The 256 x 256 relaxation plasma's axions (MB equilibrium, 120 a cell),
    streamed in a periodic box: the axion count, the summed weight and the
    momentum multiset are unchanged, and 24 sampled cells equal the oracle
    run on their 3 x 3 neighbourhoods (open box: a neighbourhood's centre
    sees every arrival)."""
    w = workloads.config2(256, 256)
    w.params["w_a"] = float(np.float32(workloads.photon_weight(3.0, w.volume_cm3, w.n_ph) * w.w_a_over_w_gamma))
    w.params.update(seed=0, tally_enable=0)
    pl = AxionPlasma(w.ncells, w.T_keV, w.n_ion, w.Z, w.A, w.volume_cm3, w.caps, w.params)
    pl.sample(w.n_el, w.n_ph, 120)
    torch.cuda.synchronize()
    nx = ny = 256
    slab = pl.slabs["axions"]
    rng = np.random.default_rng(3)
    sample = rng.choice(w.ncells, 24, replace=False)
    hood = {}
    for c in sample:
        i, j = c % nx, c // nx
        sub = []
        for dj in (-1, 0, 1):
            for di in (-1, 0, 1):
                d = slab.cell(((j + dj) % ny) * nx + (i + di) % nx)
                sub.append(Species(*[d[f].astype(np.float32) for f in FIELDS]))
        hood[c] = sub

    def moments():
        cnt = slab.count[:w.ncells].long()
        idx = torch.arange(slab.capacity, device=cnt.device)[None, :] < cnt[:, None]
        m = idx.reshape(-1)
        p = torch.stack([slab.data[f][:m.numel()][m] for f in ("px", "py", "pz")], 1)
        return int(cnt.sum()), float(slab.data["w"][:m.numel()][m].double().sum()), torch.sort(p[:, 0]).values

    n0, w0, px0 = moments()
    h, dt = 1e-4, 0.6e-4 / C
    pl.stream_axions((nx, ny, 1), h, dt, True)
    torch.cuda.synchronize()
    n1, w1, px1 = moments()
    assert n1 == n0 and abs(w1 - w0) <= 1e-12 * w0 and torch.equal(px0, px1)
    for c in sample:
        want, _, dropped = TR.stream(hood[c], (3, 3, 1), h, dt, False, slab.capacity)
        d = slab.cell(c)
        got = Species(*[d[f].astype(np.float32) for f in FIELDS])
        assert_cells_equal([got], [want[4]])
    pl.close()


@pytest.mark.parametrize("periodic", [True, False])
def test_streamed_replay_equals_step_and_stream_calls(periodic):
    """35 steps of the full method, each followed by the axions' streaming on
    a 24 x 25 grid, replayed from graphs (8 branches asked for the steps):
    the same particles, slots and counters as plain step and stream calls."""
    prm = dict(g_agg_GeV_inv=1e-10, g_ae=1e-12, dt_phys_s=2e12, w_a=3.0e9, seed=0x1234_0000_0042, T_mode=2,
               relax_r=0.1, diag_enable=0, tally_enable=0, step_branches=8)
    dims, h = (24, 25, 1), 1e-4
    dt = 0.6 * h / C

    def make_pl():
        n = 600
        pl = AxionPlasma(n, np.linspace(1.3, 5.0, n), np.full((n, 1), 6e25), [1.0], [1.00794], 1e-12,
                         (64, 1024, 2048), prm)
        pl.sample(61, 37, 13)
        torch.cuda.synchronize()
        return pl

    a, b = make_pl(), make_pl()
    for s in range(35):
        a.step(s, _lib.CH_ALL)
        a.stream_axions(dims, h, dt, periodic)
    b.run_steps_streamed(0, 35, _lib.CH_ALL, dims, h, dt, periodic)
    torch.cuda.synchronize()
    for name in ("electrons", "photons", "axions"):
        sa_, sb_ = a.slabs[name], b.slabs[name]
        assert torch.equal(sa_.count, sb_.count), name
        cap = sa_.capacity
        idx = (torch.arange(cap, device=sa_.count.device)[None, :] < sa_.count[:, None].long()).reshape(-1)
        for f in FIELDS:
            assert torch.equal(sa_.data[f][:idx.numel()][idx], sb_.data[f][:idx.numel()][idx]), (name, f)
    assert torch.equal(a.T, b.T)
    sa, sb = a.stream_stats(), b.stream_stats()
    # counts exactly; the escaped weight and energy are FP64 atomic sums,
    # whose order varies
    assert sa[0] == sb[0] and sa[3] == sb[3]
    assert np.allclose(sa[1:3], sb[1:3], rtol=1e-12, atol=0)
    assert b.launch_shape()[2] > 1
    a.close()
    b.close()
