"""Axion merging through the C ABI against the merging oracle: every field of
every slot bit for bit (group decisions by binary32 comparisons, binary32
compensated sums with each rounding fixed), empty, small, ragged and full cells; at the size
of the 256 x 256 relaxation plasma, sampled cells against the oracle and the
conservation of weight, momentum and energy per cell (needs a GB300)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import merge as MG
from oracle.step import Species

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2604_24627_gb300 import AxionPlasma, _lib, workloads  # noqa: E402

FIELDS = ("w", "px", "py", "pz", "x", "y", "z")
# |p| from 0.5 to 50 keV in m_e c, 16 log-spaced thresholds on |p|^2
EDGES = (np.geomspace(0.5, 50.0, 16) / 510.99895).astype(np.float32) ** 2


def random_axions(rng, n):
    u = rng.uniform(-1, 1, n)
    phi = rng.uniform(0, 2 * math.pi, n)
    s = np.sqrt(1 - u * u)
    pm = rng.uniform(0.3, 60, n) / 511.0
    f = np.float32
    sp = Species(rng.uniform(1, 2, n).astype(f), (pm * s * np.cos(phi)).astype(f), (pm * s * np.sin(phi)).astype(f),
                 (pm * u).astype(f), rng.uniform(0, 1, n).astype(f), rng.uniform(0, 1, n).astype(f),
                 rng.uniform(0, 1, n).astype(f))
    sp.px[rng.uniform(size=n) < 0.03] = 0.0  # a few on an axis plane
    return sp


def make(ncells, acap):
    prm = dict(g_agg_GeV_inv=1e-10, g_ae=1e-12, dt_phys_s=2e12, w_a=3.0e9, seed=7, tally_enable=0)
    return AxionPlasma(ncells, np.full(ncells, 2.0), np.full((ncells, 1), 6e25), [1.0], [1.00794], 1e-12,
                       (4, 4, acap), prm)


def gpu_cell(slab, c):
    d = slab.cell(c)
    return Species(*[d[f].astype(np.float32) for f in FIELDS])


def assert_cell_equal(g, w, c):
    assert len(g) == len(w), (c, len(g), len(w))
    for f in FIELDS:
        assert np.array_equal(getattr(g, f), np.asarray(getattr(w, f), dtype=np.float32)), (c, f)


@pytest.mark.parametrize("n_target", [0, 24, 80])
def test_merging_matches_oracle(n_target):
    rng = np.random.default_rng(100 + n_target)
    n, cap = 90, 192
    counts = [0, 1, 2, 3, cap] + [int(v) for v in rng.integers(0, 160, n - 5)]
    cells = [random_axions(rng, k) for k in counts]
    # degenerate groups: zero momenta (P = 0) and identical axions (cos theta = 1)
    f = np.float32
    z = np.zeros(40, f)
    cells[5] = Species(np.full(40, 1.25, f), z, z, z, np.full(40, .5, f), np.full(40, .5, f), np.full(40, .5, f))
    same = random_axions(rng, 1)
    cells[6] = Species(*[np.repeat(v, 60) for v in same.fields()])
    pl = make(n, cap)
    for c, sp in enumerate(cells):
        pl.slabs["axions"].set_cell(c, {f: getattr(sp, f) for f in FIELDS})
    torch.cuda.synchronize()
    pl.merge_axions(n_target, EDGES)
    want, removed = MG.merge(cells, n_target, EDGES)
    torch.cuda.synchronize()
    for c in range(n):
        assert_cell_equal(gpu_cell(pl.slabs["axions"], c), want[c], c)
    assert pl.merge_stats() == removed
    if n_target < 80:
        assert removed > 0
    pl.close()


def test_large_cells_fewer_warps_per_block():
    """Capacities of 12000 and 40000 slots leave room for six and two warps'
    member lists in a block; cells of thousands of axions, groups of
    hundreds, equal the oracle bit for bit."""
    for cap, counts in ((12000, [0, 11000, 12000, 37]), (40000, [40000, 25000])):
        rng = np.random.default_rng(cap)
        cells = [random_axions(rng, k) for k in counts]
        pl = make(len(counts), cap)
        for c, sp in enumerate(cells):
            pl.slabs["axions"].set_cell(c, {f: getattr(sp, f) for f in FIELDS})
        torch.cuda.synchronize()
        pl.merge_axions(30, EDGES)
        want, removed = MG.merge(cells, 30, EDGES)
        torch.cuda.synchronize()
        for c in range(len(counts)):
            assert_cell_equal(gpu_cell(pl.slabs["axions"], c), want[c], c)
        assert pl.merge_stats() == removed
        pl.close()


def test_invalid_merge_arguments_launch_nothing():
    pl = make(4, 8)
    for args in ((-1, EDGES), (4, EDGES[::-1]), (4, np.array([np.nan], np.float32)),
                 (4, np.zeros(31, np.float32) + np.arange(31, dtype=np.float32))):
        with pytest.raises(_lib.AxpicError):
            pl.merge_axions(*args)
    assert pl.merge_stats() == 0.0
    pl.close()


def test_relaxation_size_conserves_and_matches_sampled_cells():
    """The 256 x 256 relaxation plasma with 160 MB-equilibrium axions a cell
    merged down toward 64: every cell keeps its weight, momentum and energy
    (to binary32 rounding), and 16 sampled cells equal the oracle."""
    w = workloads.config2(256, 256)
    w.params["w_a"] = float(np.float32(workloads.photon_weight(3.0, w.volume_cm3, w.n_ph) * w.w_a_over_w_gamma))
    w.params.update(seed=0, tally_enable=0)
    pl = AxionPlasma(w.ncells, w.T_keV, w.n_ion, w.Z, w.A, w.volume_cm3, w.caps, w.params)
    pl.sample(w.n_el, w.n_ph, 160)
    torch.cuda.synchronize()
    slab = pl.slabs["axions"]
    sample = np.random.default_rng(4).choice(w.ncells, 16, replace=False)
    before = {c: gpu_cell(slab, c) for c in sample}

    def moments():
        cap = slab.capacity
        cnt = slab.count[:w.ncells].long()
        m = (torch.arange(cap, device=cnt.device)[None, :] < cnt[:, None]).double()
        d = {f: slab.data[f][:w.ncells * cap].view(w.ncells, cap).double() * m for f in FIELDS}
        pm = torch.sqrt(d["px"] ** 2 + d["py"] ** 2 + d["pz"] ** 2)
        return (d["w"].sum(1), (d["w"] * d["px"]).sum(1), (d["w"] * d["py"]).sum(1), (d["w"] * d["pz"]).sum(1),
                (d["w"] * pm).sum(1))

    m0 = moments()
    n0 = int(slab.count[:w.ncells].sum())
    pl.merge_axions(64, EDGES)
    torch.cuda.synchronize()
    m1 = moments()
    n1 = int(slab.count[:w.ncells].sum())
    assert n0 - n1 == pl.merge_stats() and n1 < 0.8 * n0
    W0, E0 = m0[0], m0[4]
    assert torch.all((m1[0] - W0).abs() <= 2e-6 * W0)
    assert torch.all((m1[4] - E0).abs() <= 2e-6 * E0)
    for k in (1, 2, 3):
        assert torch.all((m1[k] - m0[k]).abs() <= 2e-6 * E0)
    for c in sample:
        want, _ = MG.merge_cell(before[c], 64, EDGES)
        assert_cell_equal(gpu_cell(slab, c), want, c)
    pl.close()
