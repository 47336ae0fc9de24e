"""Batched boxes in one context, graph replay of the step and the launch-shape
autotuner, through the C ABI: against the oracle and against plain step calls
(needs a GB300 and the built library)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from parity_util import assert_species_close, oracle_step

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2604_24627_gb300 import AxionPlasma, _lib, workloads  # noqa: E402

A_H, A_HE = 1.00794, 4.002602
MIX_Z = np.array([1.0, 2.0])
MIX_A = np.array([A_H, A_HE])


def base_params(**kw):
    prm = dict(g_agg_GeV_inv=1e-10, g_ae=1e-12, dt_phys_s=2e12, w_a=3.0e9, seed=0x1234_0000_0042,
               T_mode=2, relax_r=0.1, diag_enable=1, tally_enable=1)
    prm.update(kw)
    return prm


def make(ncells, prm, T=None, caps=(64, 192, 512), counts=(61, 37, 13)):
    T = np.linspace(1.3, 5.0, ncells) if T is None else T
    n = 6e25 / 1.1
    n_ion = np.tile([[0.9 * n, 0.1 * n]], (ncells, 1))
    pl = AxionPlasma(ncells, T, n_ion, MIX_Z, MIX_A, 1e-12, caps, prm)
    pl.sample(*counts)
    torch.cuda.synchronize()
    return pl


def state(pl):
    """Host copy of everything a step changes: valid slots of every species,
    counts, T, carried exchange."""
    out = {}
    for name, slab in pl.slabs.items():
        cnt = slab.count[:pl.ncells].cpu().numpy()
        out[name + ".count"] = cnt
        valid = (np.arange(slab.capacity)[None, :] < cnt[:, None]).reshape(-1)
        for f, t in slab.data.items():
            out[name + "." + f] = t[:pl.ncells * slab.capacity].cpu().numpy()[valid]
    out["T"] = pl.temperatures()
    out["res"] = pl.residuals()
    return out


def assert_same(a, b, what):
    assert a.keys() == b.keys()
    for k in a:
        assert a[k].shape == b[k].shape, (what, k, a[k].shape, b[k].shape)
        diff = np.flatnonzero(a[k].view(np.uint8) != b[k].view(np.uint8))
        assert diff.size == 0, (what, k, diff[:8])


def test_run_steps_equals_step_calls():
    prm = base_params()
    a, b = make(40, prm), make(40, prm)
    for s in range(5):
        a.step(s, _lib.CH_ALL)
    b.run_steps(0, 3, _lib.CH_ALL)   # captures the graph
    b.run_steps(3, 2, _lib.CH_ALL)   # replays it from another first step
    torch.cuda.synchronize()
    assert_same(state(a), state(b), "graph replay")
    _, ta = a.tally()
    _, tb = b.tally()
    for k in ta:  # FP64 tallies are sums by atomics: order-dependent rounding
        assert abs(ta[k] - tb[k]) <= 1e-12 * abs(ta[k]), (k, ta[k], tb[k])
    a.close()
    b.close()


@pytest.mark.parametrize("branches", [1, 2, 8])
def test_branched_replay_equals_step_calls(branches):
    """Replayed steps whose cells run as several branches (ranges of whole
    event CTAs on forked streams, each with its own step counter, joined
    every 32 steps) give what plain step calls give: 35 steps take one graph
    of 32 steps and three of one step."""
    prm = base_params(step_branches=branches)
    caps = (64, 1024, 2048)  # no product dropped in 35 steps at these rates
    a, b = make(600, prm, caps=caps), make(600, prm, caps=caps)
    for s in range(35):
        a.step(s, _lib.CH_ALL)
    b.run_steps(0, 35, _lib.CH_ALL)
    torch.cuda.synchronize()
    assert_same(state(a), state(b), "%d branches" % branches)
    assert a.tally()[1]["dropped"] == 0
    a.close()
    b.close()


def make_h(ncells, prm, T=None, caps=(64, 1024, 2048), counts=(61, 37, 13)):
    """A hydrogen plasma (the rate models' records need one ion species)."""
    T = np.linspace(1.3, 5.0, ncells) if T is None else T
    pl = AxionPlasma(ncells, T, np.full((ncells, 1), 6e25), [1.0], [A_H], 1e-12, caps, prm)
    pl.sample(*counts)
    torch.cuda.synchronize()
    return pl


@pytest.mark.parametrize("model", [1, 2])
def test_branched_replay_with_records_equals_step_calls(model):
    """Evolved-T steps with spectral records (exact table; network trusted
    everywhere, table nowhere): a replay in branches (4 asked, 3 formed), each rebuilding its
    own cells' records after its temperature update, gives what plain step
    calls give, records included."""
    from paper_2604_24627_gb300.mlp import SurrogateNet
    prm = base_params(step_branches=4, rate_model=model, sr_table_nkt=24, sr_table_nne=12)
    a, b = make_h(600, prm), make_h(600, prm)
    if model == 2:
        net = SurrogateNet()
        _lib.axpic_surrogate_fit(net.h, 2048, 1, 400, 2048, 2e-3, 5)
        err = np.zeros(2 * 4 * 4 * 3, dtype=np.float32)
        for pl in (a, b):
            _lib.axpic_set_surrogate(pl.ctx, net.h, err, 4, 4, 1.0, 1.0)
        net.close()
    for s in range(35):
        a.step(s, _lib.CH_ALL)
    b.run_steps(0, 35, _lib.CH_ALL)
    torch.cuda.synchronize()
    assert_same(state(a), state(b), "records of model %d" % model)
    assert_same_records(a, b, 600)
    assert b.launch_shape()[2] == 3  # 600 cells in ranges of whole 128-cell CTAs: 256, 256, 88
    a.close()
    b.close()


def rate_records(pl, n):
    """Cell records, their sources and the spectral records of the cells
    whose rates come from one (the others' are unused)."""
    rec, src = _lib.axpic_get_cell_records(pl.ctx, 0, n)
    sr = _lib.axpic_get_spectral_records(pl.ctx, 0, n)
    sr[src == 0] = 0.0
    return rec, src, sr


def assert_same_records(a, b, n):
    for x, y in zip(rate_records(a, n), rate_records(b, n)):
        assert np.array_equal(x, y)


def test_records_rebuilt_in_a_step_equal_a_rebuild_from_scratch():
    """Cells whose trust changes as T evolves: the records the feedback kernel
    rebuilds after its temperature update (the network's prefactors where it
    is trusted, the table's record elsewhere) equal the ones a rebuild from
    scratch gives for the same temperatures."""
    from paper_2604_24627_gb300.mlp import SurrogateNet
    prm = base_params(rate_model=2, relax_r=1.0, sr_table_nkt=24, sr_table_nne=12)
    T = np.linspace(1.0, 7.0, 300)
    pl = make_h(300, prm, T=T, caps=(64, 4096, 4096))
    net = SurrogateNet()
    _lib.axpic_surrogate_fit(net.h, 2048, 1, 400, 2048, 2e-3, 5)
    nT, nne = 8, 4
    err = np.zeros((2, nne, nT, 3), dtype=np.float32)
    err[:, :, 3:5, 0] = 1.0  # an untrusted band of temperatures between two trusted ones: cells cross its borders
    _lib.axpic_set_surrogate(pl.ctx, net.h, err, nT, nne, 1e-3, 1e-3)
    net.close()
    _, src0 = _lib.axpic_get_cell_records(pl.ctx, 0, 300)
    for s in range(4):
        pl.step(s, _lib.CH_ALL)
    torch.cuda.synchronize()
    in_step = rate_records(pl, 300)
    assert np.any(in_step[1] != src0)  # some cells changed sides
    assert 0 < in_step[1].sum() < 300
    _lib.axpic_update_cells(pl.ctx)
    fresh = rate_records(pl, 300)
    for x, y in zip(in_step, fresh):
        assert np.array_equal(x, y)
    pl.close()


def test_checkpoint_and_resume_continue_bit_for_bit():
    """10 steps in one context equal 5 steps, a save (the caller's slabs and
    T, the library's state), a load into a new context and 5 more steps
    (evolved T, residual carry, cached moments, counters)."""
    prm = base_params()
    a, b = make(48, prm), make(48, prm)
    for s in range(10):
        a.step(s, _lib.CH_ALL)
    for s in range(5):
        b.step(s, _lib.CH_ALL)
    torch.cuda.synchronize()
    slabs = {name: ({f: t.clone() for f, t in slab.data.items()}, slab.count.clone()) for name, slab in b.slabs.items()}
    T = b.T.clone()
    saved = b.save_state()
    assert saved.size > 0
    b.close()
    c = make(48, prm, T=np.full(48, 2.0))  # another start: everything is overwritten
    for name, (data, count) in slabs.items():
        for f, t in data.items():
            c.slabs[name].data[f].copy_(t)
        c.slabs[name].count.copy_(count)
    c.T.copy_(T)
    c.load_state(saved)
    with pytest.raises(_lib.AxpicError):
        c.load_state(saved[:-8])
    for s in range(5, 10):
        c.step(s, _lib.CH_ALL)
    torch.cuda.synchronize()
    assert_same(state(a), state(c), "resumed")
    ta, tc = a.tally()[1], c.tally()[1]
    for k in ta:  # counts exactly, FP64 atomic sums (order-dependent) to 1e-12
        assert abs(ta[k] - tc[k]) <= 1e-12 * max(1.0, abs(ta[k])), (k, ta[k], tc[k])
    a.close()
    c.close()


@pytest.mark.parametrize("chunk,tpb", [(4, 32), (8, 64), (16, 128), (32, 64)])
def test_launch_shapes_give_identical_results(chunk, tpb):
    ref = make(29, base_params())
    other = make(29, base_params(decide_chunk=chunk, threads_per_block=tpb))
    for s in range(3):
        ref.step(s, _lib.CH_ALL)
        other.step(s, _lib.CH_ALL)
    torch.cuda.synchronize()
    assert_same(state(ref), state(other), "chunk %d tpb %d" % (chunk, tpb))
    ref.close()
    other.close()


def test_autotune_restores_state_and_keeps_results():
    prm = base_params()
    a, b = make(48, prm), make(48, prm)
    for s in range(2):
        a.step(s, _lib.CH_ALL)
        b.step(s, _lib.CH_ALL)
    torch.cuda.synchronize()
    before = state(a)
    ms, chunk, warps = a.autotune(2, 2, _lib.CH_ALL)
    assert ms > 0 and chunk in (4, 8, 16, 32) and warps in (2, 4), (ms, chunk, warps)
    assert_same(before, state(a), "after autotune")
    for s in range(2, 4):
        a.step(s, _lib.CH_ALL)
        b.step(s, _lib.CH_ALL)
    a.run_steps(4, 1, _lib.CH_ALL)
    b.step(4, _lib.CH_ALL)
    torch.cuda.synchronize()
    assert_same(state(a), state(b), "tuned shape")
    a.close()
    b.close()


def test_batched_boxes_match_oracle():
    """Uneven hydrogen boxes with their own T and n_e concatenated in one
    context: every cell's step equals the oracle's step of that cell."""
    counts = np.array([1, 5, 2, 13, 3, 7])
    T_box = np.array([1.2, 4.6, 2.5, 3.1, 1.8, 4.9])
    ne_box = np.array([1e24, 8e25, 6e25, 2e25, 1e26, 5e24])
    box = np.repeat(np.arange(len(counts)), counts)
    ncells = int(counts.sum())
    T = T_box[box]
    n_ion = ne_box[box].reshape(ncells, 1)
    Z, A = np.array([1.0]), np.array([A_H])
    prm = base_params(g_ae=2e-12)
    pl = AxionPlasma(ncells, T, n_ion, Z, A, 1e-12, (64, 192, 512), prm)
    pl.sample(61, 37, 13)
    pl.run_steps(0, 1, _lib.CH_ALL)
    torch.cuda.synchronize()
    before = [pl.cell(c) for c in range(ncells)]
    T_before = pl.temperatures().copy()
    res_before = pl.residuals()
    pl.run_steps(1, 1, _lib.CH_ALL)
    torch.cuda.synchronize()
    diag = pl.cell_diag()
    for c in range(ncells):
        got = pl.cell(c)
        parts, tally, fb = oracle_step(before[c], T_before[c], n_ion[c], Z, A, prm, 1, c, _lib.CH_ALL,
                                       res=res_before[c])
        what = "box %d cell %d" % (box[c], c)
        assert_species_close(got["a"], parts["a"], what + " axions")
        assert_species_close(got["g"], parts["g"], what + " photons")
        assert abs(diag[c][0] - tally.dE) <= 1e-5 * tally.gross_E + 1e-30, (what, diag[c][0], tally.dE)
    _, tot = pl.tally()
    assert tot["dropped"] == 0
    pl.close()


def test_c4_workload_slice_runs():
    """A slice of the 4096-box workload (first 12 boxes) through autotune and
    graph replay: populations stay within the slabs and every cell keeps its
    box's temperature range."""
    w = workloads.config4(nboxes=12, seed=3)
    prm = dict(w.params)
    prm["w_a"] = float(np.float32(workloads.photon_weight(3.0, w.volume_cm3, w.n_ph)))
    prm["tally_enable"] = 0
    pl = AxionPlasma(w.ncells, w.T_keV, w.n_ion, w.Z, w.A, w.volume_cm3, w.caps, prm)
    pl.sample(w.n_el, w.n_ph, w.n_ax)
    pl.autotune(0, 2, w.mask)
    pl.run_steps(0, 10, w.mask)
    torch.cuda.synchronize()
    _, tot = pl.tally()
    assert tot["dropped"] == 0
    cnt = pl.counts()
    assert cnt["electrons"].min() == w.n_el and cnt["axions"].max() <= w.caps[2]
    assert np.all(np.isfinite(pl.temperatures()))
    pl.close()


@pytest.mark.parametrize("model", [0, 1, 2])
def test_steps_over_cell_ranges_equal_step_calls(model):
    """Each step run as ragged, disjoint cell ranges in a shuffled order
    (axpic_step_cells; closed-form, exact-table and surrogate rate models)
    gives what plain step calls give; a range outside the context launches
    nothing."""
    prm = base_params(rate_model=model)
    caps = (64, 1024, 2048)
    a, b = make_h(300, prm, caps=caps), make_h(300, prm, caps=caps)
    if model == 2:
        from paper_2604_24627_gb300.mlp import SurrogateNet
        net = SurrogateNet()
        _lib.axpic_surrogate_fit(net.h, 2048, 1, 400, 2048, 2e-3, 5)
        err = np.zeros((2, 4, 8, 3), dtype=np.float32)
        err[:, :, 2:4, 0] = 1.0  # part of the cells on the table
        for pl in (a, b):
            _lib.axpic_set_surrogate(pl.ctx, net.h, err, 8, 4, 1e-3, 1e-3)
        net.close()
    cuts = [0, 1, 128, 131, 257, 300]
    order = np.random.default_rng(5).permutation(len(cuts) - 1)
    for s in range(6):
        a.step(s, _lib.CH_ALL)
        for r in order:
            b.step_cells(s, cuts[r], cuts[r + 1] - cuts[r])
        b.step_cells(s, 300, 0)
    torch.cuda.synchronize()
    assert_same(state(a), state(b), "cell ranges")
    if model:
        assert_same_records(a, b, 300)
    for args in ((0, 250, 51), (0, -1, 2), (-1, 0, 4)):
        with pytest.raises(_lib.AxpicError):
            b.step_cells(args[0], args[1], args[2])
    a.close()
    b.close()
