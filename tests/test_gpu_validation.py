"""Stochastic validation of the CUDA path at size, through the C ABI (needs a
GB300): every cell of a relaxed 4096-cell plasma against the oracle under
identical Philox keys, the Primakoff spectrum and power of the 1-D
photon-bath workload against the screened closed form, the thermal-bath
relaxation against the closed-form detailed-balance trajectory, and shards
of cells in separate contexts against one context."""
import math
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import constants as K
from oracle import plasma
from oracle import step as ostep
from oracle import tally as otally
from oracle.plasma import Params as OParams
from parity_util import FIELDS, assert_species_close, oracle_params, to_species

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2604_24627_gb300 import AxionPlasma, _lib, workloads  # noqa: E402
from paper_2604_24627_gb300 import dist as pdist  # noqa: E402


def host_state(pl):
    """Every slab, count and T on the host at once (per-cell views follow)."""
    out = {}
    for name, slab in pl.slabs.items():
        out[name] = ({f: t[:pl.ncells * slab.capacity].cpu().numpy().reshape(pl.ncells, slab.capacity)
                      for f, t in slab.data.items()}, slab.count[:pl.ncells].cpu().numpy(), slab.capacity)
    return out


def cell_of(hs, c):
    d = {}
    for k, name in zip("ega", ("electrons", "photons", "axions")):
        data, cnt, _ = hs[name]
        n = int(cnt[c])
        d[k] = {f: data[f][c, :n].astype(np.float64) for f in FIELDS}
    return d


def test_every_cell_of_a_relaxed_plasma_matches_the_oracle():
    """4096 cells of the 256 x 256 relaxation plasma (90 % H + 10 % He by
    number, n_e = 6e25, T = 3 keV evolved, 512 electrons, 256 photons and
    107 Maxwell-Boltzmann-equilibrium axions per cell: the relaxed axion
    population), all channels forward and inverse, two steps: with
    identical Philox keys at least 99.99 % of the 8192 cell-steps (here:
    all of them) leave the same particles as the oracle's step of that cell,
    so every per-cell event count agrees."""
    w = workloads.config2(64, 64)
    w.params["w_a"] = float(np.float32(workloads.photon_weight(3.0, w.volume_cm3, w.n_ph)))
    prm = dict(w.params, seed=0, tally_enable=1)
    pl = AxionPlasma(w.ncells, w.T_keV, w.n_ion, w.Z, w.A, w.volume_cm3, (512, 384, 384), prm)
    pl.sample(512, 256, 107)
    torch.cuda.synchronize()
    bad, events = 0, 0
    for step in range(2):
        hs = host_state(pl)
        T = pl.temperatures().copy()
        res = pl.residuals()
        pl.step(step, _lib.CH_ALL)
        torch.cuda.synchronize()
        after = host_state(pl)
        op = oracle_params(prm)
        for c in range(w.ncells):
            before = cell_of(hs, c)
            parts = {k: to_species(before[k]) for k in "ega"}
            ci = ostep.CellInput(float(T[c]), w.n_ion[c], w.Z, w.A)
            tally, _ = ostep.step_cell(ci, parts, op, step, c, _lib.CH_ALL, res[c][0], np.asarray(res[c][1:4]))
            events += sum(tally.events.values()) + sum(tally.absorbed.values())
            got = cell_of(after, c)
            try:
                for k in "ag":
                    assert_species_close(got[k], parts[k], "cell %d %s" % (c, k))
            except AssertionError:
                bad += 1
    n = 2 * w.ncells
    assert events > 10000, events
    assert bad <= int(1e-4 * n), (bad, n)
    pl.close()


def test_c1_primakoff_spectrum_against_the_screened_closed_form():
    """The 1-D photon-bath workload (hydrogen, T = 1.3 keV, n_e = 6e25,
    Planck photons, Primakoff gamma->a only, w_a = w_gamma / 4, dt giving
    about 0.1 events per 128-photon cell and step) in binary32 on the GPU:
    64000 cells of 128 photons, forward emission only, 10 emission steps from
    the same photons. The emitted spectrum (160 bins of 0.5 keV, summed into
    2 keV bins) passes a chi^2 test against the expectation over the sampled
    photons from the FP64 closed form (Eqs. prim_rate, prim_prob), the total
    emitted energy agrees with it within 4 sigma, and the power agrees with
    the Planck-law screened closed form within 1.5 % (about 3 sigma of the
    event noise; Table II reports Primakoff Q ratios 0.992-1.00)."""
    w = workloads.config1(64000)
    wg = workloads.photon_weight(1.3, w.volume_cm3, w.n_ph)
    prm = dict(w.params, w_a=float(np.float32(wg * w.w_a_over_w_gamma)), seed=0, tally_enable=1)
    pl = AxionPlasma(w.ncells, w.T_keV, w.n_ion, w.Z, w.A, w.volume_cm3, w.caps, prm)
    pl.sample(0, 128, 0)
    torch.cuda.synchronize()
    hs = host_state(pl)
    data, cnt, cap = hs["photons"]
    wgam = data["w"].astype(np.float64).reshape(-1)
    E = np.sqrt(data["px"].astype(np.float64) ** 2 + data["py"] ** 2 + data["pz"] ** 2).reshape(-1) * K.ME_C2_KEV
    op = oracle_params(prm)
    cs = plasma.cell_state(1.3, np.array([6e25]), np.array([1.0]), np.array([K.A_H]), op)
    P = ostep.primakoff_prob(cs, op, E)
    wa = float(np.float32(op.w_a))
    lam = wgam * P / wa                      # Poisson mean per photon: products of weight w_a
    nb, Emax, steps = 160, 80.0, 10
    kb = np.minimum((E / (Emax / nb)).astype(int), nb - 1)
    exp_bin = np.bincount(kb, weights=lam * wa * E, minlength=nb) * steps
    var_bin = np.bincount(kb, weights=lam * (wa * E) ** 2, minlength=nb) * steps
    pl.tally()
    for s in range(steps):
        pl.sample(0, 128, 0)                 # the same photons again (keyed sampler): independent draws per step
        pl.emit(s, _lib.CH_PRIMAKOFF)
    H, tot = pl.tally()
    h = H[0]
    assert tot["events_p"] > 4e4, tot["events_p"]
    # chi^2 over 2 keV bins holding at least 50 expected events
    hc, ec, vc = h.reshape(40, 4).sum(1), exp_bin.reshape(40, 4).sum(1), var_bin.reshape(40, 4).sum(1)
    use = ec ** 2 / np.maximum(vc, 1e-300) > 50
    chi2 = float(np.sum((hc[use] - ec[use]) ** 2 / vc[use]))
    dof = int(use.sum())
    assert dof >= 8, dof
    assert chi2 < dof + 5 * math.sqrt(2 * dof), (chi2, dof)
    # total emitted energy against the expectation over these photons
    assert abs(h.sum() - exp_bin.sum()) < 4 * math.sqrt(var_bin.sum()), (h.sum(), exp_bin.sum())
    # power against the Planck-law closed form, Q = int E (P/dt) dn_gamma/dE dE
    edges = np.linspace(0, Emax, nb + 1)
    ref = otally.bin_average(lambda x: otally.primakoff_dQdE(cs, op, np.maximum(x, 1e-9)), edges)
    Q_ref = float(np.sum(ref) * Emax / nb)
    dQ = otally.absolute_dQdE(h, w.ncells * w.volume_cm3, steps * op.dt_phys_s, Emax / nb)
    Q_mc = float(np.sum(dQ) * Emax / nb)
    assert abs(Q_mc / Q_ref - 1) < 0.015, (Q_mc, Q_ref)
    pl.close()


def _expected_relaxation(cs, p, ch, V, ks):
    """N(k), U(k) after k steps of absorb -> emit from an empty start, per
    energy n_k(E) = S(E) (1 - (1 - P(E))^k) / P(E) with S = d ndot/dE V dt /
    w_a and P = 1 - exp(-Gamma_abs dt) (Eq. gamma_abs): the closed-form
    detailed-balance trajectory."""
    from scipy import integrate

    def integrand(E, k, power):
        Pa = -np.expm1(-plasma.absorption_rate(cs, ch, E, p) * p.dt_phys_s)
        src = plasma.differential_emission(cs, ch, E, p) * V * p.dt_phys_s
        return src * (1 - (1 - Pa) ** k) / Pa * (E if power else 1.0)
    N = np.array([integrate.quad(integrand, 1e-9, 40 * cs.T_keV, args=(k, 0), limit=400)[0] for k in ks])
    U = np.array([integrate.quad(integrand, 1e-9, 40 * cs.T_keV, args=(k, 1), limit=400)[0] for k in ks])
    return N, U


@pytest.mark.parametrize("ch,eq_stats,T", [(2, 0, 3.0), (4, 1, 1.3)])
def test_thermal_bath_relaxation_reaches_the_detailed_balance_plateau(ch, eq_stats, T):
    """Compton-like (Maxwell-Boltzmann target) and bremsstrahlung (Bose-
    Einstein target) alone, fixed T, 256 cells of 256 electrons from an
    axion-free start, absorb -> emit each step (dt: absorption probability
    0.05 at x = 3): the alive axion number and energy follow the closed-form
    trajectory to their plateau within 2 % (N) and 3 % (U) over steps
    120-240, and the plateau is the equilibrium n_eq V times the
    steady-state factor of the absorb -> emit order."""
    V, ncells = 1e-12, 256
    name = "compton" if ch == 2 else "brems"
    op = OParams(g_ae=1e-13, seed=8, eq_stats=eq_stats)
    cs = plasma.cell_state(T, np.array([6e25]), np.array([1.0]), np.array([K.A_H]), op)
    op.dt_phys_s = 0.05 / plasma.absorption_rate(cs, name, np.array([3 * T]), op)[0]
    n_eq = T ** 3 / (math.pi ** 2 * K.HBARC_KEV_CM ** 3)
    if eq_stats == 1:
        from scipy import special
        n_eq *= special.zeta(3)
    op.w_a = float(np.float32(n_eq * V / 1500))
    prm = dict(g_ae=1e-13, seed=8, eq_stats=eq_stats, dt_phys_s=op.dt_phys_s, w_a=op.w_a, T_mode=0,
               tally_enable=1)
    pl = AxionPlasma(ncells, T, np.full((ncells, 1), 6e25), [1.0], [K.A_H], V, (256, 4, 4096), prm)
    pl.sample(256, 0, 0)
    torch.cuda.synchronize()
    ks = np.arange(120, 241, 10)
    N, U = [], []
    k = 0
    for target in ks:
        while k < target:
            pl.absorb(k, ch)
            pl.emit(k, ch)
            k += 1
        _, tot = pl.tally()
        N.append(tot["n_axions"] / ncells)
        U.append(tot["u_axions"] / ncells)
    Ne, Ue = _expected_relaxation(cs, op, name, V, ks)
    assert abs(np.mean(N) / Ne.mean() - 1) < 0.02, (np.mean(N), Ne.mean())
    assert abs(np.mean(U) / Ue.mean() - 1) < 0.03, (np.mean(U), Ue.mean())
    ratio = Ne[-1] / (n_eq * V)
    assert 0.8 < ratio < 1.3, ratio
    pl.close()


# ---------------------------------------------------------------- shards
NSHARD_CELLS = 200


def _shard_prm():
    return dict(g_agg_GeV_inv=1e-10, g_ae=2e-12, dt_phys_s=2e12, w_a=3.0e9, seed=0x5151, T_mode=2, relax_r=0.1,
                tally_enable=1)


def _shard_T():
    return np.linspace(1.3, 5.0, NSHARD_CELLS)


def _run_cells(first, count, steps=6):
    """A context over cells [first, first + count) of the plasma, with their
    global indices (cell_index_base = first); returns its host state and
    tally after `steps` steps."""
    T = _shard_T()[first:first + count]
    pl = AxionPlasma(count, T, np.full((count, 1), 6e25), [1.0], [K.A_H], 1e-12, (64, 1024, 2048), _shard_prm(),
                     cell_index_base=first)
    pl.sample(61, 37, 13)
    for s in range(steps):
        pl.step(s, _lib.CH_ALL)
    torch.cuda.synchronize()
    st = {name: (data, cnt) for name, (data, cnt, _) in host_state(pl).items()}
    st["T"] = pl.temperatures().copy()
    H, tot = pl.tally()
    pl.close()
    return st, H, tot


def _shard_worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    first, count = pdist.shard_range(NSHARD_CELLS, world, rank)
    st, H, tot = _run_cells(first, count)
    Hs, tots = pdist.allreduce_tally(H, tot, dist)
    q.put((rank, first, st, Hs, tots))
    dist.destroy_process_group()


def test_two_context_shards_equal_one_context():
    """Two processes (gloo ranks) each step their contiguous shard of the
    cells in a context of their own with cell_index_base at the shard's
    first cell: the particles, counts and temperatures equal one context's
    over all cells bit for bit, and the tallies summed across the ranks
    (dist.allreduce_tally) equal its tally (FP64 sums to 1e-12, counters
    exactly)."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=600) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    whole, H1, tot1 = _run_cells(0, NSHARD_CELLS)
    for rank, first, st, Hs, tots in got:
        n = len(st["T"])
        assert np.array_equal(st["T"].view(np.uint64), whole["T"][first:first + n].view(np.uint64))
        for name in ("electrons", "photons", "axions"):
            data, cnt = st[name]
            wdata, wcnt = whole[name]
            assert np.array_equal(cnt, wcnt[first:first + n]), name
            for f in FIELDS:
                for c in range(n):
                    k = int(cnt[c])
                    assert np.array_equal(data[f][c, :k].view(np.uint32), wdata[f][first + c, :k].view(np.uint32)), \
                        (name, f, first + c)
        np.testing.assert_allclose(Hs, H1, rtol=1e-12, atol=1e-300)
        for key in tot1:
            if key.startswith(("events", "absorbed", "cap", "clamp", "dropped", "macro", "remaps", "part", "calls")):
                assert tots[key] == tot1[key], key
            else:
                assert abs(tots[key] - tot1[key]) <= 1e-12 * max(1.0, abs(tot1[key])), key
    assert tot1["events_p"] + tot1["events_pinv"] > 0
