"""Throughput of the axion Monte-Carlo step on GB300.

One "step" is one fused pass of the whole hot path (absorb -> emit ->
feedback -> temperature update) over every cell of the workload. The default
workload is the 3-D 256^3 hydrogen plasma (16.8 M cells, T_e = 5 keV evolved,
n_e = 6e25 cm^-3, 64 Maxwellian electrons, 32 Planck photons and 13
Maxwell-Boltzmann-equilibrium axions per cell at the start: about 1.8e9
macroparticles), forward and inverse operators of all three channels,
binary32 rates with FP64 exchange buffers and temperature, under three rate
models: the closed forms, the exact FP32 table, and the surrogate network
(trained first by the library's own tensor-core kernels; the table where its
validated error is above the bound). The reported value is the surrogate
model's; the line carries the table's and the closed forms' beside it.

Metric: particle-steps/s = sum over timed steps of the particles (electrons +
photons + axions) present at the start of the step / device time. Under
torchrun every rank runs its own full-size plasma (weak scaling, no
data-path collective) and rank 0 reports the aggregate.

--impl reference times the oracle (plain FP64 CPU) on bounded samples of the
same workload on the host cores.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s, 3-channel emit+absorb; surrogate vs table at ≤1e-3 rate err"
# The network is trusted where the four validation nodes around a cell and
# their neighbours are within 6e-4 on the rates (the bound is 1e-3): on
# 10,000 sampled cells the worst trusted cell was then 8.2e-4 off.
TRUST_TOL = 6e-4
UNIT = "particle-steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 1000 for c2, the workload's own 100 for c3 and c4)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--e2e-ranges", type=int, default=4, help="cell ranges pipelined in the end-to-end leg")
    ap.add_argument("--stream-calls", type=int, default=20,
                    help="timed axion streaming calls after the other legs (0: none)")
    ap.add_argument("--merge-n-target", type=int, default=64,
                    help="timed axion merging call after the other legs, toward this many a cell (0: none)")
    ap.add_argument("--merge-calls", type=int, default=10, help="timed merging calls, each on the same state")
    ap.add_argument("--deposit-calls", type=int, default=10, help="timed composition deposits (0: none)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nx", type=int, default=256, help="cells per side (256: the full workload)")
    ap.add_argument("--workload", default="c5", choices=["c2", "c3", "c4", "c5"],
                    help="c5: the 256^3 plasma, surrogate vs table vs closed-form rates (the reported line); "
                         "c2: the 256x256 relaxation; c3: 512x512 temperature bump, surrogate vs table vs "
                         "closed-form rates; c4: 4096 uneven boxes in one context, autotuned launch shape, steps "
                         "replayed as a CUDA graph")
    ap.add_argument("--c5-side", type=int, default=256, help="cells per side of the c5 plasma (256: the full one)")
    ap.add_argument("--e2e-cells", type=int, default=0,
                    help="c5: cells of the end-to-end leg's sample (0: a sixteenth of the plasma)")
    ap.add_argument("--rate-err-cells", type=int, default=512, help="sampled cells for the rate-model errors")
    ap.add_argument("--boxes", type=int, default=4096, help="boxes of the c4 workload")
    ap.add_argument("--branches", type=int, default=0,
                    help="c3: cell branches of a replayed step (1, 2, 4 or 8; 0: the library's choice)")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = {"c2": 1000, "c5": 20}.get(args.workload, 100)
    return args


def workload(nx=256):
    from paper_2604_24627_gb300 import workloads
    w = workloads.config2(nx, nx)
    wg = workloads.photon_weight(3.0, w.volume_cm3, w.n_ph)
    w.params["w_a"] = float(np.float32(wg * w.w_a_over_w_gamma))
    w.params["seed"] = 0
    w.params["tally_enable"] = 0
    return w


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_bytes(tot, T_mode):
    """Algorithmic DRAM bytes of each kernel of the step, summed over the timed
    steps.

    "step": the minimum of a fused cell-local pass with feedback every step,
    28 B per electron (w, p read, p written), 16 B per photon and 16 B per
    axion (w, p read); the step's roofline is taken against it.

    Each kernel is charged the minimum it moves:
      decisions: w, p of every axion and photon present (16 B), w of
        electrons in cells without a common weight (4 B; 0 here) + counts,
        snapshot, record words and common weight per cell (48 B);
      events: the decision masks (1 bit per particle), counts, snapshot and
        flags per cell (40 B), each product written (28 B) with its parent's
        w, p and position read (28 B), each removed slot refilled (56 B);
      feedback: exchange, carried exchange, moments, count and T per cell
        (104 B), plus 80 B of record traffic in evolved-T mode, plus 28 B per
        electron of remapped cells (w, p read, p written);
      the surrogate network's record kernel (evolved T): the cell record
        read (64 B), the five prefactors written (32 B, two 16-byte stores)
        and the source byte;
      the table's record kernel (evolved T): the cell record read (64 B) and
        the 192-float spectral record written (768 B)."""
    cells = tot["cell_steps"]
    products = tot["events_p"] + tot["events_c"] + tot["events_b"] + tot["events_pinv"]
    removed = tot["events_p"] + tot["absorbed_c"] + tot["absorbed_b"] + tot["events_pinv"]
    parts = tot["part_e"] + tot["part_g"] + tot["part_a"]
    return {
        "step": 28.0 * tot["part_e"] + 16.0 * tot["part_g"] + 16.0 * tot["part_a"],
        "decide_kernel": 16.0 * tot["part_a"] + 16.0 * tot["part_g"] + 48.0 * cells,
        "event_kernel": parts / 8.0 + 40.0 * cells + 56.0 * products + 56.0 * removed,
        "feedback_kernel": (104.0 + (80.0 if T_mode == 2 else 0.0)) * cells + 28.0 * tot["remap_e"],
        "sr_cells_kernel": 97.0 * cells,
        "sr_table_kernel": 832.0 * cells,
    }


class ClockSampler:
    """nvidia-smi clocks and throttle reasons while the timed region runs."""

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None
        self.t0 = self.t1 = None

    def start(self):
        q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.5)

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append((time.time(), parts))

    def mark(self, which):
        if which == "start":
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        inside = [p for t, p in self.samples if self.t0 is not None and self.t0 - 0.06 <= t <= self.t1 + 0.06]
        use = inside if inside else [p for _, p in self.samples]
        sm = [float(p[1]) for p in use if p[1].replace(".", "").isdigit()]
        smax = [float(p[2]) for p in use if p[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for p in use:
            for name, v in zip(names, p[5:9]):
                if v.strip().lower() in ("active", "1", "yes"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(use), "samples_in_window": len(inside)}


def run_reference(args):
    """The oracle as the reference arm, on the host cores: each step is one
    pass of os.cpu_count() spawned processes side by side, each stepping its
    own 64 cells of the same workload (FP64) for a bounded time (the step's
    time is the longest process's stepping time), so that the whole run
    stays near two minutes. Under torchrun rank 0 alone runs."""
    import multiprocessing as mp
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = c5_workload(args.c5_side) if args.workload == "c5" else (
        c3_workload() if args.workload == "c3" else workload())
    cores = os.cpu_count() or 1
    per_step = min(2.0, 100.0 / max(args.steps + args.warmup, 1))
    jobs = oracle_jobs(w, per_step)
    total_p, total_t, cell_steps = 0, 0.0, 0
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_worker, [(j[0], j[1], 0.0, j[3]) for j in jobs])  # initialise the cells
        for k in range(args.warmup + args.steps):
            res = pool.map(_oracle_worker, [(j[0], j[1], j[2], j[3] + k) for j in jobs])
            dt = max(r[1] for r in res)  # the processes step side by side
            if k >= args.warmup:
                total_p += sum(r[0] for r in res)
                cell_steps += sum(r[2] for r in res)
                total_t += dt
    value = total_p / total_t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (uniform thermal plasma, seeded)",
            "config": {"workload": w.name, "cells": w.ncells, "electrons_per_cell": w.n_el,
                       "photons_per_cell": w.n_ph, "axions_at_start": w.n_ax,
                       "parallelism": "oracle on %d host cores" % cores},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d cell-steps of the workload (%d particle-steps) over %d steps, %d "
                                       "processes of 64 cells" % (cell_steps, total_p, args.steps, cores)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_batched(args):
    """The batched-box workload: 4096 independent uniform boxes of uneven cell
    counts concatenated in one context (every cell carries its box's plasma),
    launch shape picked by the library's autotuner on the context's own state
    (restored afterwards), the timed steps replayed as a CUDA graph of one
    step. Device time of the timed steps with CUDA events."""
    import torch
    from paper_2604_24627_gb300 import AxionPlasma, workloads
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    w = workloads.config4(args.boxes, seed=0)
    w.params["w_a"] = float(np.float32(workloads.photon_weight(3.0, w.volume_cm3, w.n_ph)))
    w.params["seed"] = 0
    w.params["tally_enable"] = 0
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        pl = AxionPlasma(w.ncells, w.T_keV, w.n_ion, w.Z, w.A, w.volume_cm3, w.caps, w.params, device=dev,
                         stream=stream)
        pl.sample(w.n_el, w.n_ph, w.n_ax)
    torch.cuda.synchronize(dev)
    t0 = time.time()
    tuned_ms, chunk, warps = pl.autotune(0, 3, w.mask)
    tune_s = time.time() - t0
    pl.run_steps(0, args.warmup, w.mask)
    pl.tally()
    clocks = ClockSampler(0)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    clocks.mark("start")
    e0.record(stream)
    pl.run_steps(args.warmup, args.steps, w.mask)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clocks.mark("end")
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    _, tot = pl.tally()
    particles = tot["part_e"] + tot["part_g"] + tot["part_a"]
    step_bytes = 28.0 * tot["part_e"] + 16.0 * tot["part_g"] + 16.0 * tot["part_a"]
    # kernel split from a few plain step calls after the timed region
    nprof = 5
    pl.profile_begin(nprof)
    for k in range(nprof):
        pl.step(args.warmup + args.steps + k, w.mask)
    kms, nrec = pl.profile_end()
    pl.tally()
    peak, peak_kind = measured_peaks()
    gbs = step_bytes / (ms * 1e-3) / 1e9
    line = {"metric": METRIC, "value": particles / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (uniform thermal boxes, seeded)",
            "config": {"workload": w.name, "boxes": args.boxes, "cells": w.ncells,
                       "electrons_per_cell": w.n_el, "photons_per_cell": w.n_ph, "channels": "all, fwd+inv",
                       "T_mode": "evolved",
                       "launch": "CUDA graphs of 32 steps replayed, %d branch(es)" % pl.launch_shape()[2],
                       "autotuned": {"decide_chunk": chunk, "event_warps": warps, "trial_ms_per_step": tuned_ms,
                                     "seconds": tune_s},
                       "l2": "inputs larger than L2"},
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                         "traffic": None, "peak_kind": peak_kind,
                         "kernel": "step (%s), graph replay" % " + ".join(kms),
                         "basis": "28 B per electron, 16 B per photon and axion per step",
                         "kernels_ms_per_step": {k: v / max(nrec, 1) for k, v in kms.items()},
                 "launch": "CUDA graphs of 32 steps replayed, %d branch(es)" % pl.launch_shape()[2]},
            "gpu_launches": (len(kms) + 1) * pl.launch_shape()[2] * args.steps + 1, "clocks": clk}
    print(json.dumps(line))
    pl.close()


# ---------------------------------------------------------------- c5 and c3: three rate models
def c5_workload(side=256):
    """The 3-D plasma: side^3 hydrogen cells at T = 5 keV (evolved), n_e =
    6e25 cm^-3, 64 electrons, 32 Planck photons and 13 Maxwell-Boltzmann-
    equilibrium axions per cell (n_eq / n_gamma = 0.416 of the photons: a
    relaxed start, so that absorption, a->gamma and the remap run from the
    first timed step), axion weight = photon weight."""
    from paper_2604_24627_gb300 import workloads
    w = workloads.config5(side)
    w.n_ax = 13
    w.params["w_a"] = float(np.float32(workloads.photon_weight(5.0, w.volume_cm3, w.n_ph)))
    w.params.update(seed=0, tally_enable=0)
    return w


def c3_workload(n=512):
    from paper_2604_24627_gb300 import workloads
    w = workloads.config3(n)
    w.params["w_a"] = float(np.float32(workloads.photon_weight(3.0, w.volume_cm3, w.n_ph)))
    w.params.update(seed=0, tally_enable=0, T_mode=2, relax_r=0.1)
    return w


_ORACLE_STATES = {}


def _oracle_worker(job):
    """One host process of the multi-core oracle baseline: initialises its
    cells with the oracle's own sampler (once per process), then steps them
    (cycling, new step index each round) for `budget` seconds. Returns
    (particle-steps, seconds of stepping, cell-steps)."""
    wl, cells, budget, step0 = job
    from oracle import step as ostep
    from oracle.plasma import Params
    prm = Params(**wl["params"])
    key = tuple(cells)
    if key not in _ORACLE_STATES:
        _ORACLE_STATES[key] = [ostep.init_cell(prm, c, wl["T"][i], wl["ne"][i], wl["V"], wl["n_el"], wl["n_ph"],
                                               wl["n_ax"]) for i, c in enumerate(cells)]
    states = _ORACLE_STATES[key]
    done, k = 0, 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget:
        i = k % len(cells)
        parts = {sp: v.copy() for sp, v in states[i].items()}
        done += sum(len(v) for v in parts.values())
        ci = ostep.CellInput(wl["T"][i], np.array(wl["n_ion"][i]), np.array(wl["Z"]), np.array(wl["A"]))
        ostep.step_cell(ci, parts, prm, step0 + k // len(cells), cells[i], wl["mask"])
        k += 1
    return done, time.perf_counter() - t0, k


def oracle_jobs(w, seconds, cells_per_core=64, step0=7):
    """One job per host core: 64 random cells of the workload each, stepped
    for `seconds`."""
    from oracle.plasma import Params
    cores = os.cpu_count() or 1
    keys = set(Params.__dataclass_fields__)
    wl = {"params": {k: v for k, v in w.params.items() if k in keys}, "V": w.volume_cm3, "n_el": w.n_el,
          "n_ph": w.n_ph, "n_ax": w.n_ax, "Z": list(map(float, w.Z)), "A": list(map(float, w.A)), "mask": w.mask}
    rng = np.random.default_rng(1)
    jobs = []
    for r in range(cores):
        cells = [int(c) for c in rng.choice(w.ncells, cells_per_core, replace=False)]
        d = dict(wl, T=[float(w.T_keV[c]) for c in cells], ne=[float(np.sum(w.Z * w.n_ion[c])) for c in cells],
                 n_ion=[list(map(float, w.n_ion[c])) for c in cells])
        jobs.append((d, cells, seconds, step0))
    return jobs


def cpu_baseline_multicore(w, seconds):
    """The oracle, as it stands, on every host core: os.cpu_count() spawned
    processes (one per core), each stepping its own 64 cells of the workload
    for `seconds` after initialising them. Returns (particle-steps/s, cores,
    particle-steps, cell-steps, seconds)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    jobs = oracle_jobs(w, seconds)
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_worker, [(j[0], j[1], 0.0, j[3]) for j in jobs])  # initialise the cells
        res = pool.map(_oracle_worker, jobs)
    parts = sum(r[0] for r in res)
    t = max(r[1] for r in res)
    return parts / t, cores, parts, sum(r[2] for r in res), t


def rate_errors(pl, model, w, cells):
    """Per sampled cell, the largest relative error (in ln) of the rates the
    step uses against the library's FP64 targets (axpic_surrogate_targets,
    pinned to the oracle by the tests): cells whose rates come from a
    spectral record (table model; surrogate model where the network is not
    trusted) at the record's 30 points in [0.05, 20]; the others (closed
    forms; surrogate where trusted) from axpic_eval_rates at 12 energies:
    Gamma(gamma->a) dt, Gamma_abs,C dt and Gamma_abs,B dt. Returns
    (errors [cells, 3 channels], source per cell)."""
    from paper_2604_24627_gb300 import _lib
    hc3 = 1.973269804e-8 ** 3
    prm = w.params
    ln_gP = math.log(prm["g_agg_GeV_inv"] ** 2 * prm["dt_phys_s"] * math.pi ** 2 * hc3 / 1.602176634e-9)
    ln_gA = math.log(prm["g_ae"] ** 2 * prm["dt_phys_s"] * 2 * math.pi ** 2 * hc3 / 1.602176634e-9)
    h = math.log(400.0) / 29.0
    xk = 0.05 * np.exp(h * (np.arange(1, 31) - 1.0))
    xs = np.exp(np.linspace(math.log(0.06), math.log(19.0), 12))
    errs, srcs = [], []
    for c in cells:
        c = int(c)
        rec, src = _lib.axpic_get_cell_records(pl.ctx, c, 1)
        rec, src = rec[0], int(src[0]) if model else 0
        T = float(rec[0])
        kT = 2.0 / math.sqrt(float(rec[2])) / T
        ne = float(rec[9]) * 1e24
        if src:
            x = xk
            y = _lib.axpic_surrogate_targets(np.stack([x, np.full(30, kT), np.full(30, ne), np.ones(30)], 1))
            r = _lib.axpic_get_spectral_records(pl.ctx, c, 1)[0]
            e = [np.max(np.abs(r[32 * ch + 1:32 * ch + 31] - x - y[:, 32 * ch])) for ch in range(3)]
        else:
            x = xs
            y = _lib.axpic_surrogate_targets(np.stack([x, np.full(12, kT), np.full(12, ne), np.ones(12)], 1))
            got = pl.eval_rates(c, x * T)
            lx = np.log(x)
            g_exact = np.exp(y[:, 0] + ln_gP - 4 * math.log(T) - 3 * lx) * np.expm1(x)
            tc_exact = np.exp(y[:, 32] + ln_gA - 4 * math.log(T) - 3 * lx) * np.exp(x)
            tb_exact = np.exp(y[:, 64] + ln_gA - 4 * math.log(T) - 3 * lx) * np.exp(x)
            g_gpu = -np.log1p(-got[:, 0])
            e = [np.max(np.abs(np.log(g_gpu / g_exact))), np.max(np.abs(np.log(got[:, 2] / tc_exact))),
                 np.max(np.abs(np.log(got[:, 3] / tb_exact)))]
        errs.append(e)
        srcs.append(src)
    return np.array(errs), np.array(srcs)


def e2e_leg(pl, w, args, ncells, step0, stream, dev, world=1):
    """End to end through the public API with host buffers, on cells
    [0, ncells) of the plasma: every step copies their whole state (every
    slab at capacity, counts, T) host -> device, runs the step over them and
    copies it back. The cells are split into ranges (whole event CTAs of 128
    cells); each range's copy in, step (axpic_step_cells) and copy out are
    chained by events on three streams, so one range's copies overlap
    another's step and the two copy directions overlap each other. A range's
    next copy in waits for its previous copy out: the host buffers hold the
    state."""
    import torch
    import torch.distributed as dist
    caps = {name: slab.capacity for name, slab in pl.slabs.items()}
    # the slabs' contiguous arrays: the slot records, 4 values a slot
    fields = [(name, f) for name, slab in pl.slabs.items() for f in slab.storage]
    width = {"wp": 4, "xyz": 4}
    host = {(name, f): torch.empty(ncells * caps[name] * width[f], dtype=torch.float32, pin_memory=True)
            for name, f in fields}
    host_cnt = {name: torch.empty(ncells, dtype=torch.int32, pin_memory=True) for name in pl.slabs}
    host_T = torch.empty(ncells, dtype=torch.float64, pin_memory=True)
    for (name, f), hb in host.items():
        hb.copy_(pl.slabs[name].storage[f][:ncells * caps[name] * width[f]])
    for name, hb in host_cnt.items():
        hb.copy_(pl.slabs[name].count[:ncells])
    host_T.copy_(pl.T[:ncells])
    nbytes = sum(hb.numel() * hb.element_size() for hb in list(host.values()) + list(host_cnt.values()))
    nbytes += host_T.numel() * host_T.element_size()
    part = ((ncells + args.e2e_ranges - 1) // args.e2e_ranges + 127) // 128 * 128 if args.e2e_ranges > 1 else ncells
    ranges = [(c0, min(part, ncells - c0)) for c0 in range(0, ncells, part)]

    def pairs(c0, nc):
        out = []
        for name, f in fields:
            cap = caps[name] * width[f]
            out.append((host[(name, f)][c0 * cap:(c0 + nc) * cap], pl.slabs[name].storage[f][c0 * cap:(c0 + nc) * cap]))
        for name in caps:
            out.append((host_cnt[name][c0:c0 + nc], pl.slabs[name].count[c0:c0 + nc]))
        out.append((host_T[c0:c0 + nc], pl.T[c0:c0 + nc]))
        return out

    rpairs = [pairs(c0, nc) for c0, nc in ranges]
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    pl.tally()
    out_done = [None] * len(ranges)
    e0.record(stream)
    s_in.wait_event(e0)
    for k in range(args.e2e_steps):
        for r, (c0, nc) in enumerate(ranges):
            if out_done[r] is not None:
                s_in.wait_event(out_done[r])
            with torch.cuda.stream(s_in):
                for hb, t in rpairs[r]:
                    t.copy_(hb, non_blocking=True)
            ev_in = torch.cuda.Event()
            ev_in.record(s_in)
            stream.wait_event(ev_in)
            pl.step_cells(step0 + k, c0, nc, w.mask)
            ev_c = torch.cuda.Event()
            ev_c.record(stream)
            s_out.wait_event(ev_c)
            with torch.cuda.stream(s_out):
                for hb, t in rpairs[r]:
                    hb.copy_(t, non_blocking=True)
            out_done[r] = torch.cuda.Event()
            out_done[r].record(s_out)
    for ev in out_done:
        stream.wait_event(ev)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    _, tot_e = pl.tally()
    p_e = tot_e["part_e"] + tot_e["part_g"] + tot_e["part_a"]
    e_ms = e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([e_ms, p_e], dtype=torch.float64, device=dev)
        mx = t.clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        e_ms, p_e = float(mx[0]), float(t[1])
    del host, host_cnt, host_T, rpairs
    return {"value": p_e / (e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
            "steps": args.e2e_steps, "cell_ranges": len(ranges), "cells": ncells,
            "overlap": "copies of one cell range overlap the step of another (axpic_step_cells)"}


def run_three_models(args):
    """The 256^3 plasma (default) or the 512^2 temperature bump under the
    three rate models, one context at a time on the same seeded plasma:
    closed forms, the exact FP32 table, the surrogate network (trained and
    validated on the GPU first; trusted where the four nodes of a 369 x 241
    validation grid, log-spaced in T and n_e, around a cell and their
    neighbours are within TRUST_TOL on the rates and 1e-3 on the sampled
    quantiles). Each model: W
    warm-up steps through
    axpic_run_steps (which captures the CUDA graphs), then K timed steps
    replayed from the graphs, CUDA events on the context's stream, a barrier
    and a synchronize on both sides, the max over ranks. The surrogate
    model's steps are the reported value."""
    import torch
    import torch.distributed as dist
    from paper_2604_24627_gb300 import AxionPlasma, _lib
    from paper_2604_24627_gb300.mlp import SurrogateNet
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = c5_workload(args.c5_side) if args.workload == "c5" else c3_workload(args.nx if args.nx != 256 else 512)
    stream = torch.cuda.Stream(dev)
    t0 = time.time()
    net = SurrogateNet(stream=stream)
    fit_loss = _lib.axpic_surrogate_fit(net.h, 65536, 1, 40000, 8192, 2e-3, 7)
    fit_s = time.time() - t0
    nT, nne = 369, 241
    t0 = time.time()
    verr = _lib.axpic_surrogate_validate(net.h, nT, nne)
    val_s = time.time() - t0
    network = {"fit_seconds": fit_s, "fit_loss": fit_loss, "params": 10720, "validation_grid": [nT, nne, 2],
               "validation_seconds": val_s,
               "validated_rate_err_median": float(np.median(verr[..., 0])),
               "validated_rate_err_max": float(verr[..., 0].max()),
               "validated_sampled_quantile_err_max": float(verr[..., 1].max()),
               "validated_primakoff_quantile_err_median": float(np.median(verr[..., 2])),
               "trust_tolerance_rate": TRUST_TOL, "trust_tolerance_quantile": 1e-3,
               "trusted_node_fraction": float(np.mean((verr[..., 0] <= TRUST_TOL) & (verr[..., 1] <= 1e-3)))}
    sample = np.random.default_rng(0).choice(w.ncells, min(args.rate_err_cells, w.ncells), replace=False)
    lines, headline = {}, None
    for model in (0, 1, 2):
        prm = dict(w.params, rate_model=model)
        if args.branches:
            prm["step_branches"] = args.branches
        with torch.cuda.stream(stream):
            pl = AxionPlasma(w.ncells, w.T_keV, w.n_ion, w.Z, w.A, w.volume_cm3, w.caps, prm, device=dev,
                             cell_index_base=rank * w.ncells, stream=stream)
            pl.sample(w.n_el, w.n_ph, w.n_ax)
        if model == 2:
            _lib.axpic_set_surrogate(pl.ctx, net.h, verr, nT, nne, TRUST_TOL, 1e-3)
        pl.run_steps(0, args.warmup, w.mask)  # captures the graphs
        pl.tally()
        clocks = ClockSampler(local) if model == 2 else None
        if clocks:
            clocks.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        if clocks:
            clocks.mark("start")
        e0.record(stream)
        pl.run_steps(args.warmup, args.steps, w.mask)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if clocks:
            clocks.mark("end")
        if world > 1:
            dist.barrier()
        clk = clocks.stop() if clocks else None
        ms = e0.elapsed_time(e1)
        _, tot = pl.tally()
        parts = tot["part_e"] + tot["part_g"] + tot["part_a"]
        step_bytes = kernel_bytes(tot, w.params.get("T_mode", 0))["step"]
        if world > 1:
            t = torch.tensor([ms, parts, step_bytes], dtype=torch.float64, device=dev)
            mx = t.clone()
            dist.all_reduce(mx, op=dist.ReduceOp.MAX)
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
            ms, parts, step_bytes = float(mx[0]), float(t[1]), float(t[2])
        # the kernel split: events around each kernel of 3 further steps
        nk = 3
        pl.profile_begin(nk)
        for k in range(nk):
            pl.step(args.warmup + args.steps + k, w.mask)
        kms, nrec = pl.profile_end()
        _, tot_k = pl.tally()
        entry = {"particle_steps_per_s": parts / (ms * 1e-3), "ms_per_step": ms / args.steps,
                 "kernels_ms_per_step": {k: v / max(nrec, 1) for k, v in kms.items()},
                 "launch": "CUDA graphs of 32 and 1 steps replayed, %d branch(es)" % pl.launch_shape()[2],
                 "counts": {"particle_steps": parts, "events_primakoff": tot["events_p"],
                            "events_compton": tot["events_c"], "events_brems": tot["events_b"],
                            "events_inverse": tot["events_pinv"], "absorbed": tot["absorbed_c"] + tot["absorbed_b"],
                            "remapped_cells": tot["remaps"], "dropped": tot["dropped"]}}
        if rank == 0:
            errs, srcs = rate_errors(pl, model, w, sample)
            entry["rate_err"] = {"cells": len(sample), "max": float(errs.max()), "median": float(np.median(errs)),
                                 "max_per_channel": [float(v) for v in errs.max(0)],
                                 "cells_above_1e-3": float(np.mean(errs.max(1) > 1e-3))}
            if model == 2:
                entry["rate_err"]["cells_on_network"] = float(np.mean(srcs == 0))
        if model == 2:
            headline = dict(entry, ms=ms, tot_k=tot_k, kms=kms, nrec=nrec, clk=clk, step_bytes=step_bytes,
                            branches=pl.launch_shape()[2])
            if args.e2e_steps > 0:
                n_e2e = args.e2e_cells or max(128, (w.ncells // 16) // 128 * 128)
                headline["e2e"] = e2e_leg(pl, w, args, min(n_e2e, w.ncells), args.warmup + args.steps + nk, stream,
                                          dev, world)
        lines[("closed_forms", "table", "surrogate")[model]] = entry
        pl.close()
        del pl
        torch.cuda.empty_cache()
    net.close()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    peak, peak_kind = measured_peaks()
    h = headline
    kb = kernel_bytes(h["tot_k"], w.params.get("T_mode", 0))
    per_kernel = {k: {"ms_per_launch": h["kms"][k] / max(h["nrec"], 1),
                      "algorithmic_bytes_per_launch": kb[k] / max(h["nrec"], 1),
                      "GBps": kb[k] / (h["kms"][k] * 1e-3) / 1e9 if h["kms"][k] > 0 else None,
                      "share": h["kms"][k] / sum(h["kms"].values())} for k in h["kms"]}
    dom = max(h["kms"], key=h["kms"].get)
    step_gbs = h["step_bytes"] / (h["ms"] * 1e-3) / 1e9
    traffic = None
    prof = os.path.join(ROOT, "profiles", "step_kernels_%s_traffic.json" % args.workload)
    if os.path.exists(prof):
        try:
            with open(prof) as f:
                pj = json.load(f)
            if pj.get("kernel_hash") == kernel_hash():
                traffic = pj["dram_bytes_per_launch"].get(dom)
        except Exception:
            traffic = None
    line = {"metric": METRIC, "value": lines["surrogate"]["particle_steps_per_s"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": lines["surrogate"]["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (uniform thermal plasma, seeded Philox sampler)",
            "config": {"workload": w.name, "cells": w.ncells, "electrons_per_cell": w.n_el,
                       "photons_per_cell": w.n_ph, "axions_at_start": w.n_ax, "channels": "all, fwd+inv",
                       "T_mode": "evolved", "rate_model": "surrogate network, exact table where not trusted",
                       "l2": "inputs larger than L2 (%.1f GB per step at the fused-pass minimum)"
                       % (h["step_bytes"] / args.steps / 1e9 / world),
                       "parallelism": "one full plasma per GPU" if world > 1 else "single GPU",
                       "launch": "CUDA graphs of 32 and 1 steps replayed, %d branch(es)" % h["branches"]},
            # the dominant kernel against its own minimum bytes; the whole
            # step against the fused-pass minimum (28 B per electron, 16 B
            # per photon and axion) beside it
            "roofline": {"bound": "hbm", "kernel": "axpic::" + dom,
                         "achieved": per_kernel[dom]["GBps"], "peak": peak, "unit": "GB/s",
                         "frac": per_kernel[dom]["GBps"] / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "algorithmic_bytes_per_launch": per_kernel[dom]["algorithmic_bytes_per_launch"],
                         "kernels": per_kernel,
                         "step": {"achieved": step_gbs, "frac": step_gbs / peak,
                                  "basis": "28 B per electron, 16 B per photon and axion per step",
                                  "algorithmic_bytes_per_step": h["step_bytes"] / args.steps / world}},
            "rate_models": lines,
            "surrogate_vs_table": lines["surrogate"]["particle_steps_per_s"] / lines["table"]["particle_steps_per_s"],
            "network": network,
            # the profiled kernels of a step, plus the heavy-cell event kernel
            # of each branch, per timed step; plus the step-counter kernel
            "gpu_launches": (len(h["kms"]) + 1) * h["branches"] * args.steps + 1, "clocks": h["clk"]}
    if "e2e" in h:
        line["e2e"] = h["e2e"]
        line["e2e"]["sample"] = "cells [0, %d) of the plasma, the surrogate model" % h["e2e"]["cells"]
    if world == 1 and not args.no_cpu_baseline:
        v, cores, npart, ncs, t = cpu_baseline_multicore(w, max(0.5, args.cpu_seconds / (os.cpu_count() or 1)))
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": "%d processes each stepping 64 random cells of the workload for %.1f s "
                                          "(%d cell-steps, %d particle-steps)" % (cores, t, ncs, npart)}
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload in ("c3", "c5"):
        run_three_models(args)
        return
    if args.workload == "c4":
        run_batched(args)
        return
    import torch
    import torch.distributed as dist
    from paper_2604_24627_gb300 import AxionPlasma, _lib

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workload(args.nx)
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        pl = AxionPlasma(w.ncells, w.T_keV, w.n_ion, w.Z, w.A, w.volume_cm3, w.caps, w.params, device=dev,
                         cell_index_base=rank * w.ncells, stream=stream)
        pl.sample(w.n_el, w.n_ph, w.n_ax)
    torch.cuda.synchronize(dev)

    for s in range(args.warmup):
        pl.step(s, w.mask)
    pl.tally()  # clears counters: the timed region starts from zero
    clocks = ClockSampler(local)
    clocks.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.mark("start")
    # the timed steps: one CUDA graph of a step, replayed (axpic_run_steps)
    t_start.record(stream)
    pl.run_steps(args.warmup, args.steps, w.mask)
    t_end.record(stream)
    torch.cuda.synchronize(dev)
    clocks.mark("end")
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    elapsed_ms = t_start.elapsed_time(t_end)
    H, tot = pl.tally()
    # the kernel split: events around each kernel of a few further steps
    nk = min(20, args.steps)
    pl.profile_begin(nk)
    for k in range(nk):
        pl.step(args.warmup + args.steps + k, w.mask)
    kms, nprof = pl.profile_end()
    _, tot_k = pl.tally()
    particles = tot["part_e"] + tot["part_g"] + tot["part_a"]
    kbytes = kernel_bytes(tot_k, w.params.get("T_mode", 0))
    if world > 1:
        t = torch.tensor([elapsed_ms, particles], dtype=torch.float64, device=dev)
        mx = t.clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        elapsed_ms, particles = float(mx[0]), float(t[1])

    # end to end through the public API with host buffers, the whole plasma
    e2e = None
    if args.e2e_steps > 0:
        e2e = e2e_leg(pl, w, args, w.ncells, args.warmup + args.steps + nk, stream, dev, world)

    # axion free streaming and cell migration (axpic_stream_axions) on the
    # same plasma after the legs above: the workload's grid as a periodic box
    # of cubic cells (edge from the cell volume), c dt = 0.6 of the edge. The
    # algorithmic bytes of a call: every axion's seven fields read and
    # written once (56 B).
    stream_leg = None
    if args.stream_calls > 0 and len(w.shape) >= 1:
        dims = tuple(list(w.shape) + [1] * (3 - len(w.shape)))
        if int(np.prod(dims)) == w.ncells:
            h = w.volume_cm3 ** (1.0 / 3.0)
            dt_s = 0.6 * h / 2.99792458e10
            pl.stream_axions(dims, h, dt_s, True)  # the first call makes the scratch
            torch.cuda.synchronize(dev)
            n_ax = int(pl.slabs["axions"].count[:w.ncells].sum())
            s0 = torch.cuda.Event(enable_timing=True)
            s1 = torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            for _ in range(args.stream_calls):
                pl.stream_axions(dims, h, dt_s, True)
            s1.record(stream)
            torch.cuda.synchronize(dev)
            ms = s0.elapsed_time(s1) / args.stream_calls
            gbps = 56.0 * n_ax / (ms * 1e-3) / 1e9
            stream_leg = {"call": "axpic_stream_axions", "grid": list(dims), "boundary": "periodic",
                          "c_dt_over_h": 0.6, "axions": n_ax, "calls": args.stream_calls, "ms_per_call": ms,
                          "axion_moves_per_s": n_ax / (ms * 1e-3), "algorithmic_bytes_per_axion": 56,
                          "GBps": gbps}

    # axion merging (axpic_merge_axions) on the same plasma after the other
    # legs: every cell above 64 axions, 16 |p| thresholds from 0.5 to 50 keV.
    # Each timed call merges the same state: the axion slab is restored by a
    # device copy on the context's stream before it, outside the events, so
    # the events hold the kernel alone. Algorithmic bytes: the seven fields of
    # every axion in a merged cell read and written once (56 B).
    merge_leg = None
    if args.merge_n_target > 0:
        edges = (np.geomspace(0.5, 50.0, 16) / 510.99895).astype(np.float32) ** 2
        pl.merge_axions(1 << 30, edges)  # the first call makes the scratch; nothing is merged
        torch.cuda.synchronize(dev)
        slab = pl.slabs["axions"]
        cnt = slab.count[:w.ncells]
        n_before = int(cnt.sum())
        n_in_merged = int(cnt[cnt > args.merge_n_target].sum())
        saved = {f: t.clone() for f, t in slab.storage.items()}
        saved_count = slab.count.clone()
        times = []
        for _ in range(args.merge_calls):
            with torch.cuda.stream(stream):
                for f, t in slab.storage.items():
                    t.copy_(saved[f])
                slab.count.copy_(saved_count)
            m0 = torch.cuda.Event(enable_timing=True)
            m1 = torch.cuda.Event(enable_timing=True)
            m0.record(stream)
            pl.merge_axions(args.merge_n_target, edges)
            m1.record(stream)
            torch.cuda.synchronize(dev)
            times.append(m0.elapsed_time(m1))
        ms = float(np.mean(times))
        n_after = int(slab.count[:w.ncells].sum())
        del saved, saved_count
        merge_leg = {"call": "axpic_merge_axions", "n_target": args.merge_n_target, "p_bins": 17, "octants": 8,
                     "axions_before": n_before, "axions_after": n_after, "axions_in_merged_cells": n_in_merged,
                     "calls": args.merge_calls, "ms_per_call": ms, "ms_min": float(np.min(times)),
                     "axions_per_s": n_in_merged / (ms * 1e-3),
                     "algorithmic_bytes_per_axion": 56, "GBps": 56.0 * n_in_merged / (ms * 1e-3) / 1e9}

    # composition from the deposited electron density
    # (axpic_deposit_composition) into a scratch array, 10 calls. Before each
    # call a 256 MB device copy on the context's stream flushes L2 and keeps
    # the device busy while the host enqueues the call, so the events hold
    # the kernel alone. Algorithmic bytes: each electron's weight read (4 B)
    # and each cell's count and ion densities (4 + 8 nspecies B).
    comp_leg = None
    if args.deposit_calls > 0:
        XH = 0.9 * 1.00794 / (0.9 * 1.00794 + 0.1 * 4.002602)
        out = torch.empty(w.ncells * len(w.Z), dtype=torch.float64, device=dev)
        pl.deposit_composition([XH, 1 - XH], -1, out)
        torch.cuda.synchronize(dev)
        n_el = int(pl.slabs["electrons"].count[:w.ncells].sum())
        flush_src = torch.zeros(256 << 20, dtype=torch.uint8, device=dev)
        flush_dst = torch.empty_like(flush_src)
        times = []
        for _ in range(args.deposit_calls):
            with torch.cuda.stream(stream):
                flush_dst.copy_(flush_src)
            c0 = torch.cuda.Event(enable_timing=True)
            c1 = torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            pl.deposit_composition([XH, 1 - XH], -1, out)
            c1.record(stream)
            torch.cuda.synchronize(dev)
            times.append(c0.elapsed_time(c1))
        ms = float(np.mean(times))
        nbytes = 4.0 * n_el + (4.0 + 8.0 * len(w.Z)) * w.ncells
        comp_leg = {"call": "axpic_deposit_composition", "mode": "mass fractions (X_H)", "electrons": n_el,
                    "calls": args.deposit_calls, "l2": "flushed before each call", "ms_per_call": ms,
                    "ms_min": float(np.min(times)), "algorithmic_bytes": nbytes,
                    "GBps": nbytes / (ms * 1e-3) / 1e9}
        del out, flush_src, flush_dst

    if rank == 0:
        peak, peak_kind = measured_peaks()
        if comp_leg:
            comp_leg["frac"] = comp_leg["GBps"] / peak
        if merge_leg:
            merge_leg["frac"] = merge_leg["GBps"] / peak
        if stream_leg:
            stream_leg["frac"] = stream_leg["GBps"] / peak
            stream_leg["peak_kind"] = peak_kind
        # per kernel: device time from events around each launch, and the
        # minimum bytes that kernel has to move (kernel_bytes)
        dom = max(kms, key=kms.get)
        per_kernel = {k: {"ms_per_launch": kms[k] / max(nprof, 1),
                          "algorithmic_bytes_per_launch": kbytes[k] / max(nprof, 1),
                          "GBps": kbytes[k] / (kms[k] * 1e-3) / 1e9 if kms[k] > 0 else None,
                          "share": kms[k] / sum(kms.values())} for k in kms}
        # DRAM bytes per launch from one ncu capture of the same kernels
        # (profiles/), valid only while the kernel sources are unchanged
        traffic = None
        prof = os.path.join(ROOT, "profiles", "step_kernels_c2_traffic.json")
        if os.path.exists(prof):
            try:
                with open(prof) as f:
                    pj = json.load(f)
                if pj.get("kernel_hash") == kernel_hash():
                    traffic = sum(pj["dram_bytes_per_launch"][k] for k in kms)
            except Exception:
                traffic = None
        value = particles / (elapsed_ms * 1e-3)
        # the whole step against the fused-pass minimum (28 B per electron,
        # 16 B per photon and axion) over the timed steps' device time
        step_gbs = kernel_bytes(tot, w.params.get("T_mode", 0))["step"] / (elapsed_ms * 1e-3) / 1e9
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic (uniform thermal plasma, seeded Philox sampler)",
                "config": {"workload": w.name, "cells": w.ncells, "electrons_per_cell": w.n_el,
                           "photons_per_cell": w.n_ph, "axions_at_start": w.n_ax, "channels": "all, fwd+inv",
                           "T_mode": "evolved", "l2": "inputs larger than L2 (%.2f GB per step at the fused-pass minimum)"
                           % (kernel_bytes(tot, w.params.get("T_mode", 0))["step"] / args.steps / 1e9),
                           "parallelism": "cells sharded per GPU" if world > 1 else "single GPU",
                           "launch": "CUDA graphs of 32 steps replayed, %d branches of cells on forked streams"
                           % pl.launch_shape()[2]},
                # the step's kernels as one pass of the hot path, against the
                # fused-pass minimum of 28 B per electron, 16 B per photon and
                # axion; the kernel with the largest device time is named
                "roofline": {"bound": "hbm", "achieved": step_gbs, "peak": peak, "unit": "GB/s",
                             "frac": step_gbs / peak if step_gbs else None, "traffic": traffic,
                             "peak_kind": peak_kind, "kernel": "step (%s)" % " + ".join(kms),
                             "basis": "28 B per electron, 16 B per photon and axion per step",
                             "algorithmic_bytes_per_launch": kernel_bytes(tot, w.params.get("T_mode", 0))["step"]
                             / args.steps,
                             "dominant_kernel": "axpic::" + dom, "kernels": per_kernel},
                "gpu_launches": (len(kms) + 1) * pl.launch_shape()[2] * args.steps + 1, "clocks": clk,
                "counts": {"particle_steps": particles, "events_primakoff": tot["events_p"],
                           "events_compton": tot["events_c"], "events_brems": tot["events_b"],
                           "events_inverse": tot["events_pinv"], "remapped_cells": tot["remaps"]}}
        if e2e:
            line["e2e"] = e2e
        if stream_leg:
            line["axion_streaming"] = stream_leg
        if merge_leg:
            line["axion_merging"] = merge_leg
        if comp_leg:
            line["composition_deposit"] = comp_leg
        if world == 1 and not args.no_cpu_baseline:
            v, cores, npart, ncs, t = cpu_baseline_multicore(w, max(0.5, args.cpu_seconds / (os.cpu_count() or 1)))
            line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                    "sample": "%d processes each stepping 64 random cells of the workload for %.1f s "
                                              "(%d cell-steps, %d particle-steps)" % (cores, t, ncs, npart)}
        print(json.dumps(line))
    pl.close()
    if world > 1:
        dist.destroy_process_group()


def kernel_hash():
    import hashlib
    h = hashlib.sha256()
    for name in ("step.cu", "common.cuh", "tables.h", "sr.h", "srnet.cuh"):
        with open(os.path.join(ROOT, "paper_2604_24627_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    main()
