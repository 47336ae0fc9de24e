"""Throughput of the axion Monte-Carlo step on GB300.

One "step" is one fused pass of the whole hot path (absorb -> emit ->
feedback -> temperature update) over every cell of the workload. The default
workload is the 2-D 256x256 all-channel relaxation: T_e = 3 keV, 90 % H +
10 % He by number at n_e = 6e25 cm^-3, 512 Maxwellian electrons and 256
Planck photons per cell, axion-free start, forward and inverse operators of
all three channels, binary32 rates with FP64 exchange buffers and temperature.

Metric: particle-steps/s = sum over timed steps of the particles (electrons +
photons + axions) present at the start of the step / device time. Under
torchrun every rank runs its own full-size shard (weak scaling, no data-path
collective) and rank 0 reports the aggregate.

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
# The network is trusted where the four validation nodes around a cell are
# within half the 1e-3 rate bound: errors between nodes stay within it.
TRUST_TOL = 5e-4
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
    ap.add_argument("--workload", default="c2", choices=["c2", "c3", "c4"],
                    help="c2: the 256x256 relaxation (the reported line); c3: 512x512 temperature bump, surrogate "
                         "vs table vs closed-form rates; c4: 4096 uneven boxes in one context, autotuned launch "
                         "shape, steps replayed as a CUDA graph")
    ap.add_argument("--boxes", type=int, default=4096, help="boxes of the c4 workload")
    ap.add_argument("--branches", type=int, default=0,
                    help="c3: cell branches of a replayed step (1, 2, 4 or 8; 0: the library's choice)")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 1000 if args.workload == "c2" else 100
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
        electron of remapped cells (w, p read, p written)."""
    cells = tot["cell_steps"]
    products = tot["events_p"] + tot["events_c"] + tot["events_b"] + tot["events_pinv"]
    removed = tot["events_p"] + tot["absorbed_c"] + tot["absorbed_b"] + tot["events_pinv"]
    parts = tot["part_e"] + tot["part_g"] + tot["part_a"]
    return {
        "step": 28.0 * tot["part_e"] + 16.0 * tot["part_g"] + 16.0 * tot["part_a"],
        "decide_kernel": 16.0 * tot["part_a"] + 16.0 * tot["part_g"] + 48.0 * cells,
        "event_kernel": parts / 8.0 + 40.0 * cells + 56.0 * products + 56.0 * removed,
        "feedback_kernel": (104.0 + (80.0 if T_mode == 2 else 0.0)) * cells + 28.0 * tot["remap_e"],
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


def oracle_state(w, ncells_sample):
    """Initial state of the first cells of the workload from the oracle's own
    sampler (same Philox streams as the library's sampler)."""
    from oracle import step as ostep
    from oracle.plasma import Params
    prm = Params(**{k: v for k, v in w.params.items() if k in Params.__dataclass_fields__})
    return [ostep.init_cell(prm, c, float(w.T_keV[c]), float(np.sum(w.Z * w.n_ion[c])), w.volume_cm3,
                            w.n_el, w.n_ph, w.n_ax) for c in range(ncells_sample)]


def cpu_baseline(w, seconds, state_cells, step0=7):
    """Time the oracle, as it stands, on a bounded sample of the workload: the
    given cells (all of their particles) are stepped once each, cycling with
    new step indices, until `seconds` of CPU time have passed. Returns
    particle-steps/s, cell-steps, particle-steps and seconds."""
    from oracle import step as ostep
    from oracle.plasma import Params
    prm = Params(**{k: v for k, v in w.params.items() if k in Params.__dataclass_fields__})
    done = 0
    cell_steps = 0
    t_work = 0.0
    k = 0
    while t_work < seconds:
        c = k % len(state_cells)
        parts = {s: v.copy() for s, v in state_cells[c].items()}
        n = sum(len(v) for v in parts.values())
        ci = ostep.CellInput(float(w.T_keV[c]), w.n_ion[c], w.Z, w.A)
        t0 = time.perf_counter()
        ostep.step_cell(ci, parts, prm, step0 + k // len(state_cells), c, w.mask)
        t_work += time.perf_counter() - t0
        done += n
        cell_steps += 1
        k += 1
    return done / t_work, cell_steps, done, t_work


def run_reference(args):
    """The oracle as the reference arm: each step = one oracle step over a
    bounded sample of cells of the same workload (FP64, host cores)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = workload()
    state = oracle_state(w, 16)
    # each step is a bounded sample: the whole run stays near two minutes
    per_step = min(0.5, 120.0 / max(args.steps + args.warmup, 1))
    for _ in range(args.warmup):
        cpu_baseline(w, 0.2, state)
    vals = []
    total_p = 0
    total_t = 0.0
    cells_total = 0
    for _ in range(args.steps):
        v, cells, parts, t = cpu_baseline(w, per_step, state)
        total_p += parts
        total_t += t
        cells_total += cells
        vals.append(v)
    value = total_p / total_t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (uniform thermal plasma, seeded)",
            "config": {"workload": w.name, "cells": w.ncells, "electrons_per_cell": w.n_el,
                       "photons_per_cell": w.n_ph, "parallelism": "oracle on host cores"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "%d cell-steps of the workload (%d particle-steps) over %d steps"
                                       % (cells_total, total_p, args.steps)},
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
            "gpu_launches": len(kms) * pl.launch_shape()[2] * args.steps + 1, "clocks": clk}
    print(json.dumps(line))
    pl.close()


def run_rate_models(args):
    """The temperature-bump workload (512x512 hydrogen cells, T = 1 + 4
    exp(-r^2 / 2 64^2) keV, 256 electrons + 128 photons per cell) under the
    three rate models: closed forms, the exact FP32 table and the surrogate
    network (trained first by the library's own GPU kernels on its FP64
    targets; table where its validated error exceeds 1e-3). T evolves, so the
    spectral records are rebuilt every step. Reports particle-steps/s per
    model and each model's rate error against the exact targets on sampled
    cells."""
    import torch
    from paper_2604_24627_gb300 import AxionPlasma, _lib, workloads
    from paper_2604_24627_gb300.mlp import SurrogateNet
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    n = args.nx if args.nx != 256 else 512
    w = workloads.config3(n)
    w.params["w_a"] = float(np.float32(workloads.photon_weight(3.0, w.volume_cm3, w.n_ph)))
    w.params.update(seed=0, tally_enable=0, T_mode=2, relax_r=0.1)
    stream = torch.cuda.Stream(dev)
    # the network: trained and validated on the GPU
    t0 = time.time()
    net = SurrogateNet(stream=stream)
    fit_loss = _lib.axpic_surrogate_fit(net.h, 65536, 1, 40000, 8192, 2e-3, 7)
    fit_s = time.time() - t0
    nT, nne = 24, 16
    eL, eQ = _lib.axpic_surrogate_validate(net.h, nT, nne)
    err_map = np.stack([eL, eQ], axis=-1).astype(np.float32).reshape(-1)
    sample = np.random.default_rng(0).choice(w.ncells, 256, replace=False)
    out = {"surrogate": {"fit_seconds": fit_s, "fit_loss": fit_loss, "params": 10720,
                         "validated_rate_err_median": float(np.median(eL)), "validated_rate_err_max": float(eL.max()),
                         "validated_quantile_err_median": float(np.median(eQ)),
                         "trusted_fraction_at_1e-3": float(np.mean(eL <= 1e-3)),
                         "trust_tolerance": TRUST_TOL,
                         "trusted_fraction": float(np.mean(eL <= TRUST_TOL))}}
    lines = {}
    for model in (0, 1, 2):
        prm = dict(w.params, rate_model=model)
        if args.branches:
            prm["step_branches"] = args.branches
        with torch.cuda.stream(stream):
            pl = AxionPlasma(w.ncells, w.T_keV, w.n_ion, w.Z, w.A, w.volume_cm3, w.caps, prm, device=dev,
                             stream=stream)
            pl.sample(w.n_el, w.n_ph, w.n_ax)
        if model == 2:
            _lib.axpic_set_surrogate(pl.ctx, net.h, err_map, nT, nne, TRUST_TOL)
        for s in range(args.warmup):
            pl.step(s, w.mask)
        pl.tally()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        # the timed steps: CUDA graphs of 32 steps, replayed (axpic_run_steps)
        e0.record(stream)
        pl.run_steps(args.warmup, args.steps, w.mask)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        _, tot = pl.tally()
        parts = tot["part_e"] + tot["part_g"] + tot["part_a"]
        # the kernel split: events around each kernel of 10 further steps
        pl.profile_begin(10)
        for k in range(10):
            pl.step(args.warmup + args.steps + k, w.mask)
        kms, nrec = pl.profile_end()
        entry = {"particle_steps_per_s": parts / (ms * 1e-3), "ms_per_step": ms / args.steps,
                 "kernels_ms_per_step": {k: v / max(nrec, 1) for k, v in kms.items()},
                 "launch": "CUDA graphs of 32 steps replayed, %d branch(es)" % pl.launch_shape()[2]}
        if model:
            # records of sampled cells against the exact targets at the grid points
            recs = [_lib.axpic_get_spectral_records(pl.ctx, int(c), 1)[0] for c in sample]
            info = pl.cell_info()
            errs = []
            h = math.log(400.0) / 29.0
            xk = 0.05 * np.exp(h * (np.arange(1, 31) - 1.0))
            for r, c in zip(recs, sample):
                T = float(info[c, 12])
                kT = float(info[c, 5]) / T
                ne = float(info[c, 2])
                rows = np.stack([xk, np.full(30, kT), np.full(30, ne), np.ones(30)], 1)
                y = _lib.axpic_surrogate_targets(rows)
                errs.append([np.max(np.abs(r[32 * ch + 1:32 * ch + 31] - xk - y[:, 32 * ch])) for ch in range(3)])
            errs = np.array(errs)  # [cell][channel]: largest ln-rate error over the grid points
            entry["rate_err_max_sampled"] = float(errs.max())
            entry["rate_err_median_sampled"] = float(np.median(errs))
            entry["rate_err_median_per_channel"] = [float(v) for v in np.median(errs, 0)]
            entry["rate_err_max_per_channel"] = [float(v) for v in errs.max(0)]
            entry["sampled_cells_above_1e-3"] = float(np.mean(errs.max(1) > 1e-3))
        lines[("closed_forms", "table", "surrogate")[model]] = entry
        pl.close()
    net.close()
    # transport on: the closed-form model with the axions' free streaming
    # after every step (axpic_run_steps_streamed), the workload's grid as a
    # periodic box of cubic cells, c dt = 0.6 of the edge
    dims = tuple(list(w.shape) + [1] * (3 - len(w.shape)))
    if int(np.prod(dims)) == w.ncells:
        h = w.volume_cm3 ** (1.0 / 3.0)
        dt_s = 0.6 * h / 2.99792458e10
        with torch.cuda.stream(stream):
            pl = AxionPlasma(w.ncells, w.T_keV, w.n_ion, w.Z, w.A, w.volume_cm3, w.caps, dict(w.params, rate_model=0),
                             device=dev, stream=stream)
            pl.sample(w.n_el, w.n_ph, w.n_ax)
        for s in range(args.warmup):
            pl.step(s, w.mask)
            pl.stream_axions(dims, h, dt_s, True)
        pl.tally()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        pl.run_steps_streamed(args.warmup, args.steps, w.mask, dims, h, dt_s, True)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        _, tot = pl.tally()
        parts = tot["part_e"] + tot["part_g"] + tot["part_a"]
        lines["closed_forms_with_transport"] = {
            "particle_steps_per_s": parts / (ms * 1e-3), "ms_per_step": ms / args.steps,
            "launch": "CUDA graphs of 32 steps replayed, each step's %d branch(es) joined before the streaming"
                      % pl.launch_shape()[2],
            "transport": {"grid": list(dims), "boundary": "periodic", "c_dt_over_h": 0.6}}
        pl.close()
    line = {"metric": METRIC, "value": lines["surrogate"]["particle_steps_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": lines["surrogate"]["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (temperature bump, seeded)",
            "config": {"workload": w.name, "cells": w.ncells, "electrons_per_cell": w.n_el,
                       "photons_per_cell": w.n_ph, "T_mode": "evolved (records rebuilt every step)"},
            "rate_models": lines, "surrogate_vs_table": lines["surrogate"]["particle_steps_per_s"]
            / lines["table"]["particle_steps_per_s"], "network": out["surrogate"],
            "gpu_launches": None}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "c3":
        run_rate_models(args)
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

    # end to end through the public API with host buffers: every step copies
    # the whole plasma state host -> device, runs the step, copies it back.
    # The cells are split into ranges (whole event CTAs of 128 cells); each
    # range's copy in, step (axpic_step_cells) and copy out are chained by
    # events on three streams, so one range's copies overlap another's step
    # and the two copy directions overlap each other. A range's next copy in
    # waits for its previous copy out: the host buffers hold the state.
    e2e = None
    if args.e2e_steps > 0:
        caps = {name: slab.capacity for name, slab in pl.slabs.items()}
        fields = [(name, f) for name, slab in pl.slabs.items() for f in slab.data]
        host = {(name, f): torch.empty(pl.slabs[name].data[f].shape, dtype=torch.float32, pin_memory=True)
                for name, f in fields}
        host_cnt = {name: torch.empty(slab.count.shape, dtype=torch.int32, pin_memory=True)
                    for name, slab in pl.slabs.items()}
        host_T = torch.empty(pl.T.shape, dtype=torch.float64, pin_memory=True)
        for (name, f), h in host.items():
            h.copy_(pl.slabs[name].data[f])
        for name, h in host_cnt.items():
            h.copy_(pl.slabs[name].count)
        host_T.copy_(pl.T)
        nbytes = sum(h.numel() * h.element_size() for h in list(host.values()) + list(host_cnt.values()))
        nbytes += host_T.numel() * host_T.element_size()
        n = w.ncells
        part = ((n + args.e2e_ranges - 1) // args.e2e_ranges + 127) // 128 * 128 if args.e2e_ranges > 1 else n
        ranges = [(c0, min(part, n - c0)) for c0 in range(0, n, part)]

        def pairs(c0, nc):
            out = []
            for name, f in fields:
                cap = caps[name]
                out.append((host[(name, f)][c0 * cap:(c0 + nc) * cap],
                            pl.slabs[name].data[f][c0 * cap:(c0 + nc) * cap]))
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
                    for h, t in rpairs[r]:
                        t.copy_(h, non_blocking=True)
                ev_in = torch.cuda.Event()
                ev_in.record(s_in)
                stream.wait_event(ev_in)
                pl.step_cells(args.warmup + args.steps + nk + k, c0, nc, w.mask)
                ev_c = torch.cuda.Event()
                ev_c.record(stream)
                s_out.wait_event(ev_c)
                with torch.cuda.stream(s_out):
                    for h, t in rpairs[r]:
                        h.copy_(t, non_blocking=True)
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
        e2e = {"value": p_e / (e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "steps": args.e2e_steps, "cell_ranges": len(ranges),
               "overlap": "copies of one cell range overlap the step of another (axpic_step_cells)"}
        del host, host_cnt, host_T, rpairs

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
        saved = {f: t.clone() for f, t in slab.data.items()}
        saved_count = slab.count.clone()
        times = []
        for _ in range(args.merge_calls):
            with torch.cuda.stream(stream):
                for f, t in slab.data.items():
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
                "gpu_launches": len(kms) * pl.launch_shape()[2] * args.steps + 1, "clocks": clk,
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
            cells = [pl.cell(c) for c in range(64)]
            from oracle import step as ostep
            state = [{k: ostep.Species(*[np.asarray(d[k][f]) for f in ("w", "px", "py", "pz", "x", "y", "z")])
                      for k in "ega"} for d in cells]
            v, ncell, npart, t = cpu_baseline(w, args.cpu_seconds, state_cells=state)
            line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": "%d cells of the workload stepped once (%d particle-steps, %.1f s)"
                                              % (ncell, npart, t)}
        print(json.dumps(line))
    pl.close()
    if world > 1:
        dist.destroy_process_group()


def kernel_hash():
    import hashlib
    h = hashlib.sha256()
    for name in ("step.cu", "common.cuh", "tables.h"):
        with open(os.path.join(ROOT, "paper_2604_24627_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    main()
