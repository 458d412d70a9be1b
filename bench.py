#!/usr/bin/env python3
"""Benchmark: zone-updates/s of the IMEX-RK3 step of the radiation-RMHD path.

Workload (default): a batch of 4096 independent 1D RRMHD Riemann problems from
seed 2212003701 (grid sizes U{128..2048}, log-uniform densities, pressures,
radiation energies and opacities, Lorentz factors up to 10, gamma 4/3), all
advanced together.  One "step" is one IMEX-RK3 step of every live instance
(3 stages x {PLM + PVM-int-8 fluxes, flux difference + RK, implicit
radiation-matter solve}); a zone-update is one cell advanced by one step.
The headline is the FP32-bulk form; the FP64 form (and FP64 with tangent
products) are measured beside it.  Launch shapes are autotuned before timing
(untimed, state restored).  A serving sample of the C4 arrival process (continuous
batching, time to solution) and the CPU oracle are measured too.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  ``value`` is device throughput with the state resident
in HBM, the K timed steps enqueued as one rrmhd_imex_step call; ``p50_ms`` /
``p99_ms`` are the same K steps again (restored from a checkpoint) one call per
step; ``e2e`` the same K steps once more through the C-ABI host-buffer entry
(rrmhd_imex_step_host: H2D of the state, the step, D2H of the primitives, every
step).  N > 1 (torchrun): every rank advances its own batch (seed + rank):
independent problems, no data-path collective, weak scaling.
``--impl reference`` times the FP64 CPU oracle on the host cores instead.
"""
import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# FP64-pipe instructions (DADD + DMUL + DFMA, thread level, ncu
# sm__sass_thread_inst_executed_op_d{add,mul,fma}_pred_on.sum) per cell of one launch
# of each kernel in the steady state of this workload, averaged over the three stages
# of the 4th step (their implicit weights differ, and so does the solve's work), measured
# with ncu on a 2048-instance sample of the same distribution.
FP64_INST_PER_ZONE = {"fp64": {"faces": 4832.0, "cells": 4591.0},
                      "fp32_bulk": {"faces": 4.0, "cells": 2281.0},
                      "fp64_tangent": {"faces": 5238.0, "cells": 4591.0}}
# DRAM bytes per cell of one launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)
TRAFFIC_PER_CELL = {"fp64": {"faces": 239.0, "cells": 1669.0},
                    "fp32_bulk": {"faces": 439.0, "cells": 2293.0},
                    "fp64_tangent": {"faces": 241.0, "cells": 1669.0}}
# Nominal FP64 rate of GB300: 1.25 TFLOP/s = 6.25e11 FP64-pipe instructions/s
# (2 per SM per clock on 152 SMs at 2.07 GHz).  The roofline divides by the rate
# rrmhd_probe_fp64 measures in the same run; the nominal figure is reported beside it.
FP64_NOMINAL_INST = 6.25e11
BYTES_PER_ZONE_STEP = 1392.0  # minimum HBM bytes per zone-update (state in/out per stage)
HBM_FALLBACK_GBS = 6800.0     # copy bandwidth of an earlier GB300 measurement


def hbm_peak():
    """Measured copy bandwidth (GB/s) of the GB300s, and where it comes from."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (measured)"
    except (OSError, KeyError, ValueError):
        return HBM_FALLBACK_GBS, "fallback 6.8 TB/s (no MEASURED_PEAKS.json)"


def fp64_peak(skip=False):
    """FP64-pipe rate measured now (burst: 3 x ~150 ms; sustained: 3 x ~1.5 s)."""
    from paper_2212_00370_gb300 import rrmhd
    if skip:
        return {"burst": FP64_NOMINAL_INST, "sustained": FP64_NOMINAL_INST,
                "nominal": FP64_NOMINAL_INST, "how": "not measured (--no-fp64-probe): nominal rate"}
    burst = rrmhd.probe_fp64(150.0)
    sustained = rrmhd.probe_fp64(1500.0)
    return {"burst": burst, "sustained": sustained, "nominal": FP64_NOMINAL_INST,
            "dependent_latency_ns": rrmhd.probe_fp64_latency(),
            "how": "rrmhd_probe_fp64: 8 independent DFMA chains per thread, 2048 threads per SM "
                   "on every SM, CUDA events, best of 3 runs of ~150 ms (burst) and ~1.5 s "
                   "(sustained), measured in this run"}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--instances", type=int, default=4096)
    p.add_argument("--workload", default="c1", choices=["c1", "c0"],
                   help="c1: the 4096-instance batch (the headline); c0: the 400-cell radiative "
                        "shock tube alone (FP64, to t_end), a latency-bound small grid")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--cpu-sample", type=int, default=None,
                   help="instances in the CPU sample (default: 1024 for the cpu_baseline leg, "
                        "the whole batch for --impl reference)")
    p.add_argument("--lanes", type=int, default=8, help="independent sub-batches (streams)")
    p.add_argument("--recon", default="vanleer", choices=["vanleer", "minmod", "mc", "godunov"],
                   help="reconstruction of the timed C1 lines (Sec. 3.2); godunov times the "
                        "path without PLM, whose cost it isolates")
    p.add_argument("--precision", default="both", choices=["both", "fp64", "fp32_bulk", "fp64_tangent"],
                   help="both: FP32-bulk is the headline value, FP64 (and FP64 with tangent "
                        "products) reported beside it")
    p.add_argument("--serve-requests", type=int, default=96,
                   help="requests of the C4 serving sample (0: skip the serving measurement)")
    p.add_argument("--serve-cells", type=int, default=4_000_000,
                   help="resident-cell bound of the serving loop (bounds its step time)")
    p.add_argument("--no-others", action="store_true",
                   help="skip the per-step timings of the other workloads (C0 shock tube, 2D blast, 3D box)")
    p.add_argument("--no-autotune", action="store_true",
                   help="keep the default launch shapes instead of autotuning them before timing")
    p.add_argument("--no-fp64-probe", action="store_true",
                   help="skip the FP64-pipe probe (profiling runs); the roofline then divides by "
                        "the nominal FP64 rate")
    p.add_argument("--tuning", default=None,
                   help='fixed launch shapes as JSON, e.g. \'{"cell_block": 32, "lanes": 32}\' (no autotune)')
    return p.parse_args()


# ----------------------------------------------------------------------------- CPU oracle
_WORKER = {}


def _worker_init(seed, n_inst):
    """Pool initializer: build the oracle and the workload once per worker process."""
    import oracle as O
    from paper_2212_00370_gb300 import workloads as W
    O.lib()
    _WORKER["w"] = W.riemann_batch(n_inst, seed=seed)


def _oracle_slice_steps(args):
    """Worker: the instances of one fixed slice, `warm` untimed steps, then `steps`
    timed steps of the whole slice (each instance keeps its state and Jacobian cache
    from step to step, as a run does).  Returns the wall time and the zone-updates of
    every timed step (a failed instance stops contributing)."""
    idx, warm, steps = args
    import oracle as O
    w = _WORKER["w"]
    P = O.Params(gamma=w.gamma, a_rad=w.a_rad, cfl=w.cfl)
    insts = []
    for i in idx:
        g, V, kappa, sigma = w.instance(int(i))
        V = np.ascontiguousarray(V).copy()
        grid = O.Grid(1, (g["n"][0],), (g["dx"][0],))
        insts.append([grid, O.prim2con(V, P), V, kappa, sigma, np.zeros(17 * g["n"][0]), True])

    def one_step():
        zones = 0
        for it in insts:
            grid, U, V, kappa, sigma, jc, ok = it
            if not ok:
                continue
            dt = O.grid_dt(grid, V, P)
            if not (dt > 0) or O.step(grid, dt, U, V, kappa, sigma, P, jcache=jc):
                it[6] = False
                continue
            zones += grid.ncells
        return zones

    for _ in range(warm):
        one_step()
    times, zones = [], []
    for _ in range(steps):
        t0 = time.perf_counter()
        zones.append(one_step())
        times.append(time.perf_counter() - t0)
    return times, zones


def make_pool(cores, seed, n_inst):
    pool = mp.get_context("spawn").Pool(cores, initializer=_worker_init, initargs=(seed, n_inst))
    pool.map(_noop, range(cores))  # wait until every worker is initialised
    return pool


def _noop(x):
    return x


def cpu_oracle(pool, cores, n_inst, sample, warm, steps):
    """Oracle throughput on `sample` instances evenly spread over the batch, split into
    `cores` fixed slices (one per worker process, running concurrently): `warm` untimed
    steps, then `steps` timed steps, the steady state the GPU arm times.  A step's wall
    time is that of the slowest slice.  Returns (zone-updates/s, per-step wall times in
    s, zone-updates)."""
    idx = np.linspace(0, n_inst - 1, sample).astype(int)
    slices = [idx[k::cores] for k in range(cores)]
    res = pool.map(_oracle_slice_steps, [(sl, warm, steps) for sl in slices], chunksize=1)
    walls = [max(r[0][k] for r in res) for k in range(steps)]
    zones = sum(sum(r[1]) for r in res)
    return zones / sum(walls), walls, zones


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons every 200 ms while running."""

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 7:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[3 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ----------------------------------------------------------------------------- GPU arm
def aggregate_over_ranks(t_s, zones, world):
    """Whole-job figures of replicas: the slowest rank's time and the zone-updates
    of all ranks (no data-path collective; this is the one reduction)."""
    if world <= 1:
        return t_s, zones
    import torch
    import torch.distributed as dist
    tt = torch.tensor([t_s, zones], dtype=torch.float64)
    mx = tt.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(tt, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(tt[1])


def measure(a, precision, rank, world, local, peaks):
    """Time K steps of the C1 batch in one precision; returns a dict of measurements."""
    import torch
    import torch.distributed as dist

    from paper_2212_00370_gb300 import rrmhd
    from paper_2212_00370_gb300 import workloads as W

    seed = W.SEED_BASE + 1 + rank
    w = W.riemann_batch(a.instances, seed=seed)
    grids = [rrmhd.make_grid(1, g["n"], g["dx"], g["bc"]) for g in w.grids]
    extra = {"pvm_products": 1} if precision == "fp64_tangent" else {}
    extra["recon"] = a.recon
    ctx = rrmhd.Context(grids, gamma=w.gamma, a_rad=w.a_rad, cfl=w.cfl, lanes=a.lanes,
                        precision="fp64" if precision == "fp64_tangent" else precision, **extra)
    ctx.set_opacity(torch.tensor(w.kappa, device="cuda"), torch.tensor(w.sigma, device="cuda"))
    ctx.set_state(torch.tensor(w.V, device="cuda"))
    ctx.set_times(np.zeros(w.n_inst), np.full(w.n_inst, np.inf))
    n_cells = np.array([g["n"][0] for g in w.grids], dtype=np.int64)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()

    if a.tuning:                             # fixed shapes from the first step on
        ctx.set_tuning(**json.loads(a.tuning))
    ctx.imex_step(max(a.warmup, 2))          # warm-up (also builds the step graphs)
    torch.cuda.synchronize()
    tuning, tune_ms = ctx.get_tuning(), None
    if not (a.tuning or a.no_autotune):      # untimed: shapes chosen on this state, state restored
        t0 = time.perf_counter()
        tuning, tune_ms = ctx.autotune(repeats=2)
        tune_s = time.perf_counter() - t0
        ctx.imex_step(1)                     # warm the chosen shapes' graphs
        torch.cuda.synchronize()
    st_before = ctx.inst_status()
    # the state the timed steps start from (with the implicit solver's Jacobian cache),
    # so that the step-time distribution and e2e run the same K steps
    ck = ctx.checkpoint()
    # timed: the K steps as one call (the lanes run them back to back and join once)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev[0].record(stream)
        ctx.imex_step(a.steps)
        ev[1].record(stream)
        torch.cuda.synchronize()
    barrier()
    total_ms = ev[0].elapsed_time(ev[1])
    st_after = ctx.inst_status()
    live = (st_before == 0) & (st_after == 0)
    zones = float(n_cells[live].sum()) * a.steps
    t_s, zones = aggregate_over_ranks(total_ms / 1e3, zones, world)
    value = zones / t_s
    # the step-time distribution: the same K steps, one call each (the lanes join every step)
    ctx.checkpoint_restore(ck)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps + 1)]
    evs[0].record(stream)
    for k in range(a.steps):
        ctx.imex_step(1)
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    step_ms = [evs[k].elapsed_time(evs[k + 1]) for k in range(a.steps)]

    # per-launch-group device times of two more steps (same kernels, whole-batch launches)
    prof = np.zeros(4)
    for _ in range(2):
        prof += ctx.profile_step()
    prof /= 2
    zones_step = float(n_cells[live].sum())
    groups = {"faces": prof[0] / 3.0, "cells": prof[1] / 3.0}
    counts = FP64_INST_PER_ZONE[precision]
    dom = max(groups, key=groups.get)
    per_zone = counts.get(dom)
    achieved = per_zone * zones_step / (groups[dom] / 1e3) if per_zone else None
    kname = {"fp32_bulk": "k_cells_f32 (FP32-bulk cells: FP64 con2prim + implicit solve)",
             "fp64": "k_cells (FP64)", "fp64_tangent": "k_cells (FP64, tangent products)"}[precision]
    if dom == "faces":
        kname = "k_faces_f32 (FP32-bulk faces)" if precision == "fp32_bulk" else "k_faces (FP64)"
    hbm_gbs, hbm_src = peaks["hbm"]
    peak = peaks["fp64"]["burst"]
    roofline = {
        "bound": "alu", "kernel": kname,
        "achieved": achieved, "peak": peak, "unit": "FP64-pipe inst/s",
        "frac": (achieved / peak) if achieved else None,
        "traffic": TRAFFIC_PER_CELL[precision].get(dom, 0) * zones_step or None,
        "peak_source": "burst rate, " + peaks["fp64"]["how"],
        "peak_nominal": FP64_NOMINAL_INST,
        "frac_of_nominal": (achieved / FP64_NOMINAL_INST) if achieved else None,
        "launch_ms": {"faces": round(groups["faces"], 4), "cells": round(groups["cells"], 4),
                      "fallback": round(prof[2] / 3.0, 4), "step_control": round(prof[3] / 2.0, 4)},
        "hbm_frac": BYTES_PER_ZONE_STEP * value / max(world, 1) / (hbm_gbs * 1e9),
        "hbm_peak_gbs": hbm_gbs, "hbm_peak_source": hbm_src,
    }
    # the same FP64 instruction counts over the live, lane-overlapped timed region:
    # (faces + cells) per zone and stage x 3 stages x zone-updates/s, per GPU; a
    # kernel inside a long step is held to the sustained rate
    live_rate = 3.0 * ((counts.get("faces") or 0.0) + counts["cells"]) * value / max(world, 1)
    roofline["live_achieved"] = live_rate
    roofline["live_frac"] = live_rate / peaks["fp64"]["sustained"]
    roofline["live_peak"] = peaks["fp64"]["sustained"]
    roofline["live_note"] = ("FP64-pipe instructions of the step's face and cell kernels per "
                             "zone-update x zone-updates/s of the timed region, per GPU; the "
                             "whole-batch launch above also carries its tail of slow solves")

    e2e = None
    if not a.no_e2e:
        ctx.checkpoint_restore(ck)           # the same K steps as the device-timed value
        _, Vdev = ctx.get_state()
        h_in = torch.empty(Vdev.shape, dtype=torch.float64, pin_memory=True)
        h_out = torch.empty(Vdev.shape, dtype=torch.float64, pin_memory=True)
        h_in.copy_(Vdev)
        torch.cuda.synchronize()
        ke = a.steps
        t0 = time.perf_counter()
        for _ in range(ke):
            ctx.imex_step_host(h_in, h_out, 1)
            h_in, h_out = h_out, h_in
        te = time.perf_counter() - t0
        st_e = ctx.inst_status()
        nbytes = 12 * 8 * w.ncells
        e2e = {"value": float(n_cells[st_e == 0].sum()) * ke / te, "unit": "zone-updates/s",
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "steps": ke}
    out = {"value": value, "ms_per_step": total_ms / a.steps,
           "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
           "roofline": roofline, "e2e": e2e, "gpu_launches": ctx.launches_per_step() * a.steps,
           "clocks": clk.summary(), "live": int(live.sum()), "failed": int((~live).sum()),
           "cells": int(n_cells.sum()), "ncells_state_mb": 12 * 8 * w.ncells / 1e6, "seed": seed,
           "tuning": tuning, "autotune": None if (a.no_autotune or a.tuning) else
           {"best_step_ms": tune_ms, "wall_s": round(tune_s, 1), "repeats": 2}}
    ctx.close()
    return out


def measure_variant(a, opts, tuning, steps=5):
    """Zone-updates/s of the C1 batch (FP64) with other solver options: the paper's
    variants timed beside PVM-int-8.  Same seed and launch shapes as the FP64 line;
    warm-up 2 steps, then `steps` steps timed with CUDA events."""
    import torch

    from paper_2212_00370_gb300 import rrmhd
    from paper_2212_00370_gb300 import workloads as W

    w = W.riemann_batch(a.instances, seed=W.SEED_BASE + 1)
    grids = [rrmhd.make_grid(1, g["n"], g["dx"], g["bc"]) for g in w.grids]
    ctx = rrmhd.Context(grids, gamma=w.gamma, a_rad=w.a_rad, cfl=w.cfl, precision="fp64", **opts)
    if tuning:
        ctx.set_tuning(**tuning)
    ctx.set_opacity(torch.tensor(w.kappa, device="cuda"), torch.tensor(w.sigma, device="cuda"))
    ctx.set_state(torch.tensor(w.V, device="cuda"))
    ctx.set_times(np.zeros(w.n_inst), np.full(w.n_inst, np.inf))
    n_cells = np.array([g["n"][0] for g in w.grids], dtype=np.int64)
    stream = torch.cuda.current_stream()
    ctx.imex_step(2)
    torch.cuda.synchronize()
    st0 = ctx.inst_status()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.imex_step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    live = (st0 == 0) & (ctx.inst_status() == 0)
    launches = ctx.launches_per_step() * steps
    ctx.close()
    return {"value": float(n_cells[live].sum()) * 1e3 / ms, "ms_per_step": ms, "steps": steps,
            "failed_instances": int((~live).sum()), "launches": launches}


VARS = ["D", "Sx", "Sy", "Sz", "tau", "Bx", "By", "Bz", "E", "Fx", "Fy", "Fz"]


def _rel_l1(a, b):
    out = {}
    for k in range(12):
        den = np.abs(b[k]).sum()
        if den > 0:
            out[VARS[k]] = float(np.abs(a[k] - b[k]).sum() / den)
    return out


def measure_accuracy(a, n_inst=None, steps=5):
    """Per-variable relative L1 of the FP32-bulk form against the FP64 form (which is
    bit-identical to the oracle) on the C1 batch (or an evenly spaced sample of n_inst
    instances) after `steps` steps, over the whole batch and per instance.  An instance above 1e-5 in
    some variable is checked against the FP64 N-vs-2N difference of that instance (the
    same problem on 2N cells run to the same time, averaged onto N)."""
    import torch

    from paper_2212_00370_gb300 import rrmhd
    from paper_2212_00370_gb300 import workloads as W

    w = W.riemann_batch(a.instances, seed=W.SEED_BASE + 1)
    if n_inst and n_inst < w.n_inst:
        w = w.subset(list(np.linspace(0, w.n_inst - 1, n_inst).astype(int)))

    def run(wl, prec, t_end, nsteps):
        grids = [rrmhd.make_grid(1, g["n"], g["dx"], g["bc"]) for g in wl.grids]
        ctx = rrmhd.Context(grids, gamma=wl.gamma, a_rad=wl.a_rad, cfl=wl.cfl, precision=prec)
        ctx.set_opacity(torch.tensor(wl.kappa, device="cuda"), torch.tensor(wl.sigma, device="cuda"))
        ctx.set_state(torch.tensor(wl.V, device="cuda"))
        ctx.set_times(np.zeros(wl.n_inst), t_end)
        ctx.imex_step(nsteps)
        out = (ctx.get_state()[0].cpu().numpy(), ctx.inst_status(), ctx.get_times()[0])
        ctx.close()
        return out

    inf = np.full(w.n_inst, np.inf)
    U32, s32, _ = run(w, "fp32_bulk", inf, steps)
    U64, s64, t64 = run(w, "fp64", inf, steps)
    off = w.cell_offsets()
    live = (s32 == 0) & (s64 == 0)
    keep = np.zeros(w.ncells, dtype=bool)
    above, worst = [], 0.0
    for i in np.nonzero(live)[0]:
        keep[off[i]:off[i + 1]] = True
        e = _rel_l1(U32[:, off[i]:off[i + 1]], U64[:, off[i]:off[i + 1]])
        worst = max(worst, max(e.values()))
        if max(e.values()) > 1e-5:
            above.append((int(i), e))
    l1 = _rel_l1(U32[:, keep], U64[:, keep])
    below = 0
    if above:   # the FP64 N-vs-2N difference of those instances
        parts = [w.instance(i) for i, _ in above]
        w2 = W.Workload("C1-2N", [W.grid1d(2 * g["n"][0]) for g, *_ in parts],
                        np.ascontiguousarray(np.concatenate([np.repeat(V, 2, axis=1) for _, V, _, _ in parts], 1)),
                        np.concatenate([np.repeat(k, 2) for _, _, k, _ in parts]),
                        np.concatenate([np.repeat(sg, 2) for _, _, _, sg in parts]),
                        np.array([t64[i] for i, _ in above]), w.gamma, w.a_rad, w.cfl)
        U2, s2, _ = run(w2, "fp64", w2.t_end, 40 * steps)
        off2 = w2.cell_offsets()
        for j, (i, e) in enumerate(above):
            u2 = U2[:, off2[j]:off2[j + 1]]
            trunc = _rel_l1(0.5 * (u2[:, 0::2] + u2[:, 1::2]), U64[:, off[i]:off[i + 1]])
            if s2[j] == 0 and all(v < trunc[k] for k, v in e.items() if v > 1e-5):
                below += 1
    return {"rel_l1_vs_fp64": l1, "max": max(l1.values()), "instances": int(w.n_inst),
            "compared": int(live.sum()), "steps": steps,
            "failed_one_form_only": int(((s32 == 0) != (s64 == 0)).sum()),
            "failed_both": int(((s32 != 0) & (s64 != 0)).sum()),
            "instances_above_1e-5": len(above), "of_which_below_their_n_vs_2n_difference": below,
            "worst_instance_max_variable": worst,
            "note": "FP64 form = the oracle bit for bit; bound per variable and instance: 1e-5, "
                    "or below the instance's N-vs-2N difference"}


def measure_workload(w, precision, steps, ct=0, warmup=2):
    """Per-step device times (CUDA events) of one workload in one context: zone-updates/s
    over the timed steps and p50/p99 of the step time.  Steps stop at t_end.  A grid of
    fewer than 100k cells fills few SMs with the default 128-thread blocks: its launch
    shapes are autotuned first (untimed, state restored)."""
    import torch

    from paper_2212_00370_gb300 import rrmhd

    grids = [rrmhd.make_grid(g["ndim"], g["n"], g["dx"], g["bc"]) for g in w.grids]
    ctx = rrmhd.Context(grids, gamma=w.gamma, a_rad=w.a_rad, cfl=w.cfl, precision=precision, ct=ct,
                        lanes=1)
    ctx.set_opacity(torch.tensor(w.kappa, device="cuda"), torch.tensor(w.sigma, device="cuda"))
    ctx.set_state(torch.tensor(w.V, device="cuda"))
    ctx.set_times(np.zeros(w.n_inst), w.t_end)
    stream = torch.cuda.current_stream()
    ctx.imex_step(warmup)
    torch.cuda.synchronize()
    tuning = None
    if w.ncells < 100_000:
        tuning, _ = ctx.autotune(repeats=3)
        torch.cuda.synchronize()
    ms = []
    for _ in range(steps):
        t_before = ctx.get_times()[0]
        if np.all(t_before >= w.t_end) or np.any(ctx.inst_status() != 0):
            break
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.imex_step(1)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    st = ctx.inst_status()
    ctx.close()
    torch.cuda.empty_cache()
    if not ms:
        return {"steps": 0, "status": st.tolist()}
    return {"value": w.ncells * 1e3 * len(ms) / sum(ms), "unit": "zone-updates/s", "steps": len(ms),
            "ms_per_step": sum(ms) / len(ms), "p50_ms": float(np.percentile(ms, 50)),
            "p99_ms": float(np.percentile(ms, 99)), "cells": int(w.ncells), "precision": precision,
            "ct": ct, "status": int(st.max()), "launch_shapes": tuning}


def measure_others(peaks=None):
    """The other benchmark workloads, each in its own context: the C0 radiative shock
    tube (400 cells, FP64) to t_end = 0.4 after 2 warm-up steps; the 2D 1024^2 blast
    (FP32-bulk, constrained transport) and the 3D 256^3 box (FP32-bulk and FP64,
    constrained transport) over a few steps."""
    from paper_2212_00370_gb300 import workloads as W
    out = {}
    out["shock_tube_400_fp64"] = measure_workload(W.shock_tube(400), "fp64", 1000)
    lat = (peaks or {}).get("fp64", {}).get("dependent_latency_ns")
    if lat:
        out["shock_tube_400_fp64"]["bound"] = (
            "FP64 dependent-instruction latency: 400 cells make ~13 warps, one per SM, and a "
            "dependent FP64 instruction of one warp takes %.1f ns (rrmhd_probe_fp64_latency); "
            "the per-cell Newton chains are serial, so block shapes do not change the step "
            "time" % lat)
    c2 = W.blast_2d()
    out["blast_2d_1024x1024_fp32_bulk_ct"] = measure_workload(c2, "fp32_bulk", 20, ct=1)
    c3 = W.turbulent_3d()
    out["box_3d_256cubed_fp32_bulk_ct"] = measure_workload(c3, "fp32_bulk", 5, ct=1)
    out["box_3d_256cubed_fp64_ct"] = measure_workload(c3, "fp64", 3, ct=1)
    return out


def measure_serving(a, tuning=None):
    """C4 serving sample: the first `serve_requests` requests of the C4 arrival process
    (Poisson, 200 requests/s; 70 % 1D N~U{256..4096}, 30 % planar 2D side~U{128..512};
    C1 states; t_end 0.2; FP32-bulk, constrained transport for the 2D requests)
    submitted at their arrival times from a host thread into the serving loop, which
    runs them to completion."""
    from paper_2212_00370_gb300 import rrmhd
    from paper_2212_00370_gb300 import workloads as W

    n_req = a.serve_requests
    rate = 200.0
    specs = W.serving_requests(n_req, rate=rate)
    reqs = [W.serving_request(sp) for sp in specs]
    grids = [rrmhd.make_grid(g["ndim"], g["n"], g["dx"], g["bc"]) for g, *_ in reqs]
    # zone-updates a request needs at most: steps <= t_end * sum_d 1/dx_d / cfl (speeds <= c)
    def zu_max(sp):
        n = sp["size"]
        return (n * 0.2 * n / 0.4) if sp["ndim"] == 1 else (n * n * 0.2 * 2 * n / 0.4)
    all_specs = W.serving_requests(12000, rate=rate)
    offered = sum(zu_max(sp) for sp in all_specs) / all_specs[-1]["arrival"]

    srv = rrmhd.Server(gamma=4.0 / 3.0, precision="fp32_bulk", lanes=a.lanes, ct=1,
                       max_resident_cells=a.serve_cells, tuning=tuning)
    srv.wait_idle(1.0)

    index_of = {}

    def submitter():
        t0 = time.perf_counter()
        for k, (sp, g, (gd, V, kp, sg, te)) in enumerate(zip(specs, grids, reqs)):
            delay = sp["arrival"] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            index_of[srv.submit(g, V, kp, sg, te)] = k

    th = threading.Thread(target=submitter)
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        th.start()
        results = []
        deadline = time.perf_counter() + 900
        while len(results) < n_req and time.perf_counter() < deadline:
            time.sleep(0.01)
            results += srv.poll()
        th.join()
    st = srv.stats()
    srv.close()
    ok = [r for r, _ in results if r["status"] == 0]
    tts = np.array([r["done_s"] - r["submit_s"] for r in ok])
    service = np.array([r["done_s"] - r["admit_s"] for r in ok])
    queueing = np.array([r["admit_s"] - r["submit_s"] for r in ok])
    span = max(r["done_s"] for r, _ in results) - min(r["submit_s"] for r, _ in results)

    def pct(x, q):
        return float(np.percentile(x, q)) if len(x) else None
    return {
        "workload": "C4 sample: first %d requests of Poisson arrivals at %.0f/s (70%% 1D N~U{256..4096}, "
                    "30%% planar 2D side~U{128..512}, C1 states, t_end 0.2, FP32-bulk, CT for 2D)" % (n_req, rate),
        "requests": n_req, "completed": len(results), "failed": len(results) - len(ok),
        "failed_requests": [{"index": index_of.get(r["id"]), "ndim": specs[index_of[r["id"]]]["ndim"],
                             "size": specs[index_of[r["id"]]]["size"], "status": r["status"],
                             "steps": r["steps"], "t": r["t"]}
                            for r, _ in results if r["status"] != 0 and r["id"] in index_of],
        "p50_tts_s": pct(tts, 50), "p99_tts_s": pct(tts, 99),
        "p50_service_s": pct(service, 50), "p99_service_s": pct(service, 99),
        "p50_queueing_s": pct(queueing, 50), "p99_queueing_s": pct(queueing, 99),
        "arrival_window_s": specs[-1]["arrival"] - specs[0]["arrival"],
        "sample_offered_zone_updates_per_s_at_most":
            sum(zu_max(sp) for sp in specs) / max(specs[-1]["arrival"] - specs[0]["arrival"], 1e-9),
        "zone_updates_per_s": st["zone_updates"] / span, "zone_updates": st["zone_updates"],
        "makespan_s": span, "server_steps": st["steps"], "relayouts": st["relayouts"],
        "resident_cell_bound": st["cap_cells"], "peak_resident_cells": st["peak_resident_cells"],
        "busy_frac": st["busy_s"] / span,
        "offered_zone_updates_per_s_at_most": offered,
        "note": "the full C4 process (12,000 requests at 200/s) offers up to %.2g zone-updates/s, "
                "about %.0fx what one GPU sustains: it saturates, and its p99 would be a queueing "
                "number; the sample is run to completion instead" % (offered, offered / max(st["zone_updates"] / span, 1.0)),
        "clocks": clk.summary(),
    }


DTYPE = {"fp64": "f64", "fp32_bulk": "f32 faces + f64 cells", "fp64_tangent": "f64"}
METRIC = "zone-updates/s per IMEX step (FP32-bulk vs FP64, 1 GB300; % of roofline; p50/p99 step time)"


def workload_name(n_inst, recon="vanleer"):
    names = {"vanleer": "VanLeer", "minmod": "MinMod", "mc": "MC", "godunov": "first order"}
    return ("C1: %d independent 1D RRMHD Riemann problems per GPU, N~U{128..2048}, seed "
            "2212003701+rank, gamma 4/3, PVM-int-8 + %s + IMEX-RK3" % (n_inst, names[recon]))


def run_c0(a):
    """The C0 shock tube alone: per-step device times to t_end, and the FP64 latency
    probe that bounds it."""
    from paper_2212_00370_gb300 import rrmhd
    from paper_2212_00370_gb300 import workloads as W
    r = measure_workload(W.shock_tube(400), "fp64", 1000, warmup=a.warmup)
    lat = None if a.no_fp64_probe else rrmhd.probe_fp64_latency()
    return {"metric": "zone-updates/s per IMEX step (C0 shock tube, 400 cells, FP64)",
            "value": r.get("value"), "unit": "zone-updates/s", "n_gpus": 1, "steps": r.get("steps"),
            "warmup": a.warmup, "ms_per_step": r.get("ms_per_step"), "p50_ms": r.get("p50_ms"),
            "p99_ms": r.get("p99_ms"), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "C0: 1D radiative shock tube, 400 cells, gamma 5/3, kappa 1, to t_end 0.4",
                       "launch_shapes": r.get("launch_shapes")},
            "fp64_dependent_latency_ns": lat}


def run_ours(a, rank, world, pool, cores):
    import torch

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if a.workload == "c0":
        return run_c0(a)
    precisions = ["fp32_bulk", "fp64", "fp64_tangent"] if a.precision == "both" else [a.precision]
    from paper_2212_00370_gb300 import rrmhd  # noqa: F401  (loads the library)
    peaks = {"fp64": fp64_peak(a.no_fp64_probe), "hbm": hbm_peak()}
    res = {p: measure(a, p, rank, world, local, peaks) for p in precisions}
    head = res[precisions[0]]
    out = {
        "metric": METRIC,
        "value": head["value"], "unit": "zone-updates/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[precisions[0]], "data": "synthetic",
        "config": {"workload": workload_name(a.instances, a.recon), "precision": precisions[0],
                   "instances": a.instances, "cells": head["cells"],
                   "live_instances": head["live"], "failed_instances": head["failed"],
                   "parallelism": "replicas (independent problems per GPU); %d lanes (streams) per GPU"
                                  % head["tuning"]["lanes"],
                   "launch_shapes": head["tuning"], "autotune": head["autotune"],
                   "l2": "state %.0f MB per copy > 129 MB L2 (inputs larger than L2)" % head["ncells_state_mb"]},
        "p50_ms": head["p50_ms"], "p99_ms": head["p99_ms"],
        "timing": "value and ms_per_step: the K steps as one rrmhd_imex_step call (the lanes "
                  "run them back to back and join once); p50_ms/p99_ms: K further steps, one "
                  "call each (the lanes join every step)",
        "roofline": head["roofline"], "e2e": head["e2e"], "gpu_launches": head["gpu_launches"],
        "clocks": head["clocks"], "fp64_peak": peaks["fp64"],
    }
    if len(precisions) > 1:
        f = res["fp64"]
        out["fp64"] = {"value": f["value"], "ms_per_step": f["ms_per_step"], "p50_ms": f["p50_ms"],
                       "launch_shapes": f["tuning"],
                       "p99_ms": f["p99_ms"], "roofline": f["roofline"], "e2e": f["e2e"],
                       "failed_instances": f["failed"], "clocks": f["clocks"]}
        out["fp32_bulk_speedup_over_fp64"] = head["value"] / f["value"]
        # the whole batch, after 5 and after 12 steps
        out["fp32_bulk_accuracy"] = measure_accuracy(a, steps=5)
        out["fp32_bulk_accuracy_12_steps"] = measure_accuracy(a, steps=12)
        out["gpu_launches"] += f["gpu_launches"]
        g = res["fp64_tangent"]
        out["fp64_tangent"] = {"value": g["value"], "ms_per_step": g["ms_per_step"], "p50_ms": g["p50_ms"],
                               "p99_ms": g["p99_ms"], "launch_shapes": g["tuning"],
                               "failed_instances": g["failed"], "e2e": g["e2e"],
                               "note": "FP64 with exact tangent Jacobian products instead of the "
                                       "paper's eps = 1e-8 flux differences (a variant)"}
        out["gpu_launches"] += g["gpu_launches"]
        # the paper's variants, FP64, same workload and shapes as the FP64 line
        variants = {}
        for name, opts in (("radhll", {"solver": "radhll"}), ("pvm_int16", {"pvm_k": 4}),
                           ("beta_radiation_only", {"beta": "radiation"})):
            variants[name] = measure_variant(a, opts, f["tuning"])
            out["gpu_launches"] += variants[name].pop("launches")
        variants["pvm_int8_time_over_radhll"] = variants["radhll"]["value"] / f["value"]
        variants["note"] = ("FP64 zone-updates/s of Rad-HLL (Sec. 3.2.1), PVM-int-16 and "
                            "PVM-int-8 with beta on the radiation block only on the C1 batch; "
                            "the paper reports PVM-int-8 costing ~2x HLL in CPU time")
        out["fp64_variants"] = variants
    if not a.no_others and world == 1:
        out["other_workloads"] = measure_others(peaks)
    if a.serve_requests > 0 and world == 1:
        out["serving"] = measure_serving(a, res["fp32_bulk"]["tuning"] if "fp32_bulk" in res else None)
    if rank == 0 and pool is not None:
        from paper_2212_00370_gb300 import workloads as W
        zps, walls, zc = cpu_oracle(pool, cores, a.instances, a.cpu_sample, 2, 2)
        out["cpu_baseline"] = {"value": zps, "unit": "zone-updates/s", "cores": cores, "kind": "oracle",
                               "sample": "%d of the %d instances (evenly spaced, seed %d), 2 untimed warm-up "
                                         "steps, then 2 timed steps: %d zone-updates in %.1f s wall"
                                         % (a.cpu_sample, a.instances, W.SEED_BASE + 1, zc, sum(walls))}
    return out


def run_reference(a, rank, pool, cores):
    """The reference arm: the FP64 CPU oracle on the host cores, on the same C1 batch,
    steady state as the GPU arm times it (W untimed steps, then K timed steps of the
    sampled instances)."""
    zps, walls, zones = cpu_oracle(pool, cores, a.instances, a.cpu_sample, a.warmup, a.steps)
    return {
        "impl": "reference",
        "metric": METRIC,
        "value": zps, "unit": "zone-updates/s", "n_gpus": 0, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": 1e3 * sum(walls) / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(a.instances), "precision": "fp64 (CPU oracle)",
                   "instances": a.instances, "sampled_instances": a.cpu_sample},
        "cpu_baseline": {"value": zps, "unit": "zone-updates/s", "cores": cores, "kind": "oracle",
                         "sample": "%d of the %d instances (evenly spaced), %d untimed warm-up steps, "
                                   "then %d timed steps, one fixed slice per core"
                                   % (a.cpu_sample, a.instances, a.warmup, a.steps)},
        "e2e": {"value": zps, "unit": "zone-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "p50_ms": float(np.percentile(walls, 50) * 1e3), "p99_ms": float(np.percentile(walls, 99) * 1e3),
    }


def main():
    a = parse()
    if a.cpu_sample is None:
        a.cpu_sample = a.instances if a.impl == "reference" else min(1024, a.instances)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    from oracle import build as OB
    OB.build()
    pool = None
    # the oracle pool is started (spawn) before the first GPU call, on rank 0 only
    if rank == 0 and (a.impl == "reference" or (not a.no_cpu and a.workload == "c1")):
        from paper_2212_00370_gb300 import workloads as W
        pool = make_pool(cores, W.SEED_BASE + 1, a.instances)
    try:
        if a.impl == "reference":
            if rank != 0:
                return
            out = run_reference(a, rank, pool, cores)
        else:
            if world > 1:
                import torch.distributed as dist
                dist.init_process_group("gloo")
            from paper_2212_00370_gb300 import build as B
            if rank == 0:
                B.build()
            if world > 1:
                import torch.distributed as dist
                dist.barrier()
            out = run_ours(a, rank, world, pool, cores)
            if rank != 0:
                return
        print(json.dumps(out), flush=True)
    finally:
        if pool is not None:
            pool.close()
            pool.join()


if __name__ == "__main__":
    main()
