#!/usr/bin/env python
"""Throughput benchmark of the DPDE timestep (particle-steps/s).

One "step" is one full DPDE timestep of the workload: velocity Verlet with the
cell-list rebuild, conservative forces, and the fluctuation/dissipation scheme
(default: Hybrid, which runs the SSA rounds over intra-domain pairs and the two
SER sweeps over cross-domain pairs). Default workload: 4,000,000 particles at
density 3 (L ~ 110.1), C_v = 50, mixed precision (float q/p/F, double eps).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on a bounded sub-box sample of the
same workload (same density and parameters). Under torchrun every rank runs
its own independent replica of the workload (weak scaling); rank 0 prints one
JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s at N=4M on 1 GB300 (mixed vs FP64) at stated energy drift"
UNIT = "particle-steps/s"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(values, world: int, device="cuda"):
    """Elementwise maximum of per-rank scalars over all ranks of the process
    group (the slowest rank sets a time); the values themselves at world = 1."""
    if world == 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as tdist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def whole_job_rate(n_per_rank: int, world: int, steps: int, seconds: float) -> float:
    """Particle-steps per second of the whole job: every rank advances its
    own n_per_rank particles (weak scaling) in the slowest rank's time."""
    return n_per_rank * world * steps / seconds


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"dpde_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.dev)], stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            self.proc.wait(timeout=10)
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return None
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        if not rows:
            return None
        try:
            sm = [float(r[1]) for r in rows]
            smax = max(float(r[2]) for r in rows)
        except ValueError:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        loaded = [x for x in sm if x > 0.5 * smax] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows)}


def workload_and_scheme(args):
    from paper_1507_06643_gb300 import inputs
    w = inputs.WORKLOADS[args.workload](args.precision)
    if args.bricks:
        b = tuple(int(x) for x in args.bricks.split(","))
        b = b * 3 if len(b) == 1 else b
        w.replicas = [inputs.ReplicaSpec(r.n, r.box, r.cv, r.kT, b, r.vz_split) for r in w.replicas]
    return w


# Lane operations per unique pair (counted from the kernels' formulas; see
# the roofline section of the design notes): one Gaussian triple = Philox4x32-10
# (~80 INT) + Box-Muller (~100: 2 log, 2 sqrt, sincospi, cospi, scaling);
# SSA pair map ~95 (one expm1, one rsqrt, momenta, dK, two compensated eps
# updates, two fast beta divisions); SER sweep 1 ~40, sweep 2 ~55 pair arithmetic.
OPS_GAUSS = 180.0
OPS_FORCE = 20.0    # one pair force of the soft repulsion (one rsqrt, products, sums)
OPS_PER_PAIR = {"ssa": 95.0, "ssa_gauss": OPS_GAUSS, "sweep1": OPS_GAUSS + 40.0, "sweep2": OPS_GAUSS + 55.0}
# the SSA by dependency levels (ssa_mode 2) draws each pair's Gaussian in its
# execution kernel; its "ssa_gauss" phase is the level schedule, which has no
# algorithmic operations of its own (it orders the pairs)
OPS_PER_PAIR_LEVELS = {"ssa": 95.0 + OPS_GAUSS}
KERNEL_OF_PHASE = {"ssa": "k_ssa_colour", "ssa_gauss": "k_ssa_gauss", "sweep1": "k_ser_sweep1",
                   "sweep2": "k_ser_sweep2", "force": "k_force_tile", "gather": "k_rank_gather",
                   "kick_drift": "k_kick_drift_key"}

# DRAM bytes (read + write) per launch of a kernel from an ncu capture of the
# named configuration with the caches kept warm
# (profiles/launches_large_n4m_hybrid_mixed.md); reported only for that
# configuration and kernel.
MEASURED_TRAFFIC = {("large_n4m", "HYBRID", "mixed", "k_ssa_colour", 5): 168.6e6,
                    # k_force_tile: 286.7 MB per launch on medium_n1m at tile edge 5 and
                    # 276.8 MB at edge 6, scaled to 4M particles (traffic grows with the
                    # particle count)
                    ("large_n4m", "HYBRID", "mixed", "k_force_tile", 5): 4.0 * 286.7e6,
                    ("large_n4m", "HYBRID", "mixed", "k_force_tile", 6): 4.0 * 276.8e6}


def pair_counts(w):
    """Unique pairs per step of the workload at uniform density: all pairs,
    and those inside one brick (pairs uniform in the cutoff sphere have
    E|dx_d| = 3 r_c / 8, so a pair crosses a brick face along d with
    probability ~ 3 r_c / (8 b_d) for brick side b_d)."""
    total = intra = 0.0
    for r in w.replicas:
        rho = r.n / (r.box[0] * r.box[1] * r.box[2])
        pairs = r.n * 0.5 * (4.0 / 3.0) * math.pi * rho * w.r_cut ** 3
        f = 1.0
        for d in range(3):
            b = r.box[d] / r.bricks[d]
            f *= max(0.0, 1.0 - 0.375 * w.r_cut / b) if r.bricks[d] > 1 else 1.0
        total += pairs
        intra += pairs * f
    return total, intra


def algorithmic_model(w, phase: str, scheme: str, precision: str, ssa_mode: int = 0):
    """Algorithmic work of a phase in one step: unique pairs x lane
    operations per pair for the SSA and SER phases (ALU-bound), bytes for the
    memory-bound sort / force phases."""
    n = w.n_total
    total, intra = pair_counts(w)
    pairs = {"ssa": intra if scheme == "HYBRID" else total,
             "sweep1": total - intra if scheme == "HYBRID" else total}
    pairs["ssa_gauss"] = pairs["ssa"]
    pairs["sweep2"] = pairs["sweep1"]
    state_bytes = 16 if precision == "mixed" else 32
    if ssa_mode == 2 and phase in OPS_PER_PAIR_LEVELS:
        return "alu", pairs[phase] * OPS_PER_PAIR_LEVELS[phase], "Gop/s"
    if phase in OPS_PER_PAIR:
        return "alu", pairs[phase] * OPS_PER_PAIR[phase], "Gop/s"
    if phase == "force":
        return "hbm", n * (state_bytes * 4.0), "GB/s"
    return "hbm", n * (state_bytes * 4.0 + 8 * 2 + 12), "GB/s"


def step_roofline(w, scheme, ms_step, peaks, peak_src):
    """The whole step against its modelled bound: the larger of the
    algorithmic bytes (the mixed state read and written once, 68 B per
    particle; 116 B in FP64) over the HBM peak and the algorithmic lane
    operations (per unique pair one Gaussian triple, the force, and the SSA
    map or the SER pair arithmetic of both sweeps) over the ALU peak."""
    n = w.n_total
    total, intra = pair_counts(w)
    fd = OPS_PER_PAIR["ssa"] if scheme in ("HYBRID", "SSA") else 0.0
    ser = OPS_PER_PAIR["sweep1"] - OPS_GAUSS + OPS_PER_PAIR["sweep2"] - OPS_GAUSS
    if scheme == "HYBRID":
        ops = total * (OPS_GAUSS + OPS_FORCE) + intra * fd + (total - intra) * ser
    elif scheme == "SSA":
        ops = total * (OPS_GAUSS + OPS_FORCE + fd)
    else:
        ops = total * (OPS_GAUSS + OPS_FORCE + ser)
    nbytes = n * (68.0 if w.precision == "mixed" else 116.0)
    clk_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    alu = 152 * 128 * clk_mhz * 1e6
    hbm = float(peaks["hbm_gbs"]) * 1e9
    model_s = max(nbytes / hbm, ops / alu)
    return {"bound": "alu" if ops / alu >= nbytes / hbm else "hbm", "model_us": model_s * 1e6,
            "measured_us": ms_step * 1e3, "frac": model_s / (ms_step / 1e3),
            "ops_per_particle": ops / n, "bytes_per_particle": nbytes / n,
            "peak_source": f"{peak_src} hbm_gbs; 152 SMs x 128 lanes x {clk_mhz:.0f} MHz"}


def run_ours(args):
    import torch
    import torch.distributed as tdist
    from paper_1507_06643_gb300 import dpde, inputs

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = workload_and_scheme(args)
    spec_reps = [dpde.make_replica(s.n, s.box, s.cv, s.bricks, s.walls, s.wall_u) for s in w.replicas]
    prm = dpde.make_params(w.mass, w.r_cut, w.a, w.sigma, w.seed + 7919 * rank, w.precision)
    q, p, e = inputs.workload_state(w, seed=w.seed + rank)
    stream = torch.cuda.Stream()
    S = dpde.System(prm, spec_reps, stream=stream.cuda_stream)
    S.set_state(q, p, e)
    dt = w.dt
    # tune on a relaxed state: the first steps from the random start differ
    S.step(args.warmup, dt, args.scheme)
    tuning = S.autotune(args.scheme, dt, 10) if not args.no_autotune else S.tuning()
    if args.ssa_mode is not None or args.ssa_group is not None or args.tile_edge is not None:
        S.set_tuning(ssa_mode=args.ssa_mode, ssa_group=args.ssa_group, tile_edge=args.tile_edge)
        tuning = S.tuning()
    obs0 = S.observables()

    S.step(args.warmup, dt, args.scheme)
    assert S.sync() == dpde.DPDE_OK
    if world > 1:
        tdist.barrier()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        t0.record(stream)
        S.step(args.steps, dt, args.scheme)
        t1.record(stream)
        t1.synchronize()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    status = S.sync()
    ms = max_over_ranks([ms], world)[0]
    if world > 1:
        tdist.barrier()
    obs1 = S.observables()
    n_tot = w.n_total
    value = whole_job_rate(n_tot, world, args.steps, ms / 1e3)

    # per-phase kernel times (CUDA events on the launching stream, eager launches)
    phases = S.step_profiled(args.profile_steps, dt, args.scheme)
    phase_avg = {k: v / args.profile_steps for k, v in phases.items()}
    dom = max(phase_avg, key=phase_avg.get)

    # end to end through the C ABI with pinned host buffers
    qh = torch.from_numpy(q).pin_memory()
    ph = torch.from_numpy(p).pin_memory()
    eh = torch.from_numpy(e).pin_memory()
    S2 = dpde.System(prm, spec_reps, stream=stream.cuda_stream)
    S2.set_tuning(**{k: tuning[k] for k in ("tile_edge", "block", "ssa_block", "ssa_mode", "ssa_group")})
    e2e_steps = args.e2e_steps
    S2.set_state(qh, ph, eh)
    torch.cuda.synchronize()
    tt = time.perf_counter()
    for _ in range(e2e_steps):
        try:
            dpde.dpde_set_state(S2.h, qh, ph, eh, 0, False)
        except dpde.DPDEError as err:   # input with eps <= 0: loaded and reported
            if err.code != dpde.DPDE_ERR_NEG_EPS:
                raise
        S2.step(1, dt, args.scheme)
        rc = dpde.dpde_get_state(S2.h, qh, ph, eh, False)
        # a negative internal energy is a reported outcome of the scheme
        # (state still advanced); anything else stops the run
        if rc not in (dpde.DPDE_OK, dpde.DPDE_ERR_NEG_EPS):
            raise RuntimeError(f"end-to-end step failed: {rc} {dpde.lib().dpde_last_error(S2.h).decode()}")
    e2e_s = max_over_ranks([time.perf_counter() - tt], world)[0]
    e2e_status = rc
    S2.close()
    e2e = {"value": whole_job_rate(n_tot, world, e2e_steps, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": int(q.nbytes + p.nbytes + e.nbytes),
           "d2h_bytes_per_step": int(q.nbytes + p.nbytes + e.nbytes), "status": e2e_status}

    peaks, peak_src = measured_peaks()
    mode = tuning.get("ssa_mode")

    def phase_roofline(ph, secs=None):
        bound, work, unit = algorithmic_model(w, ph, args.scheme, w.precision, mode)
        t = (phase_avg[ph] / 1e3) if secs is None else secs
        achieved = work / t / 1e9
        if bound == "alu":
            clk_mhz = float(peaks.get("sm_max_mhz", 2070.0))
            peak = 152 * 128 * clk_mhz * 1e6 / 1e9   # FP32/INT32 lane-ops per second (G)
            peak_note = f"152 SMs x 128 FP32/INT32 lanes x {clk_mhz:.0f} MHz ({peak_src} clock)"
        else:
            peak = float(peaks["hbm_gbs"])
            peak_note = f"{peak_src} hbm_gbs"
        kernel = KERNEL_OF_PHASE.get(ph, ph)
        if ph == "ssa" and args.scheme == "HYBRID" and mode == 1:
            kernel = "k_ssa_domains"
        if mode == 2 and ph in ("ssa", "ssa_gauss"):
            kernel = {"ssa": "k_ssa_exec", "ssa_gauss": "k_ssa_sched"}[ph]
        if mode == 3 and ph == "ssa":
            kernel = "k_ssa_persistent"
        traffic = None if args.bricks else MEASURED_TRAFFIC.get((w.name, args.scheme, w.precision, kernel,
                                                                tuning.get("tile_edge")))
        return {"bound": bound, "kernel": kernel, "phase": ph, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak, "traffic": traffic, "traffic_unit": "bytes per launch",
                "peak_source": peak_note}

    roofline = phase_roofline(dom)
    roofline_phases = {ph: phase_roofline(ph) for ph in ("force", "ssa", "sweep1", "sweep2")
                       if phase_avg.get(ph, 0) > 0}
    if mode == 2 and args.scheme in ("HYBRID", "SSA"):
        # the whole SSA part: the level schedule counted as overhead of the execution
        r = phase_roofline("ssa", (phase_avg["ssa"] + phase_avg["ssa_gauss"]) / 1e3)
        r.update({"kernel": "k_ssa_sched + k_ssa_exec", "phase": "ssa_gauss + ssa"})
        roofline_phases["ssa_with_schedule"] = r
    roofline_step = step_roofline(w, args.scheme, ms / args.steps, peaks, peak_src)

    drift = abs(obs1[0]["E"] - obs0[0]["E"]) / abs(obs0[0]["E"])
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if w.precision == "mixed" else "f64",
        "data": "synthetic: uniform positions, Maxwellian momenta (kT=1), eps = C_v kT (1 +- 5%)",
        "config": {"workload": w.name, "n": n_tot, "scheme": args.scheme, "precision": w.precision,
                   "pairs_per_particle": pair_counts(w)[0] / n_tot,
                   "ssa_pair_fraction": pair_counts(w)[1] / pair_counts(w)[0] if args.scheme == "HYBRID" else None,
                   "dt": dt, "bricks": list(w.replicas[0].bricks), "l2": "inputs larger than L2 "
                   f"(state ~{n_tot * (48 if w.precision == 'mixed' else 104) / 1e6:.0f} MB)",
                   "parallelism": f"replicas x{world}",
                   "tuning": {k: tuning[k] for k in ("tile_edge", "block", "ssa_block", "ssa_mode", "ssa_group")},
                   "autotuned": not args.no_autotune},
        "e2e": e2e,
        "gpu_launches": None,
        "roofline": roofline,
        "roofline_phases": roofline_phases,
        "roofline_step": roofline_step,
        "phase_ms": phase_avg,
        "energy_transient": {"rel_change_over_timed_steps": drift, "after_steps": 2 * args.warmup,
                             "status": status,
                             "note": "from an unrelaxed uniform-random start: the overlap energy relaxing, "
                                     "not the scheme's drift; the stated drift is energy_drift (relaxed 108k "
                                     "fluid)"},
    }
    nlaunch = S.step_launches(args.scheme)
    out["gpu_launches"] = nlaunch * args.steps
    S.close()
    if args.fp64_steps > 0 and w.precision == "mixed":
        f64 = fp64_run(args, spec_reps, w, q, p, e, stream)
        out["fp64_gpu"] = f64
        out["speedup_mixed_over_fp64"] = value / (f64["value"] * world)
    if args.drift_steps > 0:
        out["energy_drift"] = drift_run(args, stream)
    if args.shock_steps > 0:
        out["shock"] = shock_run(args, stream)
    if args.batched_steps > 0:
        out["batched"] = batched_run(args, stream)
    if rank == 0:
        out["clocks"] = clk.summary()
        if not args.no_cpu_baseline and world == 1:
            out["cpu_baseline"], base = cpu_baseline(w, args.scheme, args.cpu_seconds)
            out["parity"] = parity_report(w, base, args.scheme)
            if args.batched_steps > 0:
                out["cpu_baseline_batched"] = cpu_batched_baseline()
        print(json.dumps(out))
    if world > 1:
        tdist.destroy_process_group()


def fp64_run(args, spec_reps, w, q, p, e, stream):
    """The same workload and scheme with every quantity in double."""
    import torch
    from paper_1507_06643_gb300 import dpde
    prm = dpde.make_params(w.mass, w.r_cut, w.a, w.sigma, w.seed, "fp64")
    S = dpde.System(prm, spec_reps, stream=stream.cuda_stream)
    S.set_state(q, p, e)
    S.step(3, w.dt, args.scheme)
    assert S.sync() == dpde.DPDE_OK
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    S.step(args.fp64_steps, w.dt, args.scheme)
    t1.record(stream)
    t1.synchronize()
    ms = t0.elapsed_time(t1)
    S.close()
    return {"value": w.n_total * args.fp64_steps / (ms / 1e3), "unit": UNIT, "steps": args.fp64_steps,
            "warmup": 3, "ms_per_step": ms / args.fp64_steps, "dtype": "f64"}


def _energy_series(S, steps, dt, scheme, every):
    """E sampled every `every` steps over `steps` steps (E^0 first), with the
    mean kinetic and internal temperatures over the samples."""
    o = S.observables(check=True)[0]
    Es, tk, ti = [o["E"]], [], []
    done = 0
    while done < steps:
        k = min(every, steps - done)
        S.step(k, dt, scheme)
        done += k
        o = S.observables(check=True)[0]
        Es.append(o["E"])
        tk.append(o["Tkin"])
        ti.append(o["Tint"])
    return np.asarray(Es), float(np.mean(tk)), float(np.mean(ti))


def drift_run(args, stream):
    """Total-energy drift on the N=108,000 equilibrium fluid (Sec. IV.B).

    The fluid is relaxed first (Hybrid at dt = 0.01); from that one state
    both precisions then run at the drift timestep with the same noise: the
    mixed mode for --drift-steps, FP64 for --drift-steps-fp64. Reported:
    max_n |E^n - E^0| / |E^0| and the fitted drift rate of each run, and the
    precision-induced part max |(E_m^n - E_m^0) - (E_f^n - E_f^0)| / |E^0|
    over the steps both ran. At dt = 0.0035 the scheme's own drift (rate
    ~ dt^4, Sec. IV.B) over 1e5 steps is expected below 1e-6."""
    from paper_1507_06643_gb300 import dpde, inputs
    dt = args.drift_dt
    steps = {"mixed": args.drift_steps, "fp64": args.drift_steps_fp64 or args.drift_steps}
    out = {"workload": "equilibrium_n108000", "scheme": args.scheme, "equilibration_steps": args.drift_equil,
           "equilibration_dt": 0.01, "dt": dt, "steps": steps}
    w = inputs.equilibrium_n108000("mixed")
    reps = [dpde.make_replica(x.n, x.box, x.cv, x.bricks, x.walls, x.wall_u) for x in w.replicas]
    q, p, e = inputs.workload_state(w)
    R = dpde.System(dpde.make_params(w.mass, w.r_cut, w.a, w.sigma, w.seed, "mixed"), reps, stream=stream.cuda_stream)
    R.set_state(q, p, e)
    R.step(args.drift_equil, 0.01, args.scheme)
    q, p, e = R.get_state()
    R.close()
    every = max(1, min(1000, min(steps.values()) // 20))
    series = {}
    for prec in ("mixed", "fp64"):
        S = dpde.System(dpde.make_params(w.mass, w.r_cut, w.a, w.sigma, w.seed + 1, prec), reps,
                        stream=stream.cuda_stream)
        S.set_state(q, p, e)
        t = time.perf_counter()
        Es, tk, ti = _energy_series(S, steps[prec], dt, args.scheme, every)
        el = time.perf_counter() - t
        S.close()
        rel = (Es - Es[0]) / abs(Es[0])
        tt = np.arange(len(Es)) * every * dt
        out[prec] = {"max_rel_drift": float(np.max(np.abs(rel))), "final_rel_drift": float(abs(rel[-1])),
                     "alpha_per_unit_time": float(np.polyfit(tt, rel, 1)[0]) if len(Es) > 2 else None,
                     "mean_Tkin": tk, "mean_Tint": ti, "wall_s": el, "steps": steps[prec]}
        series[prec] = Es
    n = min(len(series["mixed"]), len(series["fp64"]))
    em, ef = series["mixed"][:n], series["fp64"][:n]
    out["max_rel_drift_mixed_minus_fp64"] = float(np.max(np.abs((em - em[0]) - (ef - ef[0]))) / abs(ef[0]))
    out["common_steps"] = (n - 1) * every
    out["sample_every"] = every
    out["bar"] = {"rel_drift": 1e-6, "steps": 100000,
                  "mixed_meets_bar": bool(out["mixed"]["max_rel_drift"] < 1e-6 and steps["mixed"] >= 100000)}
    return out


def shock_run(args, stream):
    """The shock workload (BASELINE config 4: box 40 x 40 x 800 at density 3,
    halves at +-2 along z, C_v = 100, dt = 0.005, mixed precision, Hybrid):
    throughput, total-energy drift over --shock-steps steps, and the mean
    internal energy in 800 slabs along z at the start, halfway and at the
    end (the analogue of the eps profiles of Sec. V)."""
    import torch
    from paper_1507_06643_gb300 import dpde, inputs
    w = inputs.shock_40x40x800("mixed")
    spec = w.replicas[0]
    reps = [dpde.make_replica(spec.n, spec.box, spec.cv, spec.bricks, spec.walls, spec.wall_u)]
    S = dpde.System(dpde.make_params(w.mass, w.r_cut, w.a, w.sigma, w.seed, "mixed"), reps, stream=stream.cuda_stream)
    q, p, e = inputs.workload_state(w)
    S.set_state(q, p, e)
    S.step(3, w.dt, "HYBRID")
    S.sync()
    nsl = 800
    Lz = spec.box[2]

    def profile():
        qq, _, ee = S.get_state()
        idx = np.minimum((qq[:, 2] / Lz * nsl).astype(np.int64), nsl - 1)
        cnt = np.bincount(idx, minlength=nsl)
        return np.bincount(idx, weights=ee, minlength=nsl) / np.maximum(cnt, 1)

    o0 = S.observables(check=False)[0]
    prof = {"t0": profile()}
    half = args.shock_steps // 2
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    S.step(half, w.dt, "HYBRID")
    t1.record(stream)
    t1.synchronize()
    ms = t0.elapsed_time(t1)
    prof["half"] = profile()
    S.step(args.shock_steps - half, w.dt, "HYBRID")
    status = S.sync()
    o1 = S.observables(check=False)[0]
    prof["end"] = profile()
    S.close()
    return {"workload": w.name, "n": spec.n, "dt": w.dt, "steps": args.shock_steps, "scheme": "HYBRID",
            "precision": "mixed", "value": spec.n * half / (ms / 1e3), "unit": UNIT, "timed_steps": half,
            "ms_per_step": ms / half, "rel_drift": abs(o1["E"] - o0["E"]) / abs(o0["E"]), "status": status,
            "neg_eps": o1["neg_eps"], "eps_profile": {"slabs": nsl, "slab_width": Lz / nsl,
                                                      "times": [0.0, half * w.dt, args.shock_steps * w.dt],
                                                      **{k: [round(float(x), 3) for x in v] for k, v in prof.items()}}}


def batched_run(args, stream):
    """The batched workload (BASELINE config 5: 256 systems of 2,000-64,000
    particles, kT in [0.5, 2], C_v in {10, 50, 100}, mixed, Hybrid): all
    replicas advance in the same launches; throughput and the largest
    relative energy change of a replica over the timed steps."""
    import torch
    from paper_1507_06643_gb300 import dpde, inputs
    w = inputs.batched_256("mixed")
    reps = [dpde.make_replica(x.n, x.box, x.cv, x.bricks, x.walls, x.wall_u) for x in w.replicas]
    S = dpde.System(dpde.make_params(w.mass, w.r_cut, w.a, w.sigma, w.seed, "mixed"), reps, stream=stream.cuda_stream)
    q, p, e = inputs.workload_state(w)
    S.set_state(q, p, e)
    S.step(200, w.dt, "HYBRID")
    S.sync()
    tuning = S.autotune("HYBRID", w.dt, 5)
    o0 = S.observables(check=False)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    S.step(args.batched_steps, w.dt, "HYBRID")
    t1.record(stream)
    t1.synchronize()
    ms = t0.elapsed_time(t1)
    status = S.sync()
    o1 = S.observables(check=False)
    launches = S.step_launches("HYBRID")
    S.close()
    drift = max(abs(b["E"] - a["E"]) / abs(a["E"]) for a, b in zip(o0, o1))
    return {"workload": w.name, "replicas": len(reps), "n": w.n_total, "dt": w.dt, "steps": args.batched_steps,
            "value": w.n_total * args.batched_steps / (ms / 1e3), "unit": UNIT,
            "ms_per_step": ms / args.batched_steps, "launches_per_step": launches,
            "max_replica_rel_drift": drift, "after_steps": 200, "status": status,
            "neg_eps_replicas": int(sum(1 for o in o1 if o["neg_eps"] > 0)),
            "tuning": {k: tuning[k] for k in ("tile_edge", "block", "ssa_block", "ssa_mode", "ssa_group")}}


def oracle_sample(w, n_target: int):
    """A cubic sub-box of the workload at the same density and parameters."""
    from paper_1507_06643_gb300 import inputs
    spec = w.replicas[0]
    vol = spec.box[0] * spec.box[1] * spec.box[2]
    rho = spec.n / vol
    n = max(1000, min(spec.n, int(n_target)))
    L = (n / rho) ** (1 / 3)
    cells_per_brick = 6
    b = max(1, int(L // cells_per_brick)) if spec.bricks != (1, 1, 1) else 1
    while b > 1 and math.floor(L / b) * b < 3:
        b -= 1
    sub = inputs.Workload(w.name + "_sample", [inputs.ReplicaSpec(n, (L, L, L), spec.cv, spec.kT, (b, b, b),
                                                                  spec.vz_split, spec.vz_shift, spec.walls,
                                                                  spec.wall_u)],
                          w.mass, w.r_cut, w.a, w.sigma, w.dt, 1, w.seed, "fp64")
    return sub


def host_cpu():
    """Core count and CPU model of the host the oracle runs on."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu part")):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"nproc": os.cpu_count(), "model": model or "unknown"}


def _oracle_replica_rate(job):
    """One replica advanced by the oracle in a worker process: returns
    (particles, steps, seconds)."""
    from oracle import oracle as O
    n, box, cv, kT, bricks, seed, steps, dt = job
    from paper_1507_06643_gb300 import inputs
    spec = inputs.ReplicaSpec(n, box, cv, kT, bricks)
    q, p, e = inputs.replica_state(spec, 1.0, np.random.default_rng(seed))
    S = O.System([O.make_replica(n, box, cv, bricks)], O.make_params(seed=seed), q, p, e)
    t = time.perf_counter()
    S.run(steps, dt, "HYBRID")
    return n, steps, time.perf_counter() - t


def cpu_batched_baseline(nrep_per_core: int = 3, steps: int = 3):
    """The oracle on the batched workload across all host cores: replicas of
    batched_256 (independent systems) spread over a process pool (spawn),
    one replica per task. Aggregate particle-steps/s = sum n_r steps /
    wall time of the pool."""
    import multiprocessing as mp
    from paper_1507_06643_gb300 import inputs
    cores = os.cpu_count() or 1
    w = inputs.batched_256("fp64")
    jobs = [(r.n, r.box, r.cv, r.kT, r.bricks, 2000 + k, steps, w.dt)
            for k, r in enumerate(w.replicas[: nrep_per_core * cores])]
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_replica_rate, jobs[:cores])          # warm the workers (imports, build)
        t = time.perf_counter()
        res = pool.map(_oracle_replica_rate, jobs)
        el = time.perf_counter() - t
    n_ps = sum(n * k for n, k, _ in res)
    return {"value": n_ps / el, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": host_cpu(),
            "sample": f"{len(jobs)} replicas of batched_256 ({sum(n for n, _, _ in res)} particles), {steps} "
                      f"Hybrid steps each, FP64 oracle, one replica per task on a {cores}-process pool, "
                      f"{el:.1f} s"}


def cpu_baseline(w, scheme: str, seconds: float, steps: int | None = None):
    from oracle import oracle as O
    from paper_1507_06643_gb300 import inputs
    rate_guess = 6.0e4
    n_target = seconds * rate_guess if steps is None else seconds * rate_guess / steps
    sub = oracle_sample(w, n_target)
    spec = sub.replicas[0]
    q, p, e = inputs.workload_state(sub, float32=False)
    S = O.System([O.make_replica(spec.n, spec.box, spec.cv, spec.bricks, spec.walls, spec.wall_u)],
                 O.make_params(sub.mass, sub.r_cut, sub.a, sub.sigma, sub.seed), q, p, e)
    nsteps = steps or 1
    t = time.perf_counter()
    S.run(nsteps, sub.dt, scheme)
    el = time.perf_counter() - t
    out = {"value": spec.n * nsteps / el, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu": host_cpu(),
           "sample": f"{nsteps} step(s) of a {spec.n}-particle cubic sub-box of {w.name} "
                     f"(same density and parameters, FP64, {scheme}, bricks {spec.bricks}), "
                     f"{el:.1f} s"}
    return out, (sub, q, p, e, S, nsteps)


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _gpu_vs_oracle(sub, q, p, e, ref, nsteps, scheme, precision):
    """Largest relative difference (q by minimum image, p, eps) between the
    library and the oracle after the same steps from the same state."""
    from paper_1507_06643_gb300 import dpde
    spec = sub.replicas[0]
    G = dpde.System(dpde.make_params(sub.mass, sub.r_cut, sub.a, sub.sigma, sub.seed, precision),
                    [dpde.make_replica(spec.n, spec.box, spec.cv, spec.bricks, spec.walls, spec.wall_u)])
    G.set_state(q, p, e)
    G.step(nsteps, sub.dt, scheme, use_graph=False)
    qg, pg, eg = G.get_state()
    G.close()
    L = np.asarray(spec.box, float)
    dq = qg - ref.q
    dq -= L * np.round(dq / L)
    moved = ref.q - q                      # the oracle's displacement from the start (minimum image)
    moved -= L * np.round(moved / L)
    return max(float(np.max(np.abs(dq)) / np.max(np.abs(moved))), _rel(pg, ref.p), _rel(eg, ref.eps))


def parity_report(w, base, scheme):
    """Parity of the GPU path against the oracle on the baseline's sub-box: FP64
    with the bench's scheme (the same oracle run the baseline timed), and the
    mixed mode with SER on a smaller sub-box (SER's result does not depend on
    cell binning, so float/double binning differences cannot enter)."""
    from oracle import oracle as O
    from paper_1507_06643_gb300 import inputs
    sub, q, p, e, ref, nsteps = base
    out = {"tolerance": {"fp64": 1e-11, "mixed": 2e-5}}
    out["fp64"] = _gpu_vs_oracle(sub, q, p, e, ref, nsteps, scheme, "fp64")
    out["fp64_scheme"] = scheme
    small = oracle_sample(w, 60000)
    spec = small.replicas[0]
    q2, p2, e2 = inputs.workload_state(small, float32=True)
    ref2 = O.System([O.make_replica(spec.n, spec.box, spec.cv, spec.bricks, spec.walls, spec.wall_u)],
                    O.make_params(small.mass, small.r_cut, small.a, small.sigma, small.seed), q2, p2, e2)
    ref2.run(2, small.dt, "SER")
    out["mixed_ser"] = _gpu_vs_oracle(small, q2, p2, e2, ref2, 2, "SER", "mixed")
    out["mixed_hybrid"] = _mixed_hybrid_parity(small, q2, p2, e2)
    out["sample"] = (f"fp64: {nsteps} step(s) of the {sub.replicas[0].n}-particle sub-box above; mixed: 2 SER steps "
                     f"and 1 Hybrid step of a {spec.n}-particle sub-box (float-rounded input on both sides)")
    return out


def _mixed_hybrid_parity(sub, q, p, e):
    """One mixed-precision Hybrid step against the oracle. The library bins
    float positions, the oracle double ones, so a particle within rounding of
    a cell face may sit in different cells on the two sides, which changes
    the SSA order around it: particles within 2 r_cut of such a particle are
    left out (their fraction is reported), the rest compared element by
    element (q by the displacement from the start)."""
    from scipy.spatial import cKDTree
    from oracle import oracle as O
    from paper_1507_06643_gb300 import dpde
    spec = sub.replicas[0]
    rep = O.make_replica(spec.n, spec.box, spec.cv, spec.bricks, spec.walls, spec.wall_u)
    ref = O.System([rep], O.make_params(sub.mass, sub.r_cut, sub.a, sub.sigma, sub.seed), q, p, e)
    ref.run(1, sub.dt, "HYBRID")
    G = dpde.System(dpde.make_params(sub.mass, sub.r_cut, sub.a, sub.sigma, sub.seed, "mixed"),
                    [dpde.make_replica(spec.n, spec.box, spec.cv, spec.bricks, spec.walls, spec.wall_u)])
    G.set_state(q, p, e)
    G.step(1, sub.dt, "HYBRID", use_graph=False)
    cells = G.get_cells()
    qg, pg, eg = G.get_state()
    G.close()
    box = np.asarray(spec.box, float)
    nc, _ = O.cell_grid(rep, sub.r_cut)
    oc = np.empty(ref.q.shape, np.int64)
    for d in range(3):
        oc[:, d] = np.minimum(nc[d] - 1, np.maximum(0, np.trunc(ref.q[:, d] * (nc[d] / box[d])).astype(np.int64)))
    flips = np.nonzero(np.any(cells != oc, axis=1))[0]
    keep = np.ones(spec.n, bool)
    if len(flips):
        tree = cKDTree(np.mod(ref.q, box), boxsize=box)
        for lst in tree.query_ball_point(np.mod(ref.q[flips], box), 2.0 * sub.r_cut):
            keep[lst] = False
    dq = qg - ref.q
    dq -= box * np.round(dq / box)
    moved = ref.q - q
    moved -= box * np.round(moved / box)
    if not keep.any():
        return {"err": None, "flipped": int(len(flips)), "excluded_fraction": 1.0}
    err = max(float(np.max(np.abs(dq[keep])) / np.max(np.abs(moved))), _rel(pg[keep], ref.p[keep]),
              _rel(eg[keep], ref.eps[keep]))
    return {"err": err, "flipped": int(len(flips)), "excluded_fraction": float(1.0 - keep.mean())}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = workload_and_scheme(args)
    from oracle import oracle as O
    from paper_1507_06643_gb300 import inputs
    total = args.steps + args.warmup
    n_target = max(2000, 150.0 * 6.0e4 / max(total, 1))
    sub = oracle_sample(w, n_target)
    spec = sub.replicas[0]
    q, p, e = inputs.workload_state(sub, float32=False)
    S = O.System([O.make_replica(spec.n, spec.box, spec.cv, spec.bricks, spec.walls, spec.wall_u)],
                 O.make_params(sub.mass, sub.r_cut, sub.a, sub.sigma, sub.seed), q, p, e)
    S.run(args.warmup, sub.dt, args.scheme)
    t = time.perf_counter()
    S.run(args.steps, sub.dt, args.scheme)
    el = time.perf_counter() - t
    value = spec.n * args.steps / el
    sample = (f"{spec.n}-particle cubic sub-box of {w.name} (same density and parameters), FP64 "
              f"oracle, {args.scheme}, {args.steps} timed steps after {args.warmup}")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / max(args.steps, 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": w.name, "scheme": args.scheme,
                                           "precision": "fp64", "sample_n": spec.n},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu": host_cpu(),
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large_n4m")
    ap.add_argument("--scheme", default="HYBRID", choices=["SER", "HYBRID", "SEM", "SSA"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--profile-steps", type=int, default=10)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--ssa-mode", type=int, choices=(0, 1, 2, 3), default=None,
                    help="force the SSA launch form: 0 one launch per colour class, 1 one launch over "
                         "whole Hybrid domains, 2 by dependency levels (schedule + execution), 3 the "
                         "colour classes in one persistent launch")
    ap.add_argument("--tile-edge", type=int, default=None, help="force the force pass's tile edge (cells)")
    ap.add_argument("--ssa-group", type=int, default=None, help="force the Hybrid domains per warp (1..8)")
    ap.add_argument("--fp64-steps", type=int, default=20,
                    help="steps of the FP64 GPU run of the same workload (0: skip)")
    ap.add_argument("--drift-steps", type=int, default=100000,
                    help="steps of the mixed-precision energy-drift run on the 108k fluid (0: skip)")
    ap.add_argument("--drift-steps-fp64", type=int, default=20000,
                    help="steps of the FP64 run of the drift study (0: as many as the mixed run)")
    ap.add_argument("--drift-dt", type=float, default=0.0035)
    ap.add_argument("--drift-equil", type=int, default=2000)
    ap.add_argument("--shock-steps", type=int, default=20000,
                    help="steps of the shock leg (40 x 40 x 800 box; 0: skip)")
    ap.add_argument("--batched-steps", type=int, default=1000,
                    help="timed steps of the batched leg (256 replicas; 0: skip)")
    ap.add_argument("--drift-only", action="store_true",
                    help="run only the energy-drift study and print its JSON")
    ap.add_argument("--bricks", default="",
                    help="override the Hybrid brick grid: B or Bx,By,Bz")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
    elif args.drift_only:
        import torch
        stream = torch.cuda.Stream()
        print(json.dumps({"energy_drift": drift_run(args, stream)}))
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
