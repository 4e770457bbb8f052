#!/usr/bin/env python3
"""Throughput of the 1D3V PIC Monte Carlo step on GB300: particle-steps/s and HBM roofline.

Default workload: the non-uniform-load case (65536 cells, 100,007,936 particles, density
~ exp(-x/(L/8)), pair source, B = 0.5 at 30 degrees, all four collision processes, per-cell
counting sort every 10 steps), FP32 particle path with int64 fixed-point deposit.  A "step" is one
full PIC MC step (gather, push, walls, MCC, deposit, source, Poisson, and the sort on every tenth
step).  Inputs (2.8 GB of particles) are larger than L2, so no flush is needed between steps.

Lines printed (rank 0): one JSON object.  ``--impl reference`` times the plain FP64 CPU oracle
(the CPU reference of this library) on the same workload at full size instead, on the host cores.

With N > 1 processes (torchrun, one per GPU) every rank advances its own replica of the workload
(its own seed, no data-path collective): the value is the particle-steps of all ranks over the
slowest rank's time, and the end-to-end leg runs on every rank.  The single-GPU sections (plain
FP64 path, ensemble, adjoint, sheath, precision, the CPU baseline) run at N = 1 only.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2606_28534_gb300 import workloads as W  # noqa: E402

METRIC = "particle-steps/s & HBM roofline %, FP32/batched vs plain FP64 grid, 1 GB300"
# algorithmic bytes per particle of the ordinary step kernel: cell word, fraction and velocity
# read (20 B) and written (20 B); the id is read only by the ~1 % of particles whose null-collision
# countdown expires (from L2, just written), which is left out
BYTES_STEP_KERNEL = 40
# the plain FP64 path's step (a workload defined in FP64): x, v (32 B) and the countdown (4 B) read
# and written
BYTES_STEP64_KERNEL = 72
# the step after a sort reads and writes each particle with its id, to its sorted slot: 28 + 28 B
BYTES_SCATTER_KERNEL = 56
# DRAM bytes per particle of one launch, from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum) of these kernels on the 50.3M-particle profiling case (c3h, large enough
# for the ordinary step's claimed chunk segments), scaled by particles to a full launch: the
# ordinary step and the step after a sort
TRAFFIC_STEP, TRAFFIC_SCATTER = 42.75, 58.80
# the same for the ensemble's particle step (ncu on a 20-run ensemble of config 4's distribution,
# large enough for its claimed chunk segments)
TRAFFIC_BSTEP = 41.56
# the neutral step reads each neutral (cell, frac, v, id: 28 B) and writes back its cell and fraction
# (8 B); on sort steps it writes each survivor, compacted, into the other buffer instead (28 B)
BYTES_NEUTRAL_KERNEL, BYTES_NEUTRAL_COMPACT = 36, 56
# DRAM bytes per neutral of one in-place neutral launch, from one ncu capture on the sheath profiling
# case (c6p), scaled by neutrals to a full launch (writes still dirty in L2 at the launch's end are
# not counted there)
TRAFFIC_NEUTRAL = 32.33


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------------------------------------
class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.idx)], stdout=open(self.path, "w"),
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [t.strip() for t in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        loaded = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------------------------------------
def oracle_timing(params: dict, steps: int, warmup: int) -> dict:
    """The FP64 oracle as it stands on the workload itself (full size): created once, ``warmup``
    untimed steps, then ``steps`` timed steps on all host cores and one more step on one thread.
    particle-steps/s = the live particles at the start of each timed step over the host time of
    those steps."""
    from oracle import oracle as O

    cores = len(os.sched_getaffinity(0))
    t0 = time.perf_counter()
    sim = O.OracleSim(params, threads=cores)
    t_create = time.perf_counter() - t0
    sim.step(max(1, warmup))  # first touch; step 0 is a sort step
    ps, t = 0, 0.0
    for _ in range(steps):
        ps += sim.count(0) + sim.count(1)  # live particles at the start of the step
        t0 = time.perf_counter()
        sim.step(1)
        t += time.perf_counter() - t0
    O.set_threads(1)
    ps1 = sim.count(0) + sim.count(1)
    t0 = time.perf_counter()
    sim.step(1)
    t1 = time.perf_counter() - t0
    O.set_threads(cores)
    n = sim.count(0) + sim.count(1)
    sim.close()
    return {"value": ps / t, "unit": "particle-steps/s", "cores": cores, "kind": "oracle",
            "sample": (f"the workload itself at full size ({n:,} particles, {params['ncells']} cells): "
                       f"{max(1, warmup)} untimed step(s), then {steps} timed steps on {cores} OpenMP threads "
                       f"({t:.2f} s); set-up {t_create:.1f} s not timed"),
            "steps": steps, "seconds": t,
            "single_thread": {"value": ps1 / t1, "unit": "particle-steps/s", "cores": 1, "steps": 1,
                              "seconds": t1}}


def cpu_baseline(params: dict, steps: int) -> dict:
    """The CPU baseline of the bench line: the oracle on the benchmarked workload, 3 timed steps."""
    return oracle_timing(params, steps, warmup=1)


def run_reference(args, rank: int, world: int) -> None:
    if rank != 0:
        return
    params = W.CONFIGS[args.workload]
    r = oracle_timing(params, args.steps, warmup=min(args.warmup, 5))
    value = r["value"]
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "particle-steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * r["seconds"] / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {W_DESC[args.workload]}"},
        "cpu_baseline": r,
        "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


W_DESC = {
    "c1": "plain PIC MC, 256 cells, 51,200 particles",
    "c2": "uniform load, 4096 cells, 8,192,000 particles, B 0.5 @ 30 deg, 4 processes",
    "c3": "non-uniform load, 65536 cells, 100,007,936 particles, exp(-x/(L/8)) + pair source, "
          "B 0.5 @ 30 deg, 4 processes, sort every 10 steps",
    "c5": "collisionless, 1024 cells, 409,600 particles",
    "c3p": "non-uniform load profiling case, 65536 cells, 12,582,912 particles",
    "c3h": "non-uniform load profiling case, 65536 cells, 50,331,648 particles",
    "c6": "D+/e/D sheath, 65536 cells, 100,007,936 charged + 50,003,968 neutral particles",
    "c6p": "D+/e/D sheath profiling case, 65536 cells, 12,582,912 charged + 6,291,456 neutral particles",
}


# ------------------------------------------------------------------------------------------------
def timed_run(sim, torch, steps: int, profile: bool):
    """K steps on the device between two events on the library's stream (bracketed by syncs)."""
    ps0 = sim.diag()["particle_steps"]
    torch.cuda.synchronize()
    if profile:
        sim.profile(True)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(sim.stream)
    sim.step(steps)
    b.record(sim.stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    kt = None
    if profile:
        kt = sim.kernel_times()
        sim.profile(False)
    ps = sim.diag()["particle_steps"] - ps0
    return ms, ps, kt


def events_ms(torch, stream, fn) -> float:
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def batched(args, torch, pic, peak: float) -> dict:
    """Config 4: 256 independent runs of uneven size in one batch (autotuned launch configuration,
    CUDA graphs), against the same runs advanced one at a time through the single-run API."""
    from paper_2606_28534_gb300 import autotune

    runs = W.c4() if args.batch_sims == W.C4_SIMS else W.ensemble(args.batch_sims)
    K = args.batch_steps
    b = pic.Batch(runs)
    if args.no_tune:
        tune = {"tuning": {"variant": 0, "ctas_per_sm": 0, "use_graph": True}, "cached": False, "trials": []}
    else:
        tune = autotune.tune(b, cache_path=os.path.join(tempfile.gettempdir(), "pic_gb300_tuning.json"))
    b.step(args.warmup)
    b.sync()

    def ps_total():
        return sum(d["particle_steps"] for d in b.diag())

    ps0 = ps_total()
    ms = events_ms(torch, b.stream, lambda: b.step(K))
    b.sync()
    ps = ps_total() - ps0
    # kernel times of whole sort cycles, launched one by one with events (no graphs)
    cyc = 2 * runs[0]["sort_interval"]
    q0 = ps_total()
    b.profile(True)
    b.step(cyc)
    kt = b.kernel_times()
    b.profile(False)
    kps = ps_total() - q0
    b.close()
    del b
    torch.cuda.empty_cache()
    step_ms = kt["step"]["ms"] / max(1, kt["step"]["launches"])
    bytes_per_launch = BYTES_STEP_KERNEL * kps / max(1, kt["step"]["launches"])
    achieved = bytes_per_launch / (step_ms / 1000.0) / 1e9
    # the same runs one at a time (same steps each; device time of the steps only)
    one_ms, one_ps = 0.0, 0
    for p in runs:
        g = pic.Simulation(p)
        g.step(args.warmup)
        g.sync()
        q = g.diag()["particle_steps"]
        one_ms += events_ms(torch, g.stream, lambda: g.step(K))
        one_ps += g.diag()["particle_steps"] - q
        g.close()
    value = ps / (ms / 1000.0)
    one = one_ps / (one_ms / 1000.0)
    return {
        "workload": f"c4: {len(runs)} independent runs, cells U[128, 8192], ppc U[50, 500], "
                    f"nu/omega_p log-U[0.001, 0.1], V_L U[-5, 0], config 2's physics; "
                    f"{sum(2 * p['ncells'] * p['ppc'][0] for p in runs):,} particles",
        "value": value, "unit": "particle-steps/s", "steps": K, "ms_per_step": ms / K,
        "tuning": dict(tune["tuning"], shape=pic.batch_variants()[tune["tuning"]["variant"]],
                       cached=tune["cached"], trials=len(tune["trials"])),
        "one_at_a_time": {"value": one, "unit": "particle-steps/s", "ms_per_step": one_ms / K,
                          "what": "each run alone through pic_init / pic_step, device time of its steps"},
        "speedup_vs_one_at_a_time": value / one,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "kernel": "k_bstep32", "bytes_per_launch": bytes_per_launch,
                     "avg_launch_ms": step_ms,
                     "traffic": TRAFFIC_BSTEP * kps / max(1, kt["step"]["launches"]) if TRAFFIC_BSTEP else None},
        "kernels": {k: {"ms": round(v["ms"], 3), "launches": v["launches"]} for k, v in kt.items()
                    if v["launches"]},
    }


DIAG_FIELDS = ("n", "wall_hits", "coll", "births", "near_threshold", "wall_charge", "net_charge_units",
               "ke", "field_energy", "wall_energy")


def _rel(a, b):
    a, b = np.atleast_1d(np.asarray(a, np.float64)).ravel(), np.atleast_1d(np.asarray(b, np.float64)).ravel()
    d = np.abs(a - b)
    scale = np.maximum(np.abs(b), 1e-300)
    return float((d / scale).max()) if d.any() else 0.0


def precision_section(args, torch, pic) -> dict:
    """The error of each diagnostic against the FP64 oracle: config 2 after 20 steps on the GPU, that
    state given to the oracle, to the FP32 path and to the plain FP64 path, one step of each; the
    relative difference of every pic_diag field (counts: the difference itself)."""
    from oracle import oracle as O

    p = W.C2
    g = pic.Simulation(p)
    g.step(20)
    blob = g.snapshot()  # FP32 values: the same state for all three codes
    g.close()
    del g
    cores = len(os.sched_getaffinity(0))
    o = O.OracleSim(p, threads=cores)
    assert o.restore(blob) == 0
    o.step(1)
    do = o.diag()
    out = {"workload": "c2 (8,192,000 particles) after 20 steps, then one step from the same state",
           "oracle_threads": cores, "fields": {}}
    res = {}
    for name, q in (("fp32", p), ("fp64_plain", W.variant(p, precision=W.PRECISION_FP64_PLAIN))):
        h = pic.Simulation(q)
        if h.restore(blob) != 0:
            raise RuntimeError("restore failed")
        h.step(1)
        res[name] = h.diag()
        h.close()
        del h
        torch.cuda.empty_cache()
    for k in DIAG_FIELDS:
        row = {}
        for name, d in res.items():
            if k in ("ke", "field_energy", "wall_energy"):
                row[name] = _rel(d[k], do[k])
            else:
                row[name] = int(np.abs(np.asarray(d[k], np.int64) - np.asarray(do[k], np.int64)).max())
        out["fields"][k] = row
    out["what"] = ("ke, field_energy, wall_energy: max relative difference; the others: max absolute "
                   "difference of counts (collision and near-threshold counts may differ by the "
                   "near-threshold draws both codes count)")
    return out


def sheath_section(args, torch, pic, peak: float) -> dict:
    """The D+/e/D sheath on config 3's grid (deuterium ions recycled into tracked neutrals at the
    walls, a neutral background of 50 M, their electron-impact ionization, two smoothing passes):
    whole-step throughput over charged and neutral particles, the neutral kernel's roofline, and the
    same plasma without the sheath physics for the cost of adding it."""
    p = W.C6
    K = args.sheath_steps
    g = pic.Simulation(p)
    g.step(args.warmup)
    g.sync()
    d0, n0 = g.diag(), g.neutral_diag()
    ms = events_ms(torch, g.stream, lambda: g.step(K))
    d1, n1 = g.diag(), g.neutral_diag()
    charged = d1["particle_steps"] - d0["particle_steps"]
    neutral = n1["particle_steps"] - n0["particle_steps"]
    # kernel split over two sort cycles, launched with events
    cyc = 2 * p["sort_interval"]
    g.profile(True)
    g.step(cyc)
    kt = g.kernel_times()
    g.profile(False)
    n2 = g.neutral_diag()
    nk = kt["neutral"]["launches"] + kt["neutral_compact"]["launches"]
    nt_launch = (n2["particle_steps"] - n1["particle_steps"]) / max(1, nk)
    nt_ms = kt["neutral"]["ms"] / max(1, kt["neutral"]["launches"])
    nt_bytes = BYTES_NEUTRAL_KERNEL * nt_launch
    achieved = nt_bytes / (nt_ms / 1000.0) / 1e9
    nc_ms = kt["neutral_compact"]["ms"] / max(1, kt["neutral_compact"]["launches"])
    nc_bytes = BYTES_NEUTRAL_COMPACT * nt_launch
    g.close()
    del g
    torch.cuda.empty_cache()
    # the same grid, load and deuterium plasma without neutrals or smoothing
    q = W.variant(p, neutrals=0, neutral_ppc=0, smooth_passes=0, recycle=0.0, K_iz=0.0)
    h = pic.Simulation(q)
    h.step(args.warmup)
    h.sync()
    e0 = h.diag()["particle_steps"]
    ms_q = events_ms(torch, h.stream, lambda: h.step(K))
    ps_q = h.diag()["particle_steps"] - e0
    h.close()
    del h
    torch.cuda.empty_cache()
    out = {
        "workload": "c6: D+/e/D sheath on config 3's grid: 65536 cells, 100,007,936 charged particles "
                    "(exp(-x/(L/8)) load, pair source), 50,003,968 initial neutrals, every absorbed ion "
                    "recycled, K_iz n_e dt = 2e-4, two smoothing passes",
        "value": (charged + neutral) / (ms / 1000.0), "unit": "particle-steps/s (charged + neutral)",
        "steps": K, "ms_per_step": ms / K, "charged_particle_steps": charged, "neutral_particle_steps": neutral,
        "neutrals": {"n": n1["n"], "recycled": n1["recycled"], "lost": n1["lost"], "ionized": n1["ionized"]},
        "without_sheath_physics": {"value": ps_q / (ms_q / 1000.0), "unit": "particle-steps/s",
                                   "ms_per_step": ms_q / K},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "kernel": "k_neutral32 (in place)", "bytes_per_neutral": BYTES_NEUTRAL_KERNEL,
                     "bytes_per_launch": nt_bytes, "avg_launch_ms": nt_ms, "traffic": TRAFFIC_NEUTRAL * nt_launch,
                     "compacting_step": {"kernel": "k_neutral32 (compacting, sort steps)",
                                         "bytes_per_neutral": BYTES_NEUTRAL_COMPACT, "avg_launch_ms": nc_ms,
                                         "achieved": nc_bytes / (nc_ms / 1000.0) / 1e9 if nc_ms else None,
                                         "frac": nc_bytes / (nc_ms / 1000.0) / 1e9 / peak if nc_ms else None}},
        "kernels": {k: {"ms": round(v["ms"], 3), "launches": v["launches"]} for k, v in kt.items() if v["launches"]},
    }
    if not args.no_cpu:
        from oracle import oracle as O

        cores = len(os.sched_getaffinity(0))
        sample = W.variant(p, ppc=(max(1, p["ppc"][0] // 64), max(1, p["ppc"][1] // 64)),
                           neutral_ppc=max(1, p["neutral_ppc"] // 64))
        o = O.OracleSim(sample, threads=cores)
        o.step(1)
        c0, m0 = o.diag()["particle_steps"], o.neutral_diag()["particle_steps"]
        # steps of the sample until about 3 s of host time have passed
        t0 = time.perf_counter()
        n = 0
        while n < 400 and time.perf_counter() - t0 < 3.0:
            o.step(5)
            n += 5
        dt = time.perf_counter() - t0
        work = o.diag()["particle_steps"] - c0 + o.neutral_diag()["particle_steps"] - m0
        out["cpu_baseline"] = {"value": work / dt, "unit": "particle-steps/s (charged + neutral)", "cores": cores,
                               "kind": "oracle", "sample": f"ppc/64 of c6, {n} steps, {dt:.2f} s"}
    return out


def adjoint_section(args, torch, pic) -> dict:
    """Config 5: forward + reverse sweep of the collisionless adjoint (checkpoint every 20 steps),
    timed on the device; its gradient against the FP64 oracle's on the host cores."""
    p = W.variant(W.C5, V_left=-1.0)
    steps = W.C5_STEPS
    a = pic.Adjoint(p, steps, 20)
    VL, Te = p["V_left"], p["T"][0]
    a.forward(VL, Te)
    a.gradient(1.0, 0.0)  # warm-up
    fwd, rev = [], []
    for _ in range(args.adj_reps):
        J = a.forward(VL, Te)
        g_flux = a.gradient(1.0, 0.0)
        f_ms, r_ms = a.times()
        fwd.append(f_ms)
        rev.append(r_ms)
    g_fe = a.gradient(0.0, 1.0)
    a.close()
    n = p["ncells"] * (p["ppc"][0] + p["ppc"][1])
    f_ms, r_ms = statistics.median(fwd), statistics.median(rev)
    out = {
        "workload": f"c5: collisionless, {p['ncells']} cells, {n:,} particles, {steps} steps, "
                    "checkpoint every 20 steps, parameters (V_left, T_e), observables (J_flux, J_fe)",
        "forward_ms": f_ms, "gradient_ms": r_ms,
        "value": n * steps / ((f_ms + r_ms) / 1000.0), "unit": "particle-steps/s (forward + one reverse sweep)",
        "J": list(J), "grad_flux": list(g_flux), "grad_fe": list(g_fe),
    }
    if not args.no_cpu:
        from oracle import oracle as O

        t0 = time.perf_counter()
        go_f, Jo, _ = O.adj_gradient(p, steps, (1.0, 0.0))
        go_e, _, _ = O.adj_gradient(p, steps, (0.0, 1.0))
        out["oracle"] = {"J": list(Jo), "grad_flux": list(go_f), "grad_fe": list(go_e),
                         "seconds": round(time.perf_counter() - t0, 2),
                         "rel_diff_flux": float(math.dist(g_flux, go_f) / math.hypot(*go_f)),
                         "rel_diff_fe": float(math.dist(g_fe, go_e) / math.hypot(*go_e))}
    return out


class Ranks:
    """Barrier, max and sum over the ranks of a torch.distributed process group (one process per
    GPU, NCCL on the GPUs, gloo on the CPU); a lone process when ``dist`` is None.  A value travels
    as a one-element float64 tensor on ``device``."""

    def __init__(self, dist, device: str):
        self.dist, self.device = dist, device

    def barrier(self) -> None:
        if self.dist is not None:
            self.dist.barrier()

    def _reduce(self, x: float, op) -> float:
        if self.dist is None:
            return float(x)
        import torch

        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, x: float) -> float:
        return self._reduce(x, None if self.dist is None else self.dist.ReduceOp.MAX)

    def sum(self, x: float) -> float:
        return self._reduce(x, None if self.dist is None else self.dist.ReduceOp.SUM)


def replica_params(workload: str, rank: int) -> dict:
    """The run rank ``rank`` advances: the workload itself, seeded seed + 1000 * rank, so that the
    replicas draw independent particles and collisions while each does a full run's work."""
    base = W.CONFIGS[workload]
    return W.variant(base, seed=base["seed"] + 1000 * rank)


def whole_job(units: float, ms: float, ranks: Ranks):
    """Whole-job throughput: the units every rank processed over the slowest rank's time.
    Returns (units per second, the slowest rank's milliseconds)."""
    ms_max = ranks.max(ms)
    return ranks.sum(units) / (ms_max / 1000.0), ms_max


def run_ours(args, rank: int, world: int, local: int) -> None:
    import torch

    from paper_2606_28534_gb300 import build, pic

    build.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    ranks = Ranks(dist, "cuda")

    # replicas: every rank advances its own simulation; no data-path collective
    params = replica_params(args.workload, rank)
    sim = pic.Simulation(params)
    sim.step(args.warmup)
    sim.sync()

    clocks = Clocks(torch.cuda.current_device()) if rank == 0 else None
    if clocks:
        clocks.start()
    ranks.barrier()
    torch.cuda.synchronize()
    # Steps of the large workloads take a millisecond or more: their kernels are timed inside the
    # timed region.  For small grids (steps of tens of microseconds) the per-launch events would add
    # gaps of their own, so those are timed without them and the kernels in a second run of the same
    # number of steps.
    short_steps = sum(sim.diag()["n"]) < 20_000_000
    ms, ps, kt = timed_run(sim, torch, args.steps, profile=not short_steps)
    if short_steps:
        kt = timed_run(sim, torch, args.steps, profile=True)[2]
    ranks.barrier()
    clk = clocks.stop() if clocks else None
    value, ms_max = whole_job(ps, ms, ranks)

    peak, peak_kind = _peaks()
    # the dominant kernel: the ordinary step (40 B per particle); the step after each sort, which
    # also moves every particle with its id to its sorted slot (56 B per particle), is reported
    # beside it
    n_launch = kt["step"]["launches"] + kt["step_scatter"]["launches"]
    per_launch_particles = ps / max(1, n_launch)
    step_ms = kt["step"]["ms"] / max(1, kt["step"]["launches"])
    plain_workload = params.get("precision") == W.PRECISION_FP64_PLAIN
    step_bytes = BYTES_STEP64_KERNEL if plain_workload else BYTES_STEP_KERNEL
    bytes_per_launch = step_bytes * per_launch_particles
    traffic = TRAFFIC_STEP * per_launch_particles if TRAFFIC_STEP and not plain_workload else None
    achieved = bytes_per_launch / (step_ms / 1000.0) / 1e9
    sc_ms = kt["step_scatter"]["ms"] / max(1, kt["step_scatter"]["launches"])
    sc_bytes = BYTES_SCATTER_KERNEL * per_launch_particles
    scatter_step = {"kernel": "k_step32 (scatter)", "launches": kt["step_scatter"]["launches"],
                    "avg_launch_ms": sc_ms, "bytes_per_launch": sc_bytes,
                    "achieved": sc_bytes / (sc_ms / 1000.0) / 1e9 if sc_ms else None,
                    "frac": sc_bytes / (sc_ms / 1000.0) / 1e9 / peak if sc_ms else None,
                    "traffic": TRAFFIC_SCATTER * per_launch_particles if TRAFFIC_SCATTER else None}
    kernel_shares = {k: round(v["ms"] / max(1e-9, sum(x["ms"] for x in kt.values())), 4)
                     for k, v in kt.items() if v["launches"]}

    # the single-GPU sections (plain path, ensemble, adjoint, sheath, precision) run only at N = 1:
    # with replicas they would repeat the same work on every rank
    single = world == 1
    # plain FP64 path on the same workload (the baseline the FP32 path is compared with)
    plain = None
    if single and not args.no_plain:
        sim.close()
        del sim
        torch.cuda.empty_cache()
        pp = W.variant(params, precision=W.PRECISION_FP64_PLAIN)
        ps_sim = pic.Simulation(pp)
        ps_sim.step(min(args.warmup, 5))
        ksteps = max(3, min(args.steps, args.plain_steps))
        pms, pps, _ = timed_run(ps_sim, torch, ksteps, profile=False)
        plain = {"value": whole_job(pps, pms, ranks)[0], "unit": "particle-steps/s",
                 "ms_per_step": pms / ksteps, "steps": ksteps, "dtype": "f64"}
        ps_sim.close()
        del ps_sim
        torch.cuda.empty_cache()
        sim = None

    # end to end through the public API: restart from a host checkpoint blob (pinned memory),
    # then steps with a device-to-host read of the diagnostics after every step
    e2e = None
    if not args.no_e2e:
        src = pic.Simulation(params)
        src.step(args.warmup)
        blob = src.snapshot()
        src.close()
        del src
        pinned = torch.empty(len(blob), dtype=torch.uint8, pin_memory=True)
        pinned.numpy()[:] = memoryview(blob)
        del blob
        ek = max(3, args.e2e_steps)  # a restart runs on from its checkpoint: its own step count
        sim2 = pic.Simulation(params)
        ranks.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc = pic.lib().pic_restore(sim2._h, pinned.data_ptr(), pinned.numel())
        if rc != 0:
            raise RuntimeError(f"pic_restore failed: {rc}")
        t1 = time.perf_counter()
        # every step's diagnostics are read back into a ring of DEPTH pinned buffers; step k's copy
        # is decoded once step k + DEPTH - 1 is enqueued, so that a host stall shorter than a few
        # steps does not leave the GPU idle
        DEPTH = 4
        nb = int(pic.lib().pic_diag_bytes())
        bufs = [torch.empty(nb, dtype=torch.uint8, pin_memory=True) for _ in range(DEPTH)]
        evs = [torch.cuda.Event() for _ in range(DEPTH)]
        dsum = 0
        for k in range(ek):
            sim2.step(1)
            sim2.diag_async(bufs[k % DEPTH], counters_only=True)
            evs[k % DEPTH].record(sim2.stream)
            j = k - (DEPTH - 1)
            if j >= 0:
                evs[j % DEPTH].synchronize()
                dsum = sim2.diag_decode(bufs[j % DEPTH])["particle_steps"]
        for j in range(max(0, ek - (DEPTH - 1)), ek):
            evs[j % DEPTH].synchronize()
            dsum = sim2.diag_decode(bufs[j % DEPTH])["particle_steps"]
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        # the same restore once more, outside the metric: it separates first-call costs of the
        # process (the temporary device buffer's first allocation, module loads) from the copy
        ta = time.perf_counter()
        rc = pic.lib().pic_restore(sim2._h, pinned.data_ptr(), pinned.numel())
        restore_again = time.perf_counter() - ta if rc == 0 else None
        sim2.close()
        # also outside the metric, after the restores (a first copy out of a freshly written pinned
        # buffer can be slower than later ones): the plain copy rate of this buffer to the device
        probe = torch.empty(pinned.numel(), dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        tp = time.perf_counter()
        probe.copy_(pinned, non_blocking=True)
        torch.cuda.synchronize()
        blob_h2d_gbs = pinned.numel() / (time.perf_counter() - tp) / 1e9
        del probe
        ranks.barrier()
        e2e = {"value": whole_job(dsum, 1e3 * (t2 - t0), ranks)[0], "unit": "particle-steps/s",
               "h2d_bytes_per_step": int(pinned.numel() / ek),
               "d2h_bytes_per_step": int(pic.lib().pic_diag_bytes()),
               "steps": ek, "restore_s": round(t1 - t0, 4),
               "restore_again_s": round(restore_again, 4) if restore_again is not None else None,
               "blob_h2d_gbs": round(blob_h2d_gbs, 1), "ms_per_step": round(1e3 * (t2 - t1) / ek, 4),
               "what": "pic_restore from a checkpoint blob in pinned host memory, then per step "
                       "pic_step(1) and pic_diag_async(PIC_DIAG_COUNTERS) (device-to-host copy of the "
                       "control block: counters, particle-steps, error word; no energy reduction) into "
                       "a ring of 4 pinned buffers, each step's copy decoded on the host three steps later"}

    batch = None
    if single and not args.no_batch:
        batch = batched(args, torch, pic, peak)
    adj = None
    if single and not args.no_adjoint:
        adj = adjoint_section(args, torch, pic)
    sheath = None
    if single and not args.no_sheath:
        sheath = sheath_section(args, torch, pic, peak)
    precision = None
    if single and not args.no_cpu and not args.no_precision:
        precision = precision_section(args, torch, pic)

    if rank != 0:
        return
    # the particle state against the L2: the default workload streams 2.8 GB per step, far beyond
    # the cache, so steps need no flush between them; the small cases say that they fit
    l2_bytes = int(getattr(torch.cuda.get_device_properties(local), "L2_cache_size", 0)) or (129 << 20)
    state = 28 * params["ncells"] * (params["ppc"][0] + params["ppc"][1])
    if state > l2_bytes:
        l2_note = f"inputs larger than L2 ({state / 1e9:.2f} GB of particles, L2 {l2_bytes >> 20} MB); no flush"
    else:
        l2_note = (f"inputs fit in L2 ({state / 1e6:.1f} MB of particles, L2 {l2_bytes >> 20} MB); not flushed: "
                   "a latency-bound small case")
    line = {
        "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if plain_workload else "f32",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: {W_DESC[args.workload]}",
                   "precision": ("FP64 particles, FP64 deposit and Poisson (the plain path)"
                                 if plain_workload else
                                 "FP32 particles/field, int64 fixed-point deposit, FP64 Poisson"),
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": l2_note,
                   "diagnostics": "kinetic energy summed by pic_diag on request (after the timed "
                                  "steps); e2e reads the counters of every step"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "k_step64" if plain_workload else "k_step32",
                     "peak_kind": peak_kind,
                     "timing": ("kernel times from a second run of the same steps with per-launch events"
                                if short_steps else "per-launch events inside the timed region"),
                     "bytes_per_launch": bytes_per_launch, "bytes_per_particle": step_bytes,
                     "avg_launch_ms": step_ms, "scatter_step": scatter_step},
        "kernels": {k: {"ms": round(v["ms"], 3), "launches": v["launches"]} for k, v in kt.items()
                    if v["launches"]},
        "kernel_shares": kernel_shares,
        "gpu_launches": int(sum(v["launches"] for v in kt.values())),
        "clocks": clk,
        "fp64_plain": plain,
        "batched": batch,
        "adjoint": adj,
        "sheath": sheath,
        "precision": precision,
        "e2e": e2e,
    }
    if world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(W.CONFIGS[args.workload], args.cpu_steps)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(W.CONFIGS), default="c3")
    ap.add_argument("--plain-steps", type=int, default=100)
    ap.add_argument("--e2e-steps", type=int, default=1000,
                    help="steps of the end-to-end leg after its restart from a host checkpoint")
    ap.add_argument("--cpu-steps", type=int, default=3, help="timed oracle steps of the CPU baseline")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--adj-reps", type=int, default=5)
    ap.add_argument("--batch-steps", type=int, default=W.C4_STEPS)
    ap.add_argument("--batch-sims", type=int, default=W.C4_SIMS, help="runs of the ensemble (config 4: 256)")
    ap.add_argument("--no-tune", action="store_true", help="default launch configuration of the batch")
    ap.add_argument("--no-sheath", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--sheath-steps", type=int, default=W.C6_STEPS)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
