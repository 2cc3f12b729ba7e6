"""Benchmark: atom-timesteps/s of the short-range MD hot path on one GB300.

Workload (one line): the 864,000-atom LJ liquid (60^3 fcc cells, rho 0.8442,
T 1.44, rc 2.5, skin 0.3, dt 0.005), mixed precision, velocity-Verlet NVE
with in-graph list rebuilds.  One bench "step" is one MD time step of the
whole path (drift, displacement check, conditional list rebuild, force +
kick).  The working set (list ~0.3 GB + state) exceeds the 129 MB L2, so no
L2 flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs N independent replicas (one per rank, torchrun); the path has no
exchange step ("replicas only").  --impl reference times the CPU oracle
(FP64 O(N^2)) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "atom-timesteps/s on 1 GB300, mixed vs plain FP64 at stated error; % roofline"
UNIT = "atom-timesteps/s"
WORKLOAD = "lj_liquid_864000_rc2.5_mixed"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cells", type=int, default=60)
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64 / rc 5.0 / EAM / batch side runs")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the CPU-oracle sample")
    ap.add_argument("--tpa", type=int, default=0, help="threads per atom (0: set-up mini-benchmark picks)")
    ap.add_argument("--list", default="auto", choices=["auto", "full", "half"])
    ap.add_argument("--vec", type=int, default=0, help="list entries per thread per load (0: default for tpa)")
    ap.add_argument("--block", type=int, default=128, help="force-kernel threads per block when --tpa is given")
    ap.add_argument("--eager", action="store_true",
                    help="step without CUDA graphs (kernels launched one by one; for profilers)")
    ap.add_argument("--profile", default=None, choices=["build", "eam_backward", "batch", "lj4000", "force", "eam"],
                    help="run one small workload for a profiler and exit: 'build' = LJ liquid (--cells, --rc), "
                         "100 steps to melt the lattice, then two list rebuilds; 'eam_backward' = EAM metal "
                         "(--cells), forces + backward twice; 'lj4000' = the 4,000-atom FP64 liquid, 100 steps "
                         "in one md_step graph launch and 100 eager steps (kernels launched one by one), both "
                         "timed; 'force' = LJ liquid (--cells), mixed, one thread per atom, full list: 50 steps, "
                         "then the force pass and its memory-only twin, each launched twice; 'eam' = EAM metal "
                         "(--cells), mixed, one thread per atom, full list: 100 steps, then the two force passes "
                         "(density and force) launched twice")
    ap.add_argument("--rc", type=float, default=2.5, help="LJ cut-off of --profile build")
    return ap.parse_args()


# ------------------------------------------------------------- distributed --

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def dist_init(ws):
    if ws <= 1:
        return None
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group("gloo")
    return dist


def max_over_ranks(dist, x):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0])


def barrier(dist):
    if dist is not None:
        dist.barrier()


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 100 ms while running,
    each sample stamped with the host clock so that the samples inside a
    region (the timed steps) can be told from the rest of the window."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([time.time()] + [c.strip() for c in line.split(",")])

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    @staticmethod
    def _summ(rows):
        # row: [host time, index, sm, max sm, power, active, hw, hw_thermal, sw_thermal, sw_power_cap]
        rows = [r[1:] for r in rows if len(r) > 9]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}

    def summary(self, t0=None, t1=None, window=""):
        """Clocks of the samples between host times t0 and t1 (the timed
        region); if that region was shorter than the sampling period, those of
        the whole window, which brackets it with the same kernels running."""
        inside = self._summ([r for r in self.rows if t0 is not None and t0 <= r[0] <= t1])
        whole = self._summ(self.rows)
        if inside is not None:
            inside["region"] = "timed steps"
            return inside
        if whole is not None:
            whole["region"] = window or "sampling window"
            return whole
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}


# ------------------------------------------------------------- workloads --

def make_lj(synth, cells, rc, prec, tpa=0, lst="auto"):
    from paper_1009_4330_gb300 import System
    d = synth.config1(rc=rc, cells=cells)
    # energies reported shifted (continuous at rc, for the drift); forces are the same
    s = System.lj(d["x"], d["v"], d["box"], cutoff=rc, skin=d["skin"], dt=d["dt"], mass=1.0, precision=prec,
                  list=lst, tpa=tpa, energy_shift=True)
    return s, d


def info0_is_full(s):
    return s.info()["list"] == "full"


def time_steps(s, K, W, eager=False, before=None, region=None):
    """W untimed steps, then K steps timed with CUDA events on the handle's
    stream (torch's current stream), synchronised on both sides.  region: a
    list that receives the host times bracketing the timed steps."""
    import torch
    s.step(W, eager=eager)
    torch.cuda.synchronize()
    if before is not None:
        before()
    i0 = s.info()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0 = time.time()
    e0.record()
    s.step(K, eager=eager)
    e1.record()
    torch.cuda.synchronize()
    t1 = time.time()
    if region is not None:
        region[:] = [t0, t1]
    i1 = s.info()
    ms = e0.elapsed_time(e1)
    return ms, i0, i1, None


def total_energy(s):
    ev = s.energy_virial()[0].cpu().numpy()
    return float(ev[0] + ev[1])


DRIFT_STEPS, DRIFT_EVERY = 1000, 50


def nve_drift(s, n, steps=DRIFT_STEPS, every=DRIFT_EVERY):
    """NVE energy conservation of a running system: E_tot/N (shifted energy)
    sampled every `every` steps over `steps` steps; the least-squares slope x
    1000 (drift per atom per 1,000 steps) and the largest excursion
    max |E(t) - E(0)| / N.  Independent of the bench's --steps."""
    es = []
    for k in range(steps // every + 1):
        es.append(total_energy(s) / n)
        if k < steps // every:
            s.step(every)
    t = np.arange(len(es)) * every
    slope = float(np.polyfit(t, np.array(es), 1)[0])
    return {"drift_per_atom_per_1000_steps": slope * 1000.0, "max_excursion_per_atom": float(np.abs(np.array(es) - es[0]).max()),
            "steps": steps, "sampled_every": every, "e_per_atom_start": es[0]}


EQUILIBRATION_STEPS = 500


def accuracy_report(s, d):
    """Accuracy stated with the throughput, on the bench workload itself,
    independent of --steps: a fresh copy of the workload with the bench run's
    kernel choice is carried 500 steps from its fcc start (the lattice melts
    in the first ~200 steps, while many pairs cross the cut-off at once),
    then (1) mixed-precision forces against the plain FP64 GPU path (which
    the tests hold to the FP64 oracle at 1e-12) at that state; (2) NVE drift
    over 1,000 further steps of the mixed run, and over 1,000 steps of the
    plain FP64 path from the same state (least-squares slope of the shifted
    total energy per atom, x 1000)."""
    from paper_1009_4330_gb300 import System
    n = d["x"].shape[0]
    k = s.info()
    with System.lj(d["x"], d["v"], d["box"], cutoff=d["rc"], skin=d["skin"], dt=d["dt"], mass=1.0, precision="mixed",
                   list=k["list"], tpa=k["tpa"], energy_shift=True) as sm:
        sm.set_kernel(k["tpa"], k["list"], k["block"], k["vec"])
        sm.step(EQUILIBRATION_STEPS)
        x, v, _ = sm.state()
        f_mixed = sm.compute_forces().cpu().numpy()
        with System.lj(x, v, d["box"], cutoff=d["rc"], skin=d["skin"], dt=d["dt"], mass=1.0, precision="fp64",
                       list="full", tpa=4, energy_shift=True) as s64:
            f64 = s64.compute_forces().cpu().numpy()
            err = float(np.abs(f_mixed - f64).max() / np.abs(f64).max())
            drift64 = nve_drift(s64, n)
        drift_mixed = nve_drift(sm, n)
    return {"mixed_force_rel_maxnorm_vs_fp64": err, "force_tolerance": 1e-5,
            "nve_drift_mixed": drift_mixed, "nve_drift_fp64": drift64, "drift_bound": 1e-4,
            "drift_definition": "least-squares slope of E_tot/N vs step, x 1000",
            "energy": "shifted LJ (continuous at rc)",
            "state": f"a fresh copy of the workload (the bench run's kernel choice) carried {EQUILIBRATION_STEPS} "
                     "steps from its fcc start"}


def e2e_run(s, d, K):
    """Same metric through the public API with host buffers: pinned H2D of x,
    v, K steps, D2H of energies and the final x, v -- all inside the timer."""
    import torch
    from paper_1009_4330_gb300 import system as sysmod  # noqa: F401
    n = d["x"].shape[0]
    hx = torch.from_numpy(d["x"]).pin_memory()
    hv = torch.from_numpy(d["v"]).pin_memory()
    ox = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    ov = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    oe = torch.empty((1, 8), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    dx = hx.to("cuda", non_blocking=True)
    dv = hv.to("cuda", non_blocking=True)
    s.set_state(x=dx, v=dv)
    s.step(K)
    ev = s.energy_virial()
    x, v, _ = s.state()
    oe.copy_(ev, non_blocking=True)
    ox.copy_(x, non_blocking=True)
    ov.copy_(v, non_blocking=True)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    h2d = 2 * n * 3 * 8
    d2h = 2 * n * 3 * 8 + 8 * 8
    return {"value": n * K / dt, "unit": UNIT, "h2d_bytes_per_step": h2d / K, "d2h_bytes_per_step": d2h / K,
            "seconds": dt, "steps": K}


def cpu_baseline(synth, cells, budget_s):
    """The oracle (FP64 O(N^2)) on a bounded sample of the same workload:
    forces of m atoms of the 864,000-atom liquid, each an O(N) sum over all
    atoms -- one atom-timestep of work per sampled atom (the integration is
    O(1) per atom and negligible)."""
    import oracle
    d = synth.config1(rc=2.5, cells=cells)
    n = d["x"].shape[0]
    rng = np.random.default_rng(7)
    m = 8
    idx = rng.choice(n, m, replace=False)
    t0 = time.perf_counter()
    oracle.lj_at(d["x"], d["box"], 2.5, idx)
    t1 = time.perf_counter() - t0
    m2 = int(max(8, min(200000, m * budget_s / max(t1, 1e-6))))
    idx = rng.choice(n, m2, replace=False)
    t0 = time.perf_counter()
    oracle.lj_at(d["x"], d["box"], 2.5, idx)
    t2 = time.perf_counter() - t0
    return {"value": m2 / t2, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"forces on {m2} random atoms of the {n}-atom LJ liquid (rc 2.5), FP64 O(N) each, "
                      f"{t2:.1f} s"}


# ------------------------------------------------------------------- arms --

def run_reference(args, ws, rank):
    if rank != 0:
        return
    import oracle
    import synth
    cells = args.cells
    d = synth.config1(rc=2.5, cells=cells)
    n = d["x"].shape[0]
    rng = np.random.default_rng(11)
    # size each step's sample so that warmup + steps fit in ~2 minutes
    probe = rng.choice(n, 4, replace=False)
    t0 = time.perf_counter()
    oracle.lj_at(d["x"], d["box"], 2.5, probe)
    per_atom = (time.perf_counter() - t0) / 4
    total = max(1, args.steps + args.warmup)
    m = int(max(1, min(5000, n, 100.0 / total / max(per_atom, 1e-9))))
    for _ in range(args.warmup):
        oracle.lj_at(d["x"], d["box"], 2.5, rng.choice(n, m, replace=False))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.lj_at(d["x"], d["box"], 2.5, rng.choice(n, m, replace=False))
    dt = time.perf_counter() - t0
    value = m * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "atoms": n, "sample_atoms_per_step": m},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"each step: FP64 O(N) forces on {m} random atoms of the {n}-atom liquid"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# DRAM bytes per atom that one launch of the force kernel moves
# (dram__bytes_read.sum + dram__bytes_write.sum), from one ncu capture of a
# 500,000-atom case of this workload, scaled by atoms (the list length per
# atom is the same).  Valid only for this kernel variant, as captured; for
# any other variant roofline.traffic is null.
K_LJ_TRAFFIC_PER_ATOM = (182.529792e6 + 3.975168e6) / 500000
K_LJ_TRAFFIC_VARIANT = {"tpa": 1, "vec": 4, "list": "full", "block": 128, "tile_atoms": 0}

# FP32 operations per list entry of the mixed full-list pair loop (a fused
# multiply-add counted as 2), counted from its source: the separation with
# the stencil offset 3 + 6 + 3 (offset decode), r^2 5, reciprocal 1, r^-6 2,
# the pair coefficient 4, the cut-off test and band minimum 2, the three
# force sums 6, the compensated round sums 3 (12 additions per 4 entries).
FP32_OPS_PER_ENTRY = 35
# FP64 operations per list entry of the FP64 pair loop, counted the same way:
# separation 9, r^2 5, Newton reciprocal 7, r^-6 2, coefficient 4, cut-off 1,
# force sums 6.
FP64_OPS_PER_ENTRY = 34


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            j = json.load(fh)
        return float(j["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def roofline_of(f_ms, f_bytes, entries, g_ms, ceil, peak, peak_kind, traffic):
    """The force pass against the three ceilings: HBM (its algorithmic bytes
    per launch), random 16-byte gathers from L2 (its list entries, one record
    gather each), the FP32 pipe (its pair-loop operations), plus its own
    access pattern's ceiling (the memory-only twin)."""
    sec = f_ms / 1000.0
    achieved = f_bytes / sec / 1e9
    out = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
           "traffic": traffic,
           "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one 500,000-atom capture of this "
                             "kernel variant, scaled by atoms" if traffic else None,
           "kernel": "k_lj (force + kick, md_step form)", "peak_kind": peak_kind,
           "force_ms": f_ms, "force_algorithmic_bytes": f_bytes}
    ceilings = {"hbm": {"peak_GBs": peak, "achieved_GBs": achieved, "frac": achieved / peak, "source": peak_kind}}
    if ceil:
        gps = entries / sec / 1e9
        ceilings["l2_gather"] = {"peak_Ggathers_s": ceil["l2_gather_gps"], "achieved_Ggathers_s": gps,
                                 "frac": gps / ceil["l2_gather_gps"], "source": "md_probe_ceilings"}
        tf = FP32_OPS_PER_ENTRY * entries / sec / 1e12
        ceilings["fp32"] = {"peak_TFLOPs": ceil["fp32_fma_tflops"], "achieved_TFLOPs": tf,
                            "frac": tf / ceil["fp32_fma_tflops"], "ops_per_entry": FP32_OPS_PER_ENTRY,
                            "source": "md_probe_ceilings"}
        ceilings["hbm_own_copy_GBs"] = ceil["hbm_copy_gbs"]
    if g_ms:
        ceilings["access_pattern_twin"] = {"twin_ms": g_ms, "frac": g_ms / f_ms,
                                           "note": "the same list stream and record gathers, no arithmetic"}
    if ceil and ceilings["l2_gather"]["frac"] > 1.0:
        ceilings["l2_gather"]["note"] = ("above the random-gather probe: the pass's gathers share records between "
                                         "neighbouring atoms and hit L1 (the twin measures its own pattern)")
    out["ceilings"] = ceilings
    # the binding ceiling: the access pattern's own (the twin) when measured,
    # else the largest fraction among the probes it does not exceed
    if g_ms:
        out["binding"] = "access_pattern_twin"
    else:
        fr = {k: v["frac"] for k, v in ceilings.items() if isinstance(v, dict) and "frac" in v and v["frac"] <= 1.0}
        out["binding"] = max(fr, key=fr.get) if fr else "hbm"
    return out


def run_ours(args, ws, rank, local):
    import torch
    import synth
    from paper_1009_4330_gb300 import probe_ceilings
    torch.cuda.set_device(local)
    dist = dist_init(ws)
    cells = args.cells
    # clocks sampled from before the warm-up to the end of the accuracy legs
    # (same kernels throughout); the timed steps' own samples are preferred
    clocks = ClockSampler(local)
    clocks.__enter__()
    # tpa 0: the set-up mini-benchmark picks threads per atom, list kind and block size
    s, d = make_lj(synth, cells, 2.5, "mixed", tpa=args.tpa, lst=args.list if args.tpa else "auto")
    tune = s.autotune_table()
    if args.tpa and args.vec:
        s.set_kernel(args.tpa, args.list if args.list != "auto" else "full", args.block, args.vec)
    n = d["x"].shape[0]
    K, W = args.steps, max(3, args.warmup)
    barrier(dist)
    region = []
    ms, i0, i1, _ = time_steps(s, K, W, eager=args.eager, region=region)
    ms = max_over_ranks(dist, ms)
    value = ws * n * K / (ms / 1000.0)
    rebuilds = i1["rebuilds"] - i0["rebuilds"]
    # our kernels in the timed region: loop control once; per step the drift,
    # its one-block bookkeeping kernel and the force pass (1 kernel with a full
    # list, 3 with a half list); 7 per list rebuild (8 with staged tiles)
    launches = 1 + K * (2 + (3 if i1["list"] == "half" else 1)) + (8 if i1["tile_atoms"] else 7) * rebuilds
    # dominant kernel: the force pass as md_step runs it, timed with CUDA events on the handle's stream
    f_ms, f_bytes = s.time_force(warmup=3, reps=20)
    info = s.info()
    # the ceiling of the same access pattern: the force pass's memory-only twin
    g_ms = s.time_gather(warmup=3, reps=20) if info["list"] == "full" else None
    accuracy = accuracy_report(s, d) if rank == 0 else None
    clocks.__exit__()
    clk = clocks.summary(region[0], region[1],
                         window="set-up, warm-up, timed steps, force timings and the 1,000-step accuracy runs "
                                "(the timed steps alone were shorter than the 100 ms sampling period)")
    peak, peak_kind = load_peaks()
    ceil = probe_ceilings() if rank == 0 else None
    same_variant = all(info[k] == v for k, v in K_LJ_TRAFFIC_VARIANT.items())
    traffic = K_LJ_TRAFFIC_PER_ATOM * n if same_variant else None
    roof = roofline_of(f_ms, f_bytes, info["list_entries"], g_ms, ceil, peak, peak_kind, traffic)
    roof["force_share_of_step"] = f_ms / (ms / K)
    # the whole step against HBM: per atom-step the force pass's bytes, the
    # drift's 104 B (x and v read, x written, the build record read, the FP32
    # record written), and the rebuilds amortised over the timed steps (list
    # written, 4 B per entry, plus the sort's ~150 B per atom)
    per_atom = f_bytes / n + 104.0 + (rebuilds / K) * (4.0 * info["list_entries"] / n + 150.0)
    step_gbs = per_atom * n / (ms / K / 1000.0) / 1e9
    roof["step"] = {"algorithmic_bytes_per_atom_step": per_atom, "achieved_GBs": step_gbs, "frac": step_gbs / peak,
                    "note": "whole md_step (force pass, drift, amortised rebuilds) against the HBM copy peak"}
    e2e = e2e_run(s, d, K)
    extras = {}
    if not args.no_extras and rank == 0:
        extras = side_runs(synth, cells, K, W, ceil, tune_rc25=tune)
    cpu = cpu_baseline(synth, cells, args.cpu_seconds) if (rank == 0 and ws == 1) else None
    s.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W,
            "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 pair math, f64 accumulate/integrate", "data": "synthetic",
            "config": {"workload": WORKLOAD, "atoms": n, "cells": cells, "rc": 2.5, "skin": 0.3, "dt": 0.005,
                       "precision": "mixed", "tpa": info["tpa"], "list": info["list"], "block": info["block"],
                       "vec": info["vec"], "graph": not args.eager,
                       "avg_list_length": info["list_entries"] / n, "rebuilds_in_timed_region": rebuilds,
                       "steps_per_rebuild": (K / rebuilds) if rebuilds else None,
                       "l2": "working set > L2 (list alone ~0.3 GB): no flush", "parallelism": "replicas" if ws > 1 else "1 GPU"},
            "roofline": roof,
            "clocks": clk,
            "e2e": e2e,
            "gpu_launches": launches,
            "accuracy": accuracy,
            "autotune": tune,
            "cpu_baseline": cpu,
            "extras": extras,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def step_arm(s, n, k, W):
    """md_step throughput of a system as configured, CUDA events."""
    ms, i0, i1, _ = time_steps(s, k, W)
    inf = s.info()
    return {"value": n * k / (ms / 1000), "ms_per_step": ms / k, "steps": k, "tpa": inf["tpa"], "list": inf["list"],
            "vec": inf["vec"], "block": inf["block"], "rebuilds": i1["rebuilds"] - i0["rebuilds"]}


def force_arm(s, ceil, prec):
    """The force pass alone (md_step form), with its pipe fraction for the precision's pipe."""
    fms, fby = s.time_force(3, 10)
    inf = s.info()
    out = {"force_ms": fms, "force_GBs": fby / (fms / 1000) / 1e9}
    if ceil and s.potential == "lj":
        # per list entry the pair term is evaluated once, full or half list
        if prec == "fp64":
            tf = FP64_OPS_PER_ENTRY * inf["list_entries"] / (fms / 1000) / 1e12
            out["fp64_TFLOPs"] = tf
            out["fp64_pipe_frac"] = tf / ceil["fp64_fma_tflops"]
        else:
            tf = FP32_OPS_PER_ENTRY * inf["list_entries"] / (fms / 1000) / 1e12
            out["fp32_TFLOPs"] = tf
            out["fp32_pipe_frac"] = tf / ceil["fp32_fma_tflops"]
    return out


def best_of(tune, lst):
    rows = [r for r in tune if r["list"] == lst]
    return min(rows, key=lambda r: r["ms"]) if rows else None


def lj_pair(synth, cells, rc, K, W, ceil, tune=None):
    """LJ liquid at cut-off rc: mixed (autotuned) with its best full-list and
    best half-list variants' step times, and the plain FP64 path (autotuned)."""
    out = {}
    k = max(50, K // 4) if rc > 3 else max(50, K // 5)
    s, d = make_lj(synth, cells, rc, "mixed", tpa=0)
    n = d["x"].shape[0]
    tune = tune if tune is not None else s.autotune_table()
    m = step_arm(s, n, k, W)
    m.update(force_arm(s, ceil, "mixed"))
    out["mixed"] = m
    for lst in ("full", "half"):
        b = best_of(tune, lst)
        if b is None:
            continue
        s.set_kernel(b["tpa"], lst, b["block"], b["vec"])
        a = step_arm(s, n, k, W)
        a["force_ms_autotune"] = b["ms"]
        out[f"mixed_{lst}_list"] = a
    out["autotune"] = tune
    s.close()
    s, _ = make_lj(synth, cells, rc, "fp64", tpa=0)
    k64 = max(20, k // 10)
    f = step_arm(s, n, k64, 3)
    f.update(force_arm(s, ceil, "fp64"))
    out["fp64"] = f
    out["fp64_autotune"] = s.autotune_table()
    s.close()
    out["mixed_over_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    return out


def side_runs(synth, cells, K, W, ceil, tune_rc25=None):
    """Context numbers: every workload in mixed precision and in plain FP64
    (same inputs), half against full lists, the design alternatives, the CPU
    cell-list baseline, the backward passes."""
    import torch
    from paper_1009_4330_gb300 import System, lj_params
    out = {}
    out["ceilings"] = ceil
    out["lj864k_rc2.5"] = lj_pair(synth, cells, 2.5, K, W, ceil)
    out["lj864k_rc5.0"] = lj_pair(synth, cells, 5.0, K, W, ceil)
    # EAM 500,000 atoms (full lists only)
    e = synth.config2()
    ne = e["x"].shape[0]
    eam = {}
    for prec in ("mixed", "fp64"):
        s = System.eam(e["x"], e["v"], e["box"], eam_params=e["eam"], skin=e["skin"], dt=e["dt"], mass=e["mass"],
                       ftm2v=e["ftm2v"], precision=prec, tpa=0)
        k = max(50, K // 2) if prec == "mixed" else max(20, K // 20)
        a = step_arm(s, ne, k, 5)
        a.update(force_arm(s, ceil, prec))
        a["autotune"] = s.autotune_table()
        eam[prec] = a
        s.close()
    eam["mixed_over_fp64"] = eam["mixed"]["value"] / eam["fp64"]["value"]
    out["eam500000"] = eam
    # batched replicas (512, log-uniform 500..20000)
    b = synth.config4()
    nb = int(sum(b["sizes"]))
    bat = {}
    for prec in ("mixed", "fp64"):
        s = System.batch(b["replicas"], params=lj_params(1.0, 1.0, 1), cutoff=2.5, skin=0.3, dt=0.005, mass=1.0,
                         precision=prec, tpa=0)
        k = max(50, K // 4) if prec == "mixed" else max(20, K // 40)
        a = step_arm(s, nb, k, 5)
        a.update(force_arm(s, ceil, prec))
        a["atoms"] = nb
        bat[prec] = a
        s.close()
    bat["mixed_over_fp64"] = bat["mixed"]["value"] / bat["fp64"]["value"]
    out["batch512"] = bat
    # 4,000-atom LJ liquid, plain FP64, 100 steps (latency-bound small system)
    c0 = synth.config0()
    s = System.lj(c0["x"], c0["v"], c0["box"], cutoff=2.5, skin=0.3, dt=0.005, mass=1.0, precision="fp64", tpa=0)
    ms, i0, i1, _ = time_steps(s, 100, 10)
    out["fp64_lj4000_100steps"] = {"value": 4000 * 100 / (ms / 1000), "ms_per_step": ms / 100, "tpa": i1["tpa"],
                                   "list": i1["list"]}
    s.close()
    # spatial decomposition on this one GPU: the 864,000-atom liquid cut into 2
    # slabs driven by two threads (every step: a host synchronisation for the
    # global rebuild decision and device-packed halo exchanges)
    out["decomposed_2slabs_lj864k"] = domain_timing(synth, cells)
    # force matching: forward forces + backward (positions and 6 parameters), 32,768 atoms
    out["force_matching_32768"] = force_matching_timing(synth)
    out["eam500000_fwd_bwd"] = eam_backward_timing(synth)
    # design alternative: block-local lists with shared-memory staging (off by
    # default), force pass and its memory-only twin against the default layout
    s, d = make_lj(synth, cells, 2.5, "mixed", tpa=1, lst="full")
    s.step(20)
    alt = {}
    for staged in (False, True):
        s.set_staging(staged)
        fms, fby = s.time_force(3, 10)
        gms = s.time_gather(3, 10)
        inf = s.info()
        alt["staged" if staged else "gathered"] = {"force_ms": fms, "twin_ms": gms, "tiles_staged": inf["tiles_staged"],
                                                   "n_tiles": inf["n_tiles_force"], "block": inf["block"]}
    # the cell-list force pass (no Verlet list) on the same staged tiles
    _, cms = s.cell_forces(reps=10)
    alt["cell_list"] = {"force_ms": cms, "note": "27 cells tested per atom, no list read or built"}
    out["staging_alternative_rc2.5"] = alt
    s.close()
    # O(N) CPU baseline: velocity Verlet with FP64 cell-list forces on the host
    # cores, 2 steps of the same 864,000-atom liquid (the cpu_baseline of the
    # line is the O(N^2) oracle)
    out["cpu_celllist"] = cpu_celllist(synth, cells)
    torch.cuda.synchronize()
    return out


def cpu_celllist(synth, cells, steps=2):
    import oracle
    d = synth.config1(rc=2.5, cells=cells)
    f = oracle.lj_cells(d["x"], d["box"], 2.5)
    t0 = time.perf_counter()
    oracle.nve_cells(d["x"], d["v"], d["box"], 2.5, d["dt"], 1.0, steps, f=f)
    dt = time.perf_counter() - t0
    n = d["x"].shape[0]
    return {"value": n * steps / dt, "unit": "atom-timesteps/s", "cores": oracle.num_threads(),
            "kind": "O(N) cell-list FP64 velocity Verlet (host)", "sample": f"{steps} steps of the {n}-atom liquid"}


def domain_timing(synth, cells, steps=100):
    """atom-timesteps/s of the slab decomposition (2 sub-domains, threads on one
    GPU), mixed precision, full lists: the cost of the exchanges and the
    per-step rebuild decision, beside md_step's single graph launch."""
    import threading
    from paper_1009_4330_gb300.domain import SlabDomain, SlabLayout, ThreadComm, ThreadWorld, split_global
    d = synth.config1(rc=2.5, cells=cells)
    lay = SlabLayout(d["box"], 2, 2.8, 0.3)
    parts = split_global(lay, d["x"], d["v"])
    world = ThreadWorld(2)
    res = [None, None]
    errors = []

    def rank(r):
        try:
            ids, xr, vr, tr = parts[r]
            dom = SlabDomain(ThreadComm(world, r), lay, xr, vr, ids, tr, params=[1.0, 1.0], cutoff=2.5, skin=0.3,
                             dt=0.005, mass=1.0, precision="mixed", list="full", tpa=1)
            dom.step(10)
            world.barrier.wait()
            t0 = time.perf_counter()
            dom.step(steps)
            world.barrier.wait()
            res[r] = (time.perf_counter() - t0, dom.rebuilds, dom.n_own)
            dom.close()
        except Exception as e:  # reported below; the other thread's waits are released
            errors.append(repr(e))
            world.barrier.abort()

    th = [threading.Thread(target=rank, args=(r,)) for r in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    if errors or None in res:
        return {"error": errors[0] if errors else "a sub-domain thread did not finish"}
    sec = max(r[0] for r in res)
    n = d["x"].shape[0]
    return {"value": n * steps / sec, "unit": UNIT, "ms_per_step": 1000 * sec / steps, "steps": steps,
            "rebuilds": res[0][1], "owned": [r[2] for r in res], "timer": "host wall clock (threads)"}


def force_matching_timing(synth, reps=20):
    """Time per forward (forces) + backward (dL/dx, dL/d(eps, sigma)) of the
    32,768-atom binary LJ force-matching workload, CUDA events."""
    import torch
    from paper_1009_4330_gb300 import System
    c = synth.config3()
    v = np.zeros_like(c["x"])
    e0, s0 = synth.pair_matrix(c["eps0"]), synth.pair_matrix(c["sig0"])
    out = {}
    for prec in ("mixed", "fp64"):
        s = System.lj(c["x"], v, c["box"], eps=e0, sig=s0, types=c["types"], n_types=2, cutoff=2.5, skin=0.3,
                      dt=0.005, mass=[1.0, 1.0], precision=prec, tpa=0)
        g = torch.ones((c["x"].shape[0], 3), dtype=torch.float64, device="cuda")
        f = torch.empty_like(g)
        for _ in range(3):
            s.compute_forces(out=f)
            s.backward(g)
        torch.cuda.synchronize()
        e0_, e1_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0_.record()
        for _ in range(reps):
            s.compute_forces(out=f)
            s.backward(g)
        e1_.record()
        torch.cuda.synchronize()
        ms = e0_.elapsed_time(e1_) / reps
        info = s.info()
        out[prec] = {"ms_per_fwd_bwd": ms, "pair_evaluations_per_s": 2 * info["list_entries"] / (ms / 1000),
                     "tpa": info["tpa"]}
        s.close()
    return out


def eam_backward_timing(synth, reps=10):
    """Time per forward (density + forces) + backward (dL/dx, dL/d(A, c0, c1, c2)) of
    the 500,000-atom EAM metal, CUDA events; the backward is two FP64 list passes."""
    import torch
    from paper_1009_4330_gb300 import System
    d = synth.config2(displacement=0.1)
    out = {}
    for prec in ("mixed", "fp64"):
        s = System.eam(d["x"], d["v"], d["box"], eam_params=d["eam"], skin=d["skin"], dt=d["dt"], mass=d["mass"],
                       ftm2v=d["ftm2v"], precision=prec, tpa=0)
        g = torch.ones((d["x"].shape[0], 3), dtype=torch.float64, device="cuda")
        f = torch.empty_like(g)
        for _ in range(3):
            s.compute_forces(out=f)
            s.backward(g)
        torch.cuda.synchronize()
        e0_, e1_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0_.record()
        for _ in range(reps):
            s.compute_forces(out=f)
            s.backward(g)
        e1_.record()
        torch.cuda.synchronize()
        ms = e0_.elapsed_time(e1_) / reps
        info = s.info()
        out[prec] = {"ms_per_fwd_bwd": ms, "atoms_per_s": d["x"].shape[0] / (ms / 1000), "tpa": info["tpa"]}
        s.close()
    return out


def run_profile(args):
    """Small workloads for profiler captures (not a bench line)."""
    import torch
    import synth
    from paper_1009_4330_gb300 import System, lj_params
    if args.profile == "lj4000":
        c0 = synth.config0()
        s = System.lj(c0["x"], c0["v"], c0["box"], cutoff=2.5, skin=0.3, dt=0.005, mass=1.0, precision="fp64",
                      tpa=args.tpa or 8, list="full")
        s.step(20)
        ms_graph, i0, i1, _ = time_steps(s, 100, 5)
        ms_eager, j0, j1, _ = time_steps(s, 100, 5, eager=True)
        print(json.dumps({"ms_per_step_graph": ms_graph / 100, "ms_per_step_eager": ms_eager / 100,
                          "rebuilds_graph": i1["rebuilds"] - i0["rebuilds"], "rebuilds_eager": j1["rebuilds"] - j0["rebuilds"],
                          "info": i1}))
        s.close()
        return
    if args.profile == "eam":
        e = synth.config2(cells=args.cells)
        s = System.eam(e["x"], e["v"], e["box"], eam_params=e["eam"], skin=e["skin"], dt=e["dt"], mass=e["mass"],
                       ftm2v=e["ftm2v"], precision="mixed", tpa=1, list="full")
        s.set_kernel(1, "full", 128, 4)
        s.step(100)
        f_ms, _ = s.time_force(0, 2)
        print(json.dumps({"force_ms": f_ms, "atoms": int(e["x"].shape[0])}))
        s.close()
        return
    if args.profile == "force":
        s, d = make_lj(synth, args.cells, args.rc, "mixed", tpa=1, lst="full")
        s.set_kernel(1, "full", 128, 4)
        s.step(50)
        f_ms, _ = s.time_force(0, 2)
        g_ms = s.time_gather(0, 2)
        print(json.dumps({"force_ms": f_ms, "twin_ms": g_ms, "atoms": int(d["x"].shape[0])}))
        s.close()
        return
    if args.profile == "build":
        s, d = make_lj(synth, args.cells, args.rc, "mixed", tpa=args.tpa or (1 if args.rc < 3 else 4), lst="full")
        s.step(100)
        s.build_neighbors()
        s.build_neighbors()
    elif args.profile == "batch":
        # the 512-replica batch: graph steps, then eager steps (kernels visible to a profiler)
        b = synth.config4()
        natoms = int(sum(b["sizes"]))
        s = System.batch(b["replicas"], params=lj_params(1.0, 1.0, 1), cutoff=2.5, skin=0.3, dt=0.005, mass=1.0,
                         precision="mixed", tpa=args.tpa or 1)
        s.step(50)
        ms_graph, _, _, _ = time_steps(s, 50, 5)
        ms_eager, _, _, _ = time_steps(s, 20, 2, eager=True)
        print(json.dumps({"ms_per_step_graph": ms_graph / 50, "ms_per_step_eager": ms_eager / 20}))
    else:
        d = synth.config2(cells=args.cells, displacement=0.1)
        s = System.eam(d["x"], d["v"], d["box"], eam_params=d["eam"], skin=d["skin"], dt=d["dt"], mass=d["mass"],
                       ftm2v=d["ftm2v"], precision="mixed", tpa=args.tpa or 1)
        g = torch.ones((d["x"].shape[0], 3), dtype=torch.float64, device="cuda")
        for _ in range(2):
            s.compute_forces()
            s.backward(g)
    if args.profile != "batch":
        natoms = int(d["x"].shape[0])
    torch.cuda.synchronize()
    print(json.dumps({"profile": args.profile, "atoms": natoms, "info": s.info()}))
    s.close()


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.profile:
        run_profile(args)
        return
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
