#!/usr/bin/env python
"""Benchmark: particle-turns per second of the tracking hot path on GB300.

Default workload (one "step"): the paper-scale single bunch -- 1e6 macro-particles
tracked 1e4 turns with each of Euler-Cromer, leap-frog and 4th-order Ruth in FP64,
with the transverse (x, x', y, y') matrix push and per-turn bunch moments (stride 1),
ring C = 6911.5 m, h = 4620, p0 = 26 GeV/c, gamma_t = 22.77, V = 4.5 MV, phi_s = 0.
Inputs are seeded synthetic bunches (matched Gaussian truncated at 80 % of the bucket
half-length, transverse Gaussians with beta = 50 m, eps_n = 2 um).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME]

Prints one JSON line (rank 0).  Under torchrun (N > 1) every rank tracks its own
bunch (weak scaling, no data-path collective); the timed region is bracketed by a
barrier and device synchronisation and the maximum over ranks is reported.
The reference arm (--impl reference) times the FP64 oracle on the host cores on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("particle-turns/s (FP64 vs FP32-compensated, batched) at stated accuracy; "
          "% FP64 peak; p50/p99")
UNIT = "particle-turns/s"

WORKLOADS = {
    "single_bunch_1e6x1e4_ec_lf_ruth4_f64": dict(
        n=1_000_000, turns=10_000, schemes=("euler_cromer", "leapfrog", "ruth4"), dtype="f64",
        voltage=4.5e6, transverse=True, stride=1),
    # the widened map: slippage expansion eta(d) = eta0 + 0.05 d + 2 d^2
    # in the drift and chromaticities xi_x = 5, xi_y = -3 (per-particle transverse phase
    # advance), the same bunch size and turns; a bunch inside half the separatrix
    "widened_map_1e6x1e4_f64": dict(
        n=1_000_000, turns=10_000, schemes=("euler_cromer", "leapfrog", "ruth4"), dtype="f64",
        voltage=4.5e6, transverse=True, stride=1, sep_frac=0.5,
        ring=dict(eta1=0.05, eta2=2.0, xi_x=5.0, xi_y=-3.0)),
    # classic RK4 (four force evaluations per turn) on a double-RF ring: second system at
    # h2 = 2h with V2 = 0.3 V in phase (bunch lengthening), 1e6 particles x 1e4 turns
    "rk4_double_rf_1e6x1e4_f64": dict(
        n=1_000_000, turns=10_000, schemes=("rk4",), dtype="f64", voltage=4.5e6,
        transverse=True, stride=1, sep_frac=0.5,
        ring=dict(harmonic2=2 * 4620, voltage2_V=0.3 * 4.5e6, phi2_rad=0.0)),
    # the three symplectic schemes on the same double-RF ring
    "double_rf_1e6x1e4_ec_lf_ruth4_f64": dict(
        n=1_000_000, turns=10_000, schemes=("euler_cromer", "leapfrog", "ruth4"), dtype="f64",
        voltage=4.5e6, transverse=True, stride=1, sep_frac=0.5,
        ring=dict(harmonic2=2 * 4620, voltage2_V=0.3 * 4.5e6, phi2_rad=0.0)),
    # accelerating bucket: a linear momentum ramp from 26 GeV/c gaining 0.4 MeV/c per turn
    # (26 -> 30 GeV/c over 1e4 turns) at 4.5 MV (phi_s ~ 0.09 rad), per-turn constants from
    # the programme table; the gain per turn, not the end momentum, is fixed, so a shorter
    # run (--turns) keeps the same bucket
    "ramp_1e6x1e4_ec_lf_ruth4_f64": dict(
        n=1_000_000, turns=10_000, schemes=("euler_cromer", "leapfrog", "ruth4"), dtype="f64",
        voltage=4.5e6, transverse=True, stride=1, sep_frac=0.5, ramp=dict(gain_eVc_per_turn=4e5)),
    # collective step after every turn: 512 uniform slices on [-0.75, 0.75) m, a decaying
    # oscillating (resonator-like) wake table, kick -5e-11 x V plus space charge 1e-9 x the
    # line-density slope; leap-frog, 1e6 x 1e4 turns
    "collective_wake_1e6x1e4_lf_f64": dict(
        n=1_000_000, turns=10_000, schemes=("leapfrog",), dtype="f64", voltage=4.5e6,
        transverse=True, stride=1, sep_frac=0.5,
        wake=dict(nslices=512, z_lo=-0.75, z_hi=0.75, alpha=-5e-11, alpha_sc=1e-9)),
    # small case for quick checks (not a bench line)
    "tiny": dict(n=20_000, turns=200, schemes=("euler_cromer", "leapfrog", "ruth4"),
                 dtype="f64", voltage=4.5e6, transverse=True, stride=1),
    # 64 uneven bunches (log-uniform 1e3-4e6 particles, ~6e7 in total; V ~ U(1, 6) MV;
    # turns ~ U(1e3, 1e5)), leap-frog FP32-compensated, per-bunch turn-by-turn monitors,
    # one graph-captured batch per step
    "batched_64_bunches_f32c_lf": dict(kind="batched", nbunch=64, total=6e7, dtype="f32c",
                                       scheme="leapfrog", stride=1),
    # the same batch with the double-float phase (no FP64 instruction on the path)
    "batched_64_bunches_f32cd_lf": dict(kind="batched", nbunch=64, total=6e7, dtype="f32cd",
                                        scheme="leapfrog", stride=1),
    # the same batch in FP64 (per-job FP64 reference point; turns scaled down by 100)
    "batched_64_bunches_f64_lf": dict(kind="batched", nbunch=64, total=6e7, dtype="f64",
                                      scheme="leapfrog", stride=1, turn_scale=0.01),
    # serving: Poisson arrivals at 200 jobs/s (the first --serving-jobs of the trace), sizes
    # log-uniform 1e4-8e6, turns log-uniform 1e2-1e5, integrator uniform over three,
    # FP64 or FP32C 50/50, 150 GB admission budget; then the same jobs at ~70 % load
    "serving_poisson_200hz": dict(kind="serving", count=2000, rate_hz=200.0, budget=150e9),
    # precision sweep: 4e6 particles x 1e6 turns leap-frog FP32C (60 % core, 40 % halo to
    # 98 % of the separatrix) against FP64 on a 1e4-particle subsample
    "precision_sweep_4e6x1e6_lf": dict(kind="precision", n=4_000_000, turns=1_000_000,
                                       subsample=10_000, voltage=2e6, stride=10_000),
}
DEFAULT_WORKLOAD = "single_bunch_1e6x1e4_ec_lf_ruth4_f64"

# Algorithmic FP64 flops per particle-turn (FMA = 2).  One drift = 1 FMA; one kick =
# phase FMA + sine + subtract + FMA; one sine = SINE_FLOPS (argument reduction by
# Cody-Waite plus a degree-13/14 polynomial on |r| <= pi/4); transverse = 2 planes x
# (2 MUL + 2 FMA).  These are counted against the FP64 peak.  The moment sums (3 planes x
# (2 ADD + 3 FMA) = 24 flops) are computed in double-float on the FP32 pipe and reported
# separately, not against the FP64 peak.
SINE_FLOPS = 20
KICK_FLOPS = 2 + SINE_FLOPS + 1 + 2
DRIFT_FLOPS = 2
SCHEME_FLOPS = {"euler_cromer": DRIFT_FLOPS + KICK_FLOPS,
                "leapfrog": 2 * DRIFT_FLOPS + KICK_FLOPS,
                "ruth4": 4 * DRIFT_FLOPS + 3 * KICK_FLOPS}
# Classic RK4 per particle-turn: four right-hand sides, each the slippage term -eta0 C d
# (1 MUL; with the expansion -(eta0 C + eta1 C d + eta2 C d^2) d, 2 FMA + 1 MUL = 5) and the
# force A F1(z) (phase FMA, sine, subtract, multiply = 24); the stage arguments z + c k,
# d + c k (2 x 2 FMA + 2 ADD = 10) and the weighted sums (per coordinate 2 ADD + 2 FMA = 6,
# x 2 = 12).
RK4_RHS_FLOPS = 1 + 2 + SINE_FLOPS + 1 + 1
RK4_SLIP_NL_EXTRA = 4
SCHEME_FLOPS["rk4"] = 4 * RK4_RHS_FLOPS + 10 + 12
# the second RF system: each force evaluation adds phase FMA, sine, subtract and FMA
RF2_FLOPS = 2 + SINE_FLOPS + 1 + 2
KICKS = {"euler_cromer": 1, "leapfrog": 1, "ruth4": 3, "rk4": 4}
# ramp programme: per particle-turn delta, x' and y' are multiplied by r_n
RAMP_FLOPS = 3
# collective step per particle-turn: the slice index (subtract, multiply) and the kick's add
COLLECTIVE_FLOPS = 3
TRANSVERSE_FLOPS = 12
MONITOR_FLOPS = 24
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12  # SMs x DFMA/clk x flops x max clock


# The widened map: a drift with the slippage expansion is 3 FMA (6 flops); a chromatic
# plane is the angle FMA (2), sine and cosine of 2 pi a (quarter-turn reduction: subtract,
# multiply; r^2; two degree-5 Horner chains; r^3, r^4 and three final FMAs: 31) and the
# rotation (b s, s / b, 2 MUL + 2 FMA: 8) = 41.
DRIFT_FLOPS_NL = 6
CHROMA_PLANE_FLOPS = 41


def alg_flops(scheme, transverse, monitor, ring=None):
    """FP64-pipe algorithmic flops per particle-turn (the monitor is FP32-pipe work): the
    method's arithmetic for the ring's parameters -- a drift takes the slippage expansion
    only where eta1 or eta2 is nonzero (the widened map's kernels, which a chromaticity or
    a second RF system also selects, execute the expansion's FMAs on zeros otherwise; those
    are not counted)."""
    ring = ring or {}
    nl = ring.get("eta1", 0.0) != 0.0 or ring.get("eta2", 0.0) != 0.0
    chroma = [ring.get("xi_x", 0.0) != 0.0, ring.get("xi_y", 0.0) != 0.0]
    dual = ring.get("voltage2_V", 0.0) != 0.0
    f = SCHEME_FLOPS[scheme]
    if nl:
        if scheme == "rk4":
            f += 4 * RK4_SLIP_NL_EXTRA
        else:
            ndrift = {"euler_cromer": 1, "leapfrog": 2, "ruth4": 4}[scheme]
            f += ndrift * (DRIFT_FLOPS_NL - DRIFT_FLOPS)
    if dual:
        f += KICKS[scheme] * RF2_FLOPS
    if transverse:
        f += sum(CHROMA_PLANE_FLOPS if c else TRANSVERSE_FLOPS // 2 for c in chroma)
    return f


# ----------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                smax.append(float(p[1]))
            except ValueError:
                continue
            for nm, v in zip(names, p[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, dist, device=None) -> float:
    """Maximum of a per-rank float over all ranks (identity when not distributed)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_inputs(wl, derived, seed):
    """Synthetic bunch of the workload, drawn with the library's own bucket geometry."""
    from paper_1610_05801_gb300 import synth

    b = synth.Bucket(k=derived.k, A=derived.A, etaC=derived.etaC, Qs=derived.Qs,
                     betagamma=derived.betagamma)
    z, dp, _ = synth.matched_bunch(seed, wl["n"], b, sep_frac=wl.get("sep_frac", 1.0))
    out = [z, dp]
    if wl["transverse"]:
        out += list(synth.transverse_gaussian(seed + 1, wl["n"], 50.0, 2e-6, derived.betagamma))
        out += list(synth.transverse_gaussian(seed + 2, wl["n"], 50.0, 2e-6, derived.betagamma))
    return out


def ramp_programme(wl):
    """(V[turns], p0[turns + 1]) of a ramp workload: a linear momentum ramp from the ring's
    p0 gaining wl['ramp']['gain_eVc_per_turn'] per turn, at the workload's voltage."""
    import numpy as np

    from paper_1610_05801_gb300 import synth

    turns = wl["turns"]
    pa = synth.ring(wl["voltage"])["p0_eVc"]
    return np.full(turns, wl["voltage"]), pa + wl["ramp"]["gain_eVc_per_turn"] * np.arange(turns + 1)


def wake_table(wl):
    """The workload's wake samples w[m] = exp(-m / 51.2) cos(m / 25.6) (512 slices)."""
    import numpy as np

    ns = wl["wake"]["nslices"]
    m = np.arange(ns)
    return np.exp(-m / (0.1 * ns)) * np.cos(m / (0.05 * ns))


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the baseline's record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu part")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


# The oracle's bounded sample of the paper-scale workload, the same in both arms: 1e4
# particles x the workload's 1e4 turns x its three schemes (transverse planes and per-turn
# moments included), i.e. 3e8 particle-turns per step.
CPU_SAMPLE_PARTICLES = 10_000


def cpu_baseline(wl, steps=1, warmup=0, n_sample=CPU_SAMPLE_PARTICLES, turns_sample=None,
                 threads=0):
    """The FP64 oracle, as it stands, on the host cores: a bounded sample of the workload
    (n_sample particles x turns_sample turns x every scheme, with the same transverse
    planes and per-turn moments); threads = 0: all cores.  Returns (particle-turns/s,
    threads, sample text, per-step seconds)."""
    import oracle
    from paper_1610_05801_gb300 import synth

    turns = turns_sample or wl["turns"]
    ring = synth.ring(wl["voltage"], transverse=True, **(wl.get("ring") or {}))
    O = oracle.load()
    O.set_num_threads(threads if threads > 0 else (os.cpu_count() or 1))
    d = O.derive(ring)
    b = synth.Bucket(k=d.k, A=d.A, etaC=d.etaC, Qs=d.Qs, betagamma=d.betagamma)
    z, dp, _ = synth.matched_bunch(1, n_sample, b)
    tr = []
    if wl["transverse"]:
        tr += list(synth.transverse_gaussian(2, n_sample, 50.0, 2e-6, d.betagamma))
        tr += list(synth.transverse_gaussian(3, n_sample, 50.0, 2e-6, d.betagamma))
    times = []
    tc = None
    if wl.get("ramp"):
        V, p0 = ramp_programme(wl)
        tc = O.ramp_derive(ring, V[:turns], p0[:turns + 1])
    for it in range(warmup + steps):
        t0 = time.perf_counter()
        for s in wl["schemes"]:
            if tc is not None:
                O.track_ramp(d, tc, s, z, dp, *tr, turns=turns, moments=wl["stride"] > 0,
                             stride=max(1, wl["stride"]))
            elif wl.get("wake"):
                wk = wl["wake"]
                O.track_collective(d, s, z, dp, *tr, turns=turns, z_lo=wk["z_lo"],
                                   inv_dz=wk["nslices"] / (wk["z_hi"] - wk["z_lo"]),
                                   w=wake_table(wl), alpha=wk["alpha"], alpha_sc=wk["alpha_sc"],
                                   moments=wl["stride"] > 0, stride=max(1, wl["stride"]))
            else:
                O.track(d, s, z, dp, *tr, turns=turns, moments=wl["stride"] > 0,
                        stride=max(1, wl["stride"]))
        dt = time.perf_counter() - t0
        if it >= warmup:
            times.append(dt)
    used = O.num_threads()
    O.set_num_threads(os.cpu_count() or 1)
    pt = n_sample * turns * len(wl["schemes"])
    sample = (f"{n_sample} particles x {turns} turns x {len(wl['schemes'])} schemes "
              f"({'+transverse' if wl['transverse'] else ''}{' +moments' if wl['stride'] else ''})"
              f" of the same workload, FP64 oracle, OpenMP over particles")
    return pt / (sum(times) / len(times)), used, sample, times


def cpu_baseline_report(wl, n_sample=CPU_SAMPLE_PARTICLES):
    """The CPU baseline the line carries: the oracle on all host cores (the value) and on one
    core, on the workload's bounded sample, plus the small workload (1e3 particles x 1e3
    leap-frog turns, FP64, no transverse planes, no monitor) both ways, and the CPU model."""
    v, cores, sample, _ = cpu_baseline(wl, steps=2, warmup=1, n_sample=n_sample)
    # one core on a tenth of the turns (the same particles and schemes): ~15 s of CPU work
    v1, _, sample1, _ = cpu_baseline(wl, steps=1, n_sample=n_sample,
                                     turns_sample=max(1, wl["turns"] // 10), threads=1)
    small = dict(n=1000, turns=1000, schemes=("leapfrog",), voltage=2e6, transverse=False,
                 stride=0)
    s_all, c_all, _, _ = cpu_baseline(small, steps=5, warmup=1, n_sample=1000)
    s_one, _, _, _ = cpu_baseline(small, steps=5, warmup=1, n_sample=1000, threads=1)
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
            "cpu_model": cpu_model(), "nproc": os.cpu_count(),
            "single_thread": {"value": v1, "sample": sample1},
            "small_workload_1e3x1e3_lf": {"all_cores": s_all, "single_thread": s_one,
                                         "cores": c_all}}


# ----------------------------------------------------------------------------------------
def run_reference(args, wl_name, wl):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    v, cores, sample, times = cpu_baseline(wl, steps=args.steps, warmup=args.warmup,
                                           n_sample=args.cpu_sample)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl_name, "n_particles": wl["n"], "turns": wl["turns"],
                   "integrators": list(wl["schemes"]), "transverse": wl["transverse"],
                   "monitor_stride": wl["stride"], "step_sample": sample},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample, "cpu_model": cpu_model()},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, wl_name, wl):
    import numpy as np
    import torch

    from paper_1610_05801_gb300 import build as _build
    from paper_1610_05801_gb300 import phtl, synth

    ws, rank, local = dist_env()
    dist = None
    if ws > 1:
        import torch.distributed as dist  # noqa: F811

        torch.cuda.set_device(local)
        dist.init_process_group(backend="nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    _build.build()

    ring = synth.ring(wl["voltage"], transverse=True, **(wl.get("ring") or {}))
    R = phtl.Ring(**ring)
    if wl.get("block") or wl.get("tpl"):
        R.set_tuning(block_threads=wl.get("block", 0), turns_per_launch=wl.get("tpl", 0))
    der = R.derived()
    host = make_inputs(wl, der, seed=1 + rank)
    n, turns, dt = wl["n"], wl["turns"], wl["dtype"]
    if dt == "f64":
        bufs = [torch.tensor(a, dtype=torch.float64, device=dev) for a in host]
    else:
        bufs = [torch.tensor(phtl.split_f32c(a), dtype=torch.float32, device=dev) for a in host]
    while len(bufs) < 6:
        bufs.append(None)
    nrows = turns // max(1, wl["stride"]) + 1
    mon = torch.zeros((nrows, phtl.MON_FIELDS), dtype=torch.float64, device=dev)
    if wl["stride"]:
        R.set_monitor(mon, stride=wl["stride"])
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2

    ev = {s: [] for s in wl["schemes"]}
    nlaunch = {s: 0 for s in wl["schemes"]}
    track = R.track_perturn if wl.get("perturn") else R.track
    if wl.get("wake"):
        wk = wl["wake"]
        R.set_wake(wake_table(wl), wk["z_lo"], wk["z_hi"], wk["alpha"], wk["alpha_sc"])
        track = R.track_collective
    if wl.get("ramp"):
        R.set_programme(*ramp_programme(wl))

        def track(*b, turns, integrator, dtype, stream):
            R.track_programme(*b, turn0=0, turns=turns, integrator=integrator, dtype=dtype,
                              stream=stream)

    def step(record=False):
        for s in wl["schemes"]:
            if record:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                l0 = R.stats().launches
                e0.record(stream)
            track(*bufs, turns=turns, integrator=s, dtype=dt, stream=stream)
            if record:
                e1.record(stream)
                ev[s].append((e0, e1))
                nlaunch[s] += R.stats().launches - l0

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    st0 = R.stats()
    wall0 = time.perf_counter()
    step_events = []
    for _ in range(args.steps):
        flush.zero_()  # L2 flush between timed steps, outside the step's events
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step(record=True)
        b.record(stream)
        step_events.append((a, b))
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    st1 = R.stats()
    # every kernel of the library in the timed region: the tracking launches and the
    # one-thread cancellation gate in front of each persistent launch
    launches = (st1.launches - st0.launches) + (st1.gate_launches - st0.gate_launches)
    step_ms = [a.elapsed_time(b) for a, b in step_events]
    t_local = sum(step_ms) / 1e3
    t_max = max_over_ranks(t_local, dist, dev)
    units = n * turns * len(wl["schemes"]) * args.steps * ws
    value = units / t_max

    # dominant kernel: the most expensive scheme's persistent kernel
    per_scheme_ms = {s: sum(a.elapsed_time(b) for a, b in ev[s]) / len(ev[s]) for s in ev}
    dom = max(per_scheme_ms, key=per_scheme_ms.get)
    launches_per_call = max(1, nlaunch[dom] // args.steps)
    if wl.get("wake"):
        # two launches per turn (turn + slicing, potential): the turn kernel's duration is
        # bounded above by the call's time per turn (the potential kernel and the gaps
        # included), so the achieved rate below is a lower bound
        launches_per_call = turns
    tpl = math.ceil(turns / launches_per_call)
    dur_s = per_scheme_ms[dom] / 1e3 / launches_per_call
    flops_pt = alg_flops(dom, wl["transverse"], wl["stride"] > 0, wl.get("ring"))
    if wl.get("ramp"):
        flops_pt += RAMP_FLOPS
    if wl.get("wake"):
        # per particle the slice index (subtract, multiply) and the kick's add (the map's
        # flops are the ring's, linear or widened, as for the other workloads)
        flops_pt += COLLECTIVE_FLOPS
    flops = flops_pt * n * tpl
    achieved = flops / dur_s / 1e12

    if args.no_e2e or wl.get("perturn") or wl.get("ramp") or wl.get("wake"):
        e2e_value, h2d, d2h, e2e_steps, phases = None, 0, 0, 0, None
    else:
        e2e_value, h2d, d2h, e2e_steps, phases = e2e_host(R, host, wl, args, dist, dev, ws)
    roof = per_turn_roofline(wl, per_scheme_ms, n, turns, dt) if wl.get("perturn") else None
    kname = (f"k_track_{'f64' if dt == 'f64' else 'f32c'}<{dom}"
             f"{', transverse' if wl['transverse'] else ''}{', monitor' if wl['stride'] else ''}"
             f"{', widened map' if wl.get('ring') else ''}{', ramp programme' if wl.get('ramp') else ''}>")
    if wl.get("ramp"):
        kname = kname.replace("k_track_", "k_ramp_")
    if wl.get("wake"):
        kname = f"k_coll_turn<{dom}> (one turn + slicing + previous turn's wake kick)"

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dt,
        "data": "synthetic (seeded matched bunch + transverse Gaussians; no dataset)",
        "config": {"workload": wl_name, "n_particles": n, "turns": turns,
                   "integrators": list(wl["schemes"]), "transverse": wl["transverse"],
                   "monitor_stride": wl["stride"], "ring": "C=6911.5 m h=4620 p0=26 GeV/c "
                   "gamma_t=22.77 V=4.5 MV phi_s=0" + "".join(
                       f" {k}={v}" for k, v in (wl.get("ring") or {}).items()) + (
                       f" ramp p0 26 GeV/c + {wl['ramp']['gain_eVc_per_turn'] / 1e6:g} MeV/c "
                       f"per turn" if wl.get("ramp") else ""),
                   "l2": "flushed between timed steps (256 MiB write); state 48 MB resident",
                   "parallelism": f"replica per GPU x{ws}",
                   "launch": "per-turn" if wl.get("perturn") else "persistent"},
        "roofline": roof or (issue_roofline(
            kname, (dt, dom, bool(wl["transverse"]), bool(wl["stride"]),
                    False if map_variant(wl) == "plain" else map_variant(wl)),
            n * tpl / dur_s, clk.get("sm_mhz")) if dt != "f64" else None) or fp64_roofline(
            kname, dt, dom, wl, n, tpl, dur_s, flops_pt, achieved),
        "gpu_launches": launches,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": e2e_steps,
                "api": "phtl_track_host (pinned host buffers; alloc, H2D, kernels, D2H, free)",
                "last_call_phases_ms": phases},
        "clocks": clk,
        "per_scheme_ms": per_scheme_ms,
        "wall_s_timed_region": wall,
    }
    if wl.get("wake") and line["roofline"].get("basis"):
        line["roofline"]["basis"] += ("; the time per turn includes the potential kernel and "
                                      "the launch gaps, so the fraction is a lower bound")
    return finish_line(line, args, wl, rank, R, dist, ws)


# DRAM bytes per particle per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# persistent FP64 kernel, from one ncu capture (--set full) of the current kernel on a
# 3e6-particle case (state larger than L2); the launch's traffic grows in proportion to its
# particles.  Summary: profiles/k_track_f64_ruth4_transverse_monitor_3e6x100.md.
NCU_TRAFFIC_BYTES_PER_PARTICLE = {("f64", "ruth4", True, True): (144.729600e6 + 83.410688e6) / 3e6}


# FP64 flops the kernel executes per particle-turn, from the same ncu capture:
# (2 x DFMA + DMUL + DADD thread instructions per cycle) x cycles / particle-turns, i.e.
# (2 x 225.068198 + 33.760230 + 0.474220) x 22.946400 ms x 2.044726 GHz / (3e6 x 88).
# Fewer than the algorithmic count: for phi_s = 0 the kernel skips the phase addition and the
# sin(phi_s) subtraction of the general kick and flips the sine's sign with an integer XOR.
NCU_EXEC_FLOPS_PER_PARTICLE_TURN = {("f64", "ruth4", True, True, "plain"):
                                    (2 * 225.068198 + 33.760230 + 0.474220) * 22.946400e-3
                                    * 2.044726e9 / (3e6 * 88)}
# The map variants, from thread-instruction totals of one launch each
# (smsp__sass_thread_inst_executed_op_{dfma,dmul,dadd}_pred_on.sum; 3e6 particles, the automatic
# turns per launch: 88 for Ruth4, 66 for RK4): (DFMA, DMUL, DADD, particle-turns).
NCU_EXEC_COUNTS = {
    # chromaticity and amplitude detuning: a sine and cosine of each plane's phase per turn
    ("f64", "ruth4", True, True, "widened"): (19_536_000_000, 5_814_000_000, 550_250_000, 3e6 * 88),
    # second RF system: a second sine per kick
    ("f64", "ruth4", True, True, "double_rf"): (21_384_000_000, 3_174_000_000, 814_250_000, 3e6 * 88),
    ("f64", "rk4", True, True, "double_rf"): (20_196_000_000, 4_752_000_000, 1_996_750_000, 3e6 * 66),
    # ramp programme: the general kick (phi_s != 0), delta, x' and y' rescaled every turn
    ("f64", "ruth4", True, True, "ramp"): (11_352_000_000, 2_376_000_000, 814_250_000, 3e6 * 88),
    # the batched FP64 kernel, leap-frog bunches with monitors: one launch of the 64-bunch batch
    # scaled to 4.0e6 particles at full turns, 200 turns for every bunch, 256-thread blocks
    # (profiles/k_batched_f64_leapfrog_monitor_4e6.md)
    ("f64", "leapfrog", False, True, "batched"): (9_646_080_000, 1_607_680_000, 9_467_100,
                                                  4005158 * 200),
    # the collective step's turn kernel (k_coll_turn, leap-frog, transverse, monitor): one turn
    # of 3e6 particles (profiles/k_coll_turn_leapfrog_collective_3e6x20.md)
    ("f64", "leapfrog", True, True, "collective"): (54_001_152, 9_000_128, 6_187_504, 3e6),
}
for _k, (_fma, _mul, _add, _pt) in NCU_EXEC_COUNTS.items():
    NCU_EXEC_FLOPS_PER_PARTICLE_TURN[_k] = (2 * _fma + _mul + _add) / _pt


def map_variant(wl):
    """The kernel variant a workload runs: 'plain', 'widened' (second-order slippage,
    chromaticity), 'double_rf', 'ramp', 'batched', 'collective', or None for the per-turn
    path."""
    if wl.get("perturn"):
        return None
    if wl.get("wake"):
        return "collective"
    if wl.get("kind") == "batched":
        return "batched"
    if wl.get("ramp"):
        return "ramp"
    ring = wl.get("ring") or {}
    if ring.get("voltage2_V"):
        return "double_rf"
    return "widened" if ring else "plain"


def executed_flops(dt, scheme, wl, particle_turns_per_s):
    """ncu's executed DP FLOP/s rescaled to the live launch duration, where a capture of
    this kernel exists: the fraction of the FP64 peak the pipe's own flop count gives."""
    key = (dt, scheme, bool(wl["transverse"]), bool(wl["stride"]), map_variant(wl))
    f = NCU_EXEC_FLOPS_PER_PARTICLE_TURN.get(key)
    if f is None:
        return {}
    tf = f * particle_turns_per_s / 1e12
    return {"executed_flops_per_particle_turn_ncu": f, "executed_tflops": tf,
            "executed_frac": tf / FP64_PEAK_TFLOPS}


def fp64_roofline(kname, dt, dom, wl, n, tpl, dur_s, flops_pt, achieved_alg):
    """FP64-pipe roofline of the dominant persistent kernel.  The cost of an FP64 sine is
    implementation-defined, so the fraction of the FP64 peak is taken from the FP64 flops the
    kernel executes (ncu: 2 x DFMA + DMUL + DADD per particle-turn, stored per kernel variant)
    at the live launch duration; where no capture of the variant exists, from the
    algorithmic count with each sine costed at SINE_FLOPS.  Both counts are reported, and
    the sine-free count of the method's drifts, kick multiply-adds and transverse push."""
    exe = executed_flops(dt, dom, wl, n * tpl / dur_s)
    base = {"bound": "alu", "kernel": kname, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "traffic": kernel_traffic(dt, dom, wl, n),
            "peak_source": "FP64: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (recipe unit "
                           "counts and max clock); DFMA rate confirmed by a microbenchmark",
            "launch_ms": dur_s * 1e3, "turns_per_launch": tpl,
            "alg_flops_per_particle_turn": flops_pt,
            "alg_sine_flops": SINE_FLOPS, "alg_achieved": achieved_alg,
            "alg_frac": achieved_alg / FP64_PEAK_TFLOPS,
            "moment_flops_per_particle_turn_fp32_pipe": MONITOR_FLOPS if wl["stride"] else 0}
    nosine = flops_pt - SINE_FLOPS * KICKS.get(dom, 0) * (
        1 + (1 if (wl.get("ring") or {}).get("voltage2_V") else 0))
    base["alg_flops_per_particle_turn_without_sines"] = nosine
    base["alg_frac_without_sines"] = nosine * n * tpl / dur_s / 1e12 / FP64_PEAK_TFLOPS
    if exe:
        base.update(exe)
        base.update(achieved=exe["executed_tflops"], frac=exe["executed_frac"],
                    basis="ncu-executed FP64 flops per particle-turn (2 DFMA + DMUL + DADD) "
                          "x live particle-turns/s; alg_frac counts each sine as "
                          f"{SINE_FLOPS} flops")
    else:
        base.update(achieved=achieved_alg, frac=achieved_alg / FP64_PEAK_TFLOPS,
                    basis=f"algorithmic FP64 flops, each sine costed at {SINE_FLOPS} flops "
                          "(no ncu count of this kernel variant stored)")
    return base


def kernel_traffic(dt, scheme, wl, n):
    key = (dt, scheme, bool(wl["transverse"]), bool(wl["stride"]))
    b = NCU_TRAFFIC_BYTES_PER_PARTICLE.get(key)
    return None if b is None or wl.get("perturn") else b * n


def per_turn_roofline(wl, per_scheme_ms, n, turns, dt):
    """HBM roofline of the per-turn variant: the state is read and written every turn."""
    import json as _j  # noqa: F401

    peaks = measured_peaks()
    coords = 6 if wl["transverse"] else 2
    bytes_pt = coords * 2 * 8  # FP64: 8 B per coordinate; FP32C: hi + comp = 8 B; read + write
    dom = max(per_scheme_ms, key=per_scheme_ms.get)
    achieved = bytes_pt * n * turns / (per_scheme_ms[dom] / 1e3) / 1e9
    return {"bound": "hbm", "kernel": f"per-turn launches, {dom}, {dt}", "achieved": achieved,
            "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
            "traffic": None, "peak_source": peaks["source"],
            "alg_bytes_per_particle_turn": bytes_pt}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            m = json.load(f)
        return {"hbm_gbs": float(m["hbm_gbs"]), "source": "measured (MEASURED_PEAKS.json copy)"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "source": "fallback 6.8 TB/s"}


def e2e_host(R, host, wl, args, dist, dev, ws):
    """The same metric through phtl_track_host on pinned host buffers (H2D, kernels, D2H
    inside the timed region)."""
    import torch

    from paper_1610_05801_gb300 import phtl

    n, turns, dt = wl["n"], wl["turns"], wl["dtype"]
    if dt == "f64":
        hbufs = [torch.tensor(a, dtype=torch.float64).pin_memory() for a in host]
    else:
        hbufs = [torch.tensor(phtl.split_f32c(a), dtype=torch.float32).pin_memory() for a in host]
    while len(hbufs) < 6:
        hbufs.append(None)
    nrows = turns // max(1, wl["stride"]) + 1
    hmon = torch.zeros((nrows, phtl.MON_FIELDS), dtype=torch.float64).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    R.track_host(*hbufs, turns=turns, integrator=wl["schemes"][0], dtype=dt,
                 mon_rows=hmon if wl["stride"] else None, mon_stride=max(1, wl["stride"]))
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for s in wl["schemes"]:
            R.track_host(*hbufs, turns=turns, integrator=s, dtype=dt,
                         mon_rows=hmon if wl["stride"] else None, mon_stride=max(1, wl["stride"]))
    e2e_t = max_over_ranks(time.perf_counter() - t0, dist, dev)
    nb = sum(h.numel() * h.element_size() for h in hbufs if h is not None)
    h2d = nb * len(wl["schemes"])
    d2h = (nb + (hmon.numel() * 8 if wl["stride"] else 0)) * len(wl["schemes"])
    return (n * turns * len(wl["schemes"]) * e2e_steps * ws / e2e_t, h2d, d2h, e2e_steps,
            R.phase_times())


def finish_line(line, args, wl, rank, R, dist, ws=1):
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_report(wl, n_sample=args.cpu_sample)
    R.close()
    if rank == 0 and ws == 1 and not args.no_extras and args.workload == DEFAULT_WORKLOAD:
        line.update(default_extras(args))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def _clocked(fn):
    """Run fn() with the clock sampler on; returns (fn's value, clocks)."""
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    try:
        v = fn()
    finally:
        clk = clocks.stop()
    return v, clk


# Executed warp-instructions per particle-turn of the FP32-compensated persistent kernels
# (sm__inst_executed.sum / particle-turns of the launch), from one ncu capture per kernel:
# 2e6 particles x 200 turns per launch, transverse planes, stride-1 monitor (summary:
# profiles/k_track_f32c_instruction_counts_2e6x200.md); keyed by (dtype, scheme,
# transverse, monitor, batched).
NCU_WARP_INST_PER_PARTICLE_TURN = {
    # FP32C at its 64-register budget (4 resident 256-thread blocks), the phase split with
    # the phase forms of the integer widening and split
    ("f32c", "leapfrog", True, True, False): 4410069242 / (2e6 * 200),
    ("f32c", "ruth4", True, True, False): 9480594061 / (2e6 * 200),
    ("f32cd", "leapfrog", True, True, False): 3924877111 / (2e6 * 200),
    ("f32cd", "ruth4", True, True, False): 8228979485 / (2e6 * 200),
    ("f32cs", "leapfrog", True, True, False): 2326276064 / (2e6 * 200),
    ("f32cs", "ruth4", True, True, False): 3477286084 / (2e6 * 200),
    # the batched FP32C kernel (leap-frog bunches, stride-1 monitors, no transverse planes): the
    # first launch of the 64-bunch batch scaled to 4.0e6 particles, 200 turns for every bunch,
    # 256-thread blocks (profiles/k_batched_f32c_leapfrog_monitor_4e6.md)
    ("f32c", "leapfrog", False, True, True): 6160999306 / (4005158 * 200),
    # the batched FP32CD kernel, the same batch and shape
    ("f32cd", "leapfrog", False, True, True): 5468097246 / (4005158 * 200),
}
# the general (widened-map and double-RF) FP32 kernels: one 2e6 x 200-turn launch each, transverse,
# stride-1 monitor (profiles/k_track_f32c_general_instruction_counts_2e6x200.md)
for _dt, _counts in (("f32c", (10580001894, 16535668547, 24935241314)),
                     ("f32cd", (10161272287, 15357883224, 22700504514)),
                     ("f32cs", (2700933979, 3972666386, 4572386973))):
    NCU_WARP_INST_PER_PARTICLE_TURN[(_dt, "leapfrog", True, True, "widened")] = _counts[0] / 4e8
    NCU_WARP_INST_PER_PARTICLE_TURN[(_dt, "ruth4", True, True, "widened")] = _counts[1] / 4e8
    NCU_WARP_INST_PER_PARTICLE_TURN[(_dt, "rk4", True, True, "double_rf")] = _counts[2] / 4e8
ISSUE_PER_SM_PER_CLK = 4  # one warp-instruction per clock per SM sub-partition


def issue_roofline(kname, key=None, pts=None, sm_mhz=None):
    """Issue-rate roofline of an FP32-compensated kernel: executed warp-instructions per
    particle-turn (ncu) x particle-turns per second / (SMs x 4 issue slots x SM clock).  The
    double-float arithmetic runs on the FP32 and integer pipes at one instruction per issue
    slot, so instruction issue, not FP64 flops, bounds it."""
    clk = (sm_mhz or 2070.0) * 1e6
    peak = 152 * ISSUE_PER_SM_PER_CLK * clk / 1e9
    per = NCU_WARP_INST_PER_PARTICLE_TURN.get(key) if key else None
    out = {"bound": "issue", "kernel": kname, "peak": peak, "unit": "G warp-instructions/s",
           "peak_source": f"152 SMs x {ISSUE_PER_SM_PER_CLK} warp-instructions/clk x "
                          f"{clk / 1e9:.3f} GHz (median SM clock sampled during the run)",
           "traffic": None}
    if per is None or pts is None:
        out.update(achieved=None, frac=None,
                   note="no ncu instruction count for this kernel variant")
        return out
    ach = per * pts / 1e9
    out.update(achieved=ach, frac=ach / peak, warp_inst_per_particle_turn_ncu=per)
    return out


def batch_jobs(wl, dev):
    """The batched workload's bunches as device buffers (seeded, matched to each voltage)."""
    import torch

    from paper_1610_05801_gb300 import phtl, synth

    specs = synth.batched_jobs(seed=3, nbunch=wl["nbunch"], total=wl["total"])
    scale = wl.get("turn_scale", 1.0)
    ring = synth.ring(2e6)
    dt = wl["dtype"]
    jobs, keep = [], []
    for sp in specs:
        der = phtl.Ring(**dict(ring, voltage_V=sp["voltage_V"])).derived()
        b = synth.Bucket(k=der.k, A=der.A, etaC=der.etaC, Qs=der.Qs, betagamma=der.betagamma)
        z, d, _ = synth.matched_bunch(sp["seed"], sp["n"], b)
        turns = max(1, int(sp["turns"] * scale))
        if dt == "f64":
            bz = torch.tensor(z, dtype=torch.float64, device=dev)
            bd = torch.tensor(d, dtype=torch.float64, device=dev)
        else:
            bz = torch.tensor(phtl.split_f32c(z), dtype=torch.float32, device=dev)
            bd = torch.tensor(phtl.split_f32c(d), dtype=torch.float32, device=dev)
        mon = torch.zeros((turns // wl["stride"] + 1, 16), dtype=torch.float64, device=dev)
        jobs.append(phtl.make_job(bz, bd, turns=turns, voltage_V=sp["voltage_V"],
                                  integrator=wl["scheme"], dtype=dt, monitor=mon,
                                  stride=wl["stride"]))
        keep += [bz, bd, mon]
    return specs, ring, jobs, keep


def measure_batched(wl, steps, warmup):
    """64 uneven bunches, one graph-captured batch per step: particle-turns/s over the timed
    runs (CUDA events on the launching stream), with the clocks sampled meanwhile."""
    import torch

    from paper_1610_05801_gb300 import phtl

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    specs, ring, jobs, keep = batch_jobs(wl, dev)
    R = phtl.Ring(**ring)
    if wl.get("block") or wl.get("tpl"):  # a fixed launch shape instead of the autotuner's
        R.set_tuning(block_threads=wl.get("block", 0), turns_per_launch=wl.get("tpl", 0))
    dt = wl["dtype"]
    t_create = time.perf_counter()
    B = phtl.Batch(R, jobs, use_graph=True)
    t_create = time.perf_counter() - t_create
    stream = torch.cuda.current_stream(dev)
    for _ in range(warmup):
        B.run(stream)
    torch.cuda.synchronize()
    info = B.info()
    pt = info.particle_turns_per_run

    def timed():
        evs = []
        for _ in range(steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            B.run(stream)
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in evs]

    st0 = R.stats()
    ms, clk = _clocked(timed)
    launches = R.stats().launches - st0.launches
    t = sum(ms) / 1e3
    slot = phtl.DTYPES[dt]
    value = pt * steps / t
    out = {
        "value": value, "unit": UNIT, "steps": steps, "warmup": warmup,
        "ms_per_step": sum(ms) / len(ms), "dtype": dt,
        "config": {"bunches": len(specs),
                   "particles_total": int(sum(s["n"] for s in specs)),
                   "particle_turns_per_step": pt, "integrator": wl["scheme"],
                   "monitor_stride": wl["stride"], "turn_scale": wl.get("turn_scale", 1.0),
                   "block_threads": info.block_threads[slot],
                   "turns_per_launch": info.turns_per_launch[slot],
                   "launches_per_step": info.launches_per_run, "graph": bool(info.graph),
                   "autotune_probe_pts": info.probe_particle_turns_per_s[slot],
                   "create_s": t_create,
                   "l2": "state ~1 GB (> L2) resident in HBM"},
        "gpu_launches": launches, "clocks": clk,
    }
    if dt != "f64":
        out["roofline"] = issue_roofline(f"k_batched_f32c<{dt}, {wl['scheme']}, monitor>",
                                         (dt, wl["scheme"], False, True, True), value,
                                         clk.get("sm_mhz"))
    else:
        # FP64-pipe roofline at the rate over whole batch runs (many launches per run)
        wlb = dict(wl, transverse=False)
        fpt = alg_flops(wl["scheme"], False, bool(wl["stride"]))
        r = fp64_roofline(f"k_batched_f64<{wl['scheme']}, monitor>", "f64", wl["scheme"], wlb,
                          pt * steps, 1, t, fpt, fpt * value / 1e12)
        r.pop("launch_ms", None)
        r.pop("turns_per_launch", None)
        r["basis"] += "; rate over whole batch runs (CUDA events)"
        out["roofline"] = r
    B.close()
    R.close()
    del keep
    return out


def run_batched(args, wl_name, wl):
    from paper_1610_05801_gb300 import build as _build

    _build.build()
    m = measure_batched(wl, args.steps, args.warmup)
    line = {"metric": METRIC, "value": m.pop("value"), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": m.pop("ms_per_step"),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": m.pop("dtype"), "data": "synthetic (seeded uneven bunches)"}
    m["config"]["workload"] = wl_name
    line.update(m)
    print(json.dumps(line), flush=True)
    return 0


def _play(S, trace, hosts, times, dtype_override=None):
    """Submit the trace's jobs at their arrival times (host buffers in, results in place)
    and wait for all of them; returns the makespan in seconds."""
    from paper_1610_05801_gb300 import phtl

    t0 = time.perf_counter()
    tickets = []
    for j, (z, d), ta in zip(trace, hosts, times):
        now = time.perf_counter() - t0
        if ta > now:
            time.sleep(ta - now)
        tickets.append(S.submit(z, d, turns=j["turns"], integrator=j["integrator"],
                                dtype=dtype_override if dtype_override else j["dtype"],
                                out=[z, d, None, None, None, None]))
    for t in tickets:
        rc, st = S.wait(t, 3_600_000)
        assert rc == phtl.OK and st.state == phtl.DONE, (rc, st.state, st.error)
    return time.perf_counter() - t0


def measure_serving(count, rate_hz=200.0, budget=150e9, load70=False, cd_leg=False, waves=0,
                    f32c_leg=True, f64_leg=True):
    """Serving: the first `count` arrivals of the 2000-arrival Poisson trace (seed 4), through
    the continuous-batching loop with their own arithmetic (FP64 or FP32C); then the same
    jobs every one FP32C through the loop (the batched FP32-compensated serving path), and
    every one FP64 through the plain per-job path (one phtl_track_host call per job, in
    arrival order) -- the comparison the throughput claim rests on.  f32c_leg / f64_leg False
    skip those two legs (long traces)."""
    import numpy as np

    from paper_1610_05801_gb300 import phtl, synth

    trace = synth.serving_trace(seed=4, count=2000, rate_hz=rate_hz)[:count]
    ring = synth.ring(2e6)
    R = phtl.Ring(**ring)
    der = R.derived()
    b = synth.Bucket(k=der.k, A=der.A, etaC=der.etaC, Qs=der.Qs, betagamma=der.betagamma)
    fp64 = []
    for j in trace:
        z, d, _ = synth.matched_bunch(j["seed"], j["n"], b)
        fp64.append((np.ascontiguousarray(z), np.ascontiguousarray(d)))

    def host(dt_of):
        return [(z.copy(), d.copy()) if dt_of(j) == 0 else (phtl.split_f32c(z), phtl.split_f32c(d))
                for j, (z, d) in zip(trace, fp64)]

    arrivals = [j["t_arrive_s"] for j in trace]
    work = sum(j["n"] * j["turns"] for j in trace)

    def served(hosts, times, dtype_override=None):
        S = phtl.Server(R, memory_budget_bytes=int(budget), max_active=64, waves=waves)
        mk, clk = _clocked(lambda: _play(S, trace, hosts, times, dtype_override))
        st = S.stats()
        S.stop()
        return mk, st, clk

    mixed = host(lambda j: j["dtype"])
    mk1, s1, clk = served(mixed, arrivals)
    out = {
        "jobs": len(trace), "trace": "first arrivals of the 2000-arrival Poisson trace (seed 4)",
        "offered_rate_hz": rate_hz, "particle_turns": work, "budget_bytes": budget,
        "max_active": 64, "f64_jobs": sum(1 for j in trace if j["dtype"] == 0),
        "mixed": {"throughput_pts": s1.throughput_pts, "p50_s": s1.p50_latency_s,
                  "p99_s": s1.p99_latency_s, "mean_s": s1.mean_latency_s, "makespan_s": mk1,
                  "rounds": s1.rounds, "bytes_peak": s1.bytes_peak, "gpu_launches": s1.launches,
                  "clocks": clk},
        "e2e": {"value": s1.throughput_pts, "unit": UNIT,
                "h2d_bytes_per_step": int(sum(z.nbytes + d.nbytes for z, d in mixed)),
                "d2h_bytes_per_step": int(sum(z.nbytes + d.nbytes for z, d in mixed)),
                "api": "phtl_submit / phtl_wait on host buffers"},
    }
    if load70:
        cap = s1.throughput_pts
        gaps = np.diff(np.concatenate([[0.0], np.array(arrivals)]))
        scale = (work / len(trace)) / (0.7 * cap) / max(gaps.mean(), 1e-12)
        mk2, s2, _ = served(host(lambda j: j["dtype"]), list(np.cumsum(gaps * scale)))
        out["at_70pct_load"] = {"rate_hz": len(trace) / float(np.sum(gaps * scale)),
                                "throughput_pts": s2.throughput_pts, "p50_s": s2.p50_latency_s,
                                "p99_s": s2.p99_latency_s, "makespan_s": mk2}
    del mixed  # a long trace holds tens of GB of host state per copy
    if not f32c_leg:
        R.close()
        return out
    mk3, s3, clk3 = served(host(lambda j: 1), arrivals, "f32c")
    out["all_jobs_f32c_serving"] = {
        "throughput_pts": s3.throughput_pts, "p50_s": s3.p50_latency_s,
        "p99_s": s3.p99_latency_s, "makespan_s": mk3, "clocks": clk3,
        "arithmetic": "PHTL_F32C: double-float state and sine, FP64 RF phase argument"}
    if cd_leg:
        mk5, s5, _ = served(host(lambda j: 1), arrivals, "f32cd")
        out["all_jobs_f32cd_serving"] = {
            "throughput_pts": s5.throughput_pts, "p50_s": s5.p50_latency_s,
            "p99_s": s5.p99_latency_s, "makespan_s": mk5,
            "arithmetic": "PHTL_F32CD: as F32C with the phase in double-float (a measured "
                          "variant)"}

    def per_job():
        lat = []
        t0 = time.perf_counter()
        for j, (z, d) in zip(trace, fp64):
            now = time.perf_counter() - t0
            if j["t_arrive_s"] > now:
                time.sleep(j["t_arrive_s"] - now)
            zz, dd = z.copy(), d.copy()
            R.track_host(zz, dd, turns=j["turns"], integrator=j["integrator"], dtype="f64")
            lat.append(time.perf_counter() - t0 - j["t_arrive_s"])
        return time.perf_counter() - t0, np.sort(np.array(lat))

    if not f64_leg:
        R.close()
        return out
    (mk4, lat), clk4 = _clocked(per_job)
    out["all_jobs_f64_plain_per_job"] = {
        "throughput_pts": work / mk4, "p50_s": float(np.percentile(lat, 50)),
        "p99_s": float(np.percentile(lat, 99)), "makespan_s": mk4, "clocks": clk4,
        "api": "one phtl_track_host call per job, arrival order"}
    out["f32c_served_over_f64_per_job"] = s3.throughput_pts / (work / mk4)
    R.close()
    return out


def run_serving(args, wl_name, wl):
    from paper_1610_05801_gb300 import build as _build

    _build.build()
    legs = set(args.serving_legs.split(","))
    m = measure_serving(args.serving_jobs or wl["count"], wl["rate_hz"], wl["budget"],
                        load70="load70" in legs, cd_leg="f32cd" in legs,
                        f32c_leg="f32c" in legs, f64_leg="f64" in legs)
    line = {"metric": METRIC, "value": m["mixed"]["throughput_pts"], "unit": UNIT, "n_gpus": 1,
            "steps": 1, "warmup": 0, "ms_per_step": m["mixed"]["makespan_s"] * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "mixed f64/f32c", "data": "synthetic Poisson trace",
            "config": {"workload": wl_name},
            "latency": {"p50_s": m["mixed"]["p50_s"], "p99_s": m["mixed"]["p99_s"]},
            "gpu_launches": m["mixed"]["gpu_launches"], "clocks": m["mixed"]["clocks"],
            "e2e": m.pop("e2e"), "serving": m}
    print(json.dumps(line), flush=True)
    return 0


def hamiltonian(der, z, dp):
    """Smooth single-RF Hamiltonian eta C d^2 / 2 + (A / k)(1 - cos k z) (phi_s = 0)."""
    import numpy as np

    return 0.5 * der.etaC * dp * dp + (der.A / der.k) * (1.0 - np.cos(der.k * z))


def moment_rel_errors(m, mref):
    """Max over rows of the relative moment errors: means relative to the matching rms, rms
    to itself, emittance relative to rms_z * rms_d (longitudinal plane)."""
    import numpy as np

    out = {}
    for name, j, sc in (("mean_z", 0, 2), ("mean_dp", 1, 3), ("rms_z", 2, 2), ("rms_dp", 3, 3)):
        out[name] = float(np.max(np.abs(m[:, j] - mref[:, j]) / np.abs(mref[:, sc])))
    out["eps_z"] = float(np.max(np.abs(m[:, 4] - mref[:, 4]) / (mref[:, 2] * mref[:, 3])))
    out["max"] = max(out.values())
    return out


class OracleThread(threading.Thread):
    """The FP64 oracle tracking a sample on a background host thread (its C loops run
    without the interpreter lock), with a set number of OpenMP threads."""

    def __init__(self, der, scheme, z, dp, turns, stride, threads):
        super().__init__(daemon=True)
        self.args = (der, scheme, z, dp, turns, stride)
        self.threads = threads
        self.ref = None
        self.secs = None
        self.error = None

    def run(self):
        try:
            import oracle

            O = oracle.load()
            O.set_num_threads(self.threads)
            der, scheme, z, dp, turns, stride = self.args
            t0 = time.perf_counter()
            self.ref = O.track(der, scheme, z.copy(), dp.copy(), turns=turns, moments=True,
                               stride=stride)
            self.secs = time.perf_counter() - t0
        except Exception as e:  # reported in the line, never swallowed silently
            self.error = repr(e)


def precision_setup(wl):
    """The precision sweep's ring, bunch (4e6 particles: 60 % matched core, 40 % halo to 98 %
    of the separatrix) and the oracle's constants; the subsample is a prefix."""
    import oracle
    from paper_1610_05801_gb300 import synth

    ring = synth.ring(wl["voltage"])
    O = oracle.load()
    dO = O.derive(ring)
    b = synth.Bucket(k=dO.k, A=dO.A, etaC=dO.etaC, Qs=dO.Qs, betagamma=dO.betagamma)
    z, d = synth.halo_bunch(2, wl["n"], b)
    return ring, dO, z, d


def measure_precision_subsample(wl, ring, z, d, oracle_thread=None):
    """The subsample tracked 1e6 leap-frog turns on the GPU in FP32C, FP32CD, FP32CS and FP64
    (monitor every `stride` turns); moment errors against the FP64 oracle (its result from
    oracle_thread) and against the FP64 GPU path, and the Hamiltonian drift of each."""
    import numpy as np
    import torch

    from paper_1610_05801_gb300 import phtl

    dev = torch.device("cuda", 0)
    R = phtl.Ring(**ring)
    der = R.derived()
    turns, sub, stride = wl["turns"], wl["subsample"], wl["stride"]
    rows = turns // stride + 1
    zs, ds = np.ascontiguousarray(z[:sub]), np.ascontiguousarray(d[:sub])
    res = {}
    for dt in ("f64", "f32c", "f32cd", "f32cs"):
        if dt == "f64":
            bz = torch.tensor(zs, dtype=torch.float64, device=dev)
            bd = torch.tensor(ds, dtype=torch.float64, device=dev)
        else:
            bz = torch.tensor(phtl.split_f32c(zs), dtype=torch.float32, device=dev)
            bd = torch.tensor(phtl.split_f32c(ds), dtype=torch.float32, device=dev)
        mon = torch.zeros((rows, 16), dtype=torch.float64, device=dev)
        R.set_monitor(mon, stride=stride)
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        R.track(bz, bd, turns=turns, integrator="leapfrog", dtype=dt)
        e.record()
        torch.cuda.synchronize()
        R.set_monitor(None)
        zf = bz.cpu().numpy() if dt == "f64" else phtl.join_f32c(bz.cpu().numpy())
        df = bd.cpu().numpy() if dt == "f64" else phtl.join_f32c(bd.cpu().numpy())
        res[dt] = dict(ms=a.elapsed_time(e), z=zf, d=df,
                       mom=phtl.moments_from_sums(mon.cpu().numpy()))
    R.close()
    h0 = hamiltonian(der, zs, ds)
    out = {"subsample": sub, "turns": turns, "monitor_stride": stride, "integrator": "leapfrog",
           "bunch": f"{wl['n']} particles, 60 % matched core + 40 % halo to 98 % of the "
                    f"separatrix, {wl['voltage'] / 1e6:g} MV; the subsample is its first {sub}"}
    ref = None
    if oracle_thread is not None:
        oracle_thread.join()
        if oracle_thread.error:
            out["oracle_error"] = oracle_thread.error
        else:
            ref = oracle_thread.ref
            out["oracle_s"] = oracle_thread.secs
            out["oracle_threads"] = oracle_thread.threads
            hr = hamiltonian(der, ref[0], ref[1])
            out["oracle_hamiltonian_drift_median"] = float(np.median((hr - h0) / h0))
            out["oracle_hamiltonian_drift_abs_max"] = float(np.max(np.abs(hr - h0) / h0))
    for dt, r in res.items():
        h = hamiltonian(der, r["z"], r["d"])
        e = {"kernel_ms_subsample": r["ms"],
             "hamiltonian_drift_median": float(np.median((h - h0) / h0)),
             "hamiltonian_drift_abs_max": float(np.max(np.abs(h - h0) / h0))}
        if ref is not None:
            e["moment_rel_err_vs_oracle"] = moment_rel_errors(r["mom"], ref[6])
            hr = hamiltonian(der, ref[0], ref[1])
            e["hamiltonian_drift_diff_vs_oracle_abs_max"] = float(np.max(np.abs(h - hr) / h0))
        if dt != "f64":
            e["moment_rel_err_vs_f64_gpu"] = moment_rel_errors(r["mom"], res["f64"]["mom"])
            if ref is not None:
                e["meets_1e-4"] = e["moment_rel_err_vs_oracle"]["max"] <= 1e-4
        out[dt] = e
    return out


def default_extras(args):
    """The rest of the headline metric, measured after the FP64 line: the FP32-compensated
    batch of 64 uneven bunches, the precision sweep's moment accuracy after 1e6 turns against
    the FP64 oracle, and the serving trace with its p50/p99 and the FP32C-served against
    FP64-per-job comparison.  The oracle's 1e6-turn run of the precision subsample goes on a
    background host thread (two cores left to the GPU work) while the batch runs."""
    import numpy as np

    out = {}
    pw = dict(WORKLOADS["precision_sweep_4e6x1e6_lf"])
    pw["subsample"] = args.precision_subsample
    ring, dO, z, d = precision_setup(pw)
    sub = pw["subsample"]
    othr = OracleThread(dO, "leapfrog", np.ascontiguousarray(z[:sub]),
                        np.ascontiguousarray(d[:sub]), pw["turns"], pw["stride"],
                        max(1, (os.cpu_count() or 4) - 2))
    othr.start()
    try:
        out["batched_f32c_64_bunches"] = measure_batched(
            WORKLOADS["batched_64_bunches_f32c_lf"], steps=1, warmup=1)
    except Exception as e:
        out["batched_f32c_64_bunches"] = {"error": repr(e)}
    try:
        out["precision_sweep"] = measure_precision_subsample(pw, ring, z, d, othr)
    except Exception as e:
        out["precision_sweep"] = {"error": repr(e)}
    try:
        out["serving"] = measure_serving(args.serving_jobs)
    except Exception as e:
        out["serving"] = {"error": repr(e)}
    return out


def run_precision(args, wl_name, wl):
    """Precision sweep: FP32C / CD / CS at full size (4e6 x 1e6 turns) for throughput, and the
    subsample against the FP64 oracle (with --oracle) and the FP64 GPU path."""
    import numpy as np
    import torch

    from paper_1610_05801_gb300 import build as _build
    from paper_1610_05801_gb300 import phtl

    _build.build()
    dev = torch.device("cuda", 0)
    wl = dict(wl, subsample=args.precision_subsample)
    ring, dO, z, d = precision_setup(wl)
    othr = None
    if args.oracle:
        sub = wl["subsample"]
        othr = OracleThread(dO, "leapfrog", np.ascontiguousarray(z[:sub]),
                            np.ascontiguousarray(d[:sub]), wl["turns"], wl["stride"],
                            max(1, (os.cpu_count() or 4) - 2))
        othr.start()
    R = phtl.Ring(**ring)
    full = {}
    for dt in ("f32c", "f32cd", "f32cs"):
        bz = torch.tensor(phtl.split_f32c(z), dtype=torch.float32, device=dev)
        bd = torch.tensor(phtl.split_f32c(d), dtype=torch.float32, device=dev)
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        R.track(bz, bd, turns=wl["turns"], integrator="leapfrog", dtype=dt)
        e.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(e)
        full[dt] = {"pts": wl["n"] * wl["turns"] / (ms / 1e3), "kernel_ms": ms}
        del bz, bd
    R.close()
    out = {"metric": "moment relative error FP32C vs FP64 after 1e6 turns", "workload": wl_name,
           "n": wl["n"], "turns": wl["turns"], "full_size_longitudinal": full}
    out.update(measure_precision_subsample(wl, ring, z, d, othr))
    print(json.dumps(out), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-sample", type=int, default=CPU_SAMPLE_PARTICLES,
                    help="particles in the oracle's bounded CPU-baseline sample (both arms)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle", action="store_true",
                    help="precision sweep: also re-track the subsample with the FP64 oracle")
    # overrides of the single-bunch workload (profiling captures and sweeps; the headline
    # line uses the workload as defined)
    ap.add_argument("--n", type=int)
    ap.add_argument("--turns", type=int)
    ap.add_argument("--schemes", help="comma-separated integrators")
    ap.add_argument("--dtype", choices=("f64", "f32c", "f32cd", "f32cs"))
    ap.add_argument("--stride", type=int, help="monitor stride (0 = no monitor)")
    ap.add_argument("--no-transverse", action="store_true")
    ap.add_argument("--perturn", action="store_true", help="one launch per turn (HBM-bound variant)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload: print the FP64 line without the FP32C batch, "
                         "precision-sweep and serving keys")
    ap.add_argument("--batch-total", type=float,
                    help="batched workload: total particles (profiling captures; default 6e7)")
    ap.add_argument("--turn-scale", type=float,
                    help="batched workload: scale of every bunch's turns (profiling captures)")
    ap.add_argument("--serving-legs", default="mixed,load70,f32c,f32cd,f64",
                    help="serving workload: the legs to run (the mixed trace always runs)")
    ap.add_argument("--serving-jobs", type=int, default=64,
                    help="serving: the first N arrivals of the 2000-arrival trace")
    ap.add_argument("--precision-subsample", type=int, default=10_000,
                    help="precision sweep: particles compared with the FP64 oracle")
    ap.add_argument("--block", type=int, help="threads per block (default: the library's)")
    ap.add_argument("--turns-per-launch", type=int, help="turns per launch (default: automatic)")
    args = ap.parse_args(argv)
    wl = dict(WORKLOADS[args.workload])
    kind = wl.get("kind", "single")
    if kind == "single":
        for key in ("n", "turns", "dtype", "stride"):
            if getattr(args, key) is not None:
                wl[key] = getattr(args, key)
        if args.schemes:
            wl["schemes"] = tuple(args.schemes.split(","))
        if args.no_transverse:
            wl["transverse"] = False
        wl["perturn"] = args.perturn
        wl["block"] = args.block or 0
        wl["tpl"] = args.turns_per_launch or 0
    if kind == "batched":
        wl["block"] = args.block or 0
        wl["tpl"] = args.turns_per_launch or 0
        if args.batch_total:
            wl["total"] = args.batch_total
        if args.turn_scale:
            wl["turn_scale"] = args.turn_scale
    if args.impl == "reference":
        if kind != "single":
            print(json.dumps({"impl": "reference", "unavailable":
                              "the oracle reference arm covers the single-bunch workload only"}))
            return 0
        return run_reference(args, args.workload, wl)
    if kind == "batched":
        return run_batched(args, args.workload, wl)
    if kind == "serving":
        return run_serving(args, args.workload, wl)
    if kind == "precision":
        return run_precision(args, args.workload, wl)
    return run_ours(args, args.workload, wl)


if __name__ == "__main__":
    sys.exit(main())
