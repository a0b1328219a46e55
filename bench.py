#!/usr/bin/env python3
"""Benchmark of the hybrid symplectic N-body step on GB300.

Workload: 16384 fully interacting equal-mass bodies (1e-3 Earth masses,
a uniform in 0.5-3 au, e and i Rayleigh 0.01 / 0.005, radii from 2 g/cm^3),
dt = 0.01 yr, critical radius 3 Hill radii; synthetic, seeded (opal_ic).
A step is one full pass of the method: kick, jump, drift, encounter scan,
Bulirsch-Stoer of the flagged groups, jump, kick.

Prints one JSON line.  `value` is the mixed form's steps/s summed over
ranks (each rank advances its own replica: independent systems, no
collective on the data path); the FP64 form, interactions/s, |dE/E|, the
kick's roofline (against the nominal FP32 peak and the device's measured
ALU peaks), the end-to-end rate through the C ABI with host buffers, the
256-system ensemble, the small-body, removal and encounter-heavy
workloads, clocks and the oracle's CPU rate are reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
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

import opal_ic as ic  # noqa: E402

METRIC = "steps/s and pair interactions/s at N=16384, mixed vs FP64 form, |dE/E| stated"
UNIT = "steps/s"
N_SMS = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0
# algorithmic FP32 flops of one pair interaction of the kick (FMA = 2):
# 3 subtractions, r^2 (1 mul + 2 fma = 5), rsqrt (1), m r^-3 (3 mul), 3 fma (6)
FLOPS_PER_INTERACTION = 18
# DRAM bytes (read + written) of one launch of the mixed kick, from the ncu
# capture summarised in profiles/kick_mixed_disk16384.md (launch shape
# "mixed t128 i1 6" with the step graph's 912 blocks); the other one-i-body
# shapes run the same code with another register cap, so they move the same
# bytes.  Other shapes report none.
_KICK_I1_TRAFFIC = 0.821248e6 + 0.0
KICK_TRAFFIC = {"mixed t128 i1": _KICK_I1_TRAFFIC, "mixed t128 i1 6": _KICK_I1_TRAFFIC,
                "mixed t128 i1 8": _KICK_I1_TRAFFIC}


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--fp64-steps", type=int, default=20)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the ensemble vs per-system comparison")
    ap.add_argument("--ensemble-steps", type=int, default=10)
    ap.add_argument("--no-small", action="store_true", help="skip the small-body (planetesimal) workload")
    ap.add_argument("--small-steps", type=int, default=50)
    ap.add_argument("--no-removals", action="store_true", help="skip the star-collision / ejection run")
    ap.add_argument("--no-heavy", action="store_true", help="skip the encounter-heavy 131072-body run")
    ap.add_argument("--heavy-steps", type=int, default=3)
    ap.add_argument("--seed", type=int, default=0)
    return ap.parse_args(argv)


# ---------------------------------------------------------------- ranks
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def job_rate(local_ms_total: float, steps: int, world: int) -> tuple[float, float]:
    """Whole-job steps/s of N replicas that each ran `steps` steps: the job took
    as long as its slowest rank, and every rank advanced its own system."""
    total_ms = max_over_ranks(local_ms_total, world)
    return world * steps / (total_ms * 1e-3), total_ms


def max_over_ranks(value: float, world: int) -> float:
    """Largest value over ranks (the job's time is the slowest rank's)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu = gpu_id
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [t.strip() for t in line.split(",")]
                if len(f) >= 9 and f[1].replace(".", "").isdigit():
                    rows.append(f)
        finally:
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3] not in ("[N/A]", ""))}


# ---------------------------------------------------------------- timing
def time_steps(sim, steps: int, warmup: int, flush):
    """Device time of each step (CUDA events on the simulation's stream,
    L2 flushed before each step) and of its kick kernel (events captured in
    the step graph on the same stream)."""
    import torch
    stream = torch.cuda.ExternalStream(sim.stream)
    sim.step(warmup)
    sim.time_kick(True)
    step_ms, kick_ms = [], []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
            ev[k][0].record(stream)
        sim.step_async(1)
        with torch.cuda.stream(stream):
            ev[k][1].record(stream)
        kick_ms.append(sim.last_kick_ms())
    sim.wait()
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    sim.time_kick(False)
    return step_ms, kick_ms


def e2e_rate(system, steps: int, precision: int):
    """Steps/s through the public API with host buffers: create from host
    arrays (host->device, with the kick autotuning and the step graph's
    capture), then every step opal_step and opal_get_state (device->host of
    ids, masses, positions, velocities, radii).  The value covers create and
    the steps; create's time and the per-step rate are reported beside it."""
    from paper_2601_19654_gb300 import opal
    n = system.n
    t0 = time.perf_counter()
    sim = opal.Simulation.from_system(system, precision=precision)
    t1 = time.perf_counter()
    for _ in range(steps):
        sim.step(1)
        st = sim.state()
    t2 = time.perf_counter()
    sim.close()
    assert st["x"].shape[0] > 0
    h2d = n * 8 * (1 + 3 + 3 + 1)
    d2h = n * (8 + 8 + 24 + 24 + 8)
    return {"value": steps / (t2 - t0), "unit": UNIT, "steps": steps, "h2d_bytes_per_step": h2d / steps,
            "d2h_bytes_per_step": d2h, "create_ms": (t1 - t0) * 1e3, "steps_per_s_after_create": steps / (t2 - t1),
            "note": "host clock; create (H2D of the state, kick autotuning, graph capture) and the steps, each "
                    "step followed by the state read back to host"}


def ensemble_rates(seed: int, steps: int, warmup: int):
    """The 256-system ensemble (N log-uniform in 64-4096, each drawn like the
    10-body workload) advanced as one simulation, against the same systems as
    256 simulations of their own: launched one after another (each step
    waits for its system), and launched all at once on their own streams.
    All rates are ensemble steps/s (every system advanced one step).  The
    ensemble and the 256 streams are timed with CUDA events (the streams
    start from one event and a final event waits for all of them); the
    one-after-another arm, whose steps each end in a host wait, by the host
    clock."""
    import torch
    from paper_2601_19654_gb300 import opal
    systems = ic.ensemble(seed, 256)
    ens = opal.Simulation.ensemble(systems, precision=1)
    E0 = ens.energy()[0]
    ens.step(warmup)
    es = torch.cuda.ExternalStream(ens.stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(es)
    ens.step_async(steps)
    e1.record(es)
    ens.wait()
    e1.synchronize()
    t_ens = e0.elapsed_time(e1) * 1e-3
    dE = abs(ens.energy()[0] - E0) / abs(E0)
    st = ens.stats()
    ens.close()
    per = [opal.Simulation.from_system(s, precision=1) for s in systems]
    for sim in per:
        sim.step(warmup)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        for sim in per:
            sim.step(1)
    t_serial = time.perf_counter() - t0
    streams = [torch.cuda.ExternalStream(sim.stream) for sim in per]
    head = torch.cuda.Stream()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s0.record(head)
    for sim, st_ in zip(per, streams):
        st_.wait_event(s0)
    for _ in range(steps):
        for sim in per:
            sim.step_async(1)
    for st_ in streams:
        ev = torch.cuda.Event()
        ev.record(st_)
        head.wait_event(ev)
    s1.record(head)
    for sim in per:
        sim.wait()
    s1.synchronize()
    t_async = s0.elapsed_time(s1) * 1e-3
    for sim in per:
        sim.close()
    r_ens, r_ser, r_asy = steps / t_ens, steps / t_serial, steps / t_async
    return {"workload": "256 systems, N log-uniform 64-4096 (each like the 10-body workload), mixed form",
            "bodies": int(sum(s.n for s in systems)), "steps": steps, "warmup": warmup,
            "ensemble_steps_per_s": r_ens, "per_system_serial_steps_per_s": r_ser,
            "per_system_streams_steps_per_s": r_asy, "over_serial": r_ens / r_ser,
            "over_streams": r_ens / r_asy, "dE_over_E": dE, "encounters_last_step": st,
            "timing": "CUDA events for the ensemble and the 256 streams; host clock for the steps one after another"}


def removal_rates(system, steps: int, warmup: int, flush, plain_ms: float):
    """The headline workload with star collisions and ejections on, at the
    paper's settings (Sec. 2.1.2: bodies beyond 400 au removed every 200 yr;
    the star's radius 0.00465 au): the cost of the removal stages, which run
    every step (and return at once when nothing is removed)."""
    from paper_2601_19654_gb300 import opal
    every = int(round(200.0 / 0.01))
    sim = opal.Simulation.from_system(system, precision=1, r_star=0.00465, r_eject=400.0, eject_every=every)
    step_ms, _ = time_steps(sim, steps, warmup, flush)
    kernels = sim.graph_kernels
    sim.close()
    ms = float(np.mean(step_ms))
    return {"r_star_au": 0.00465, "r_eject_au": 400.0, "eject_every": every, "steps_per_s": 1e3 / ms,
            "ms_per_step": ms, "overhead_vs_value": ms / plain_ms - 1.0, "kernels_per_step": kernels}


def small_body_rates(seed: int, steps: int, warmup: int, flush):
    """The production regime of the paper's Sec. 2.1: 1023 embryos and Jupiter
    (big bodies) with 262144 massless planetesimals (small bodies), mixed
    form, device-timed like the headline.  Each step costs (N_big + N_small)
    x N_big kick interactions (small bodies are sources of nothing)."""
    from paper_2601_19654_gb300 import opal
    system = ic.embryos_planetesimals(seed)
    nb, n = system.meta["n_big"], system.n
    sim = opal.Simulation.from_system(system, precision=1)
    E0 = sim.energy()[0]
    step_ms, kick_ms = time_steps(sim, steps, warmup, flush)
    dE = abs(sim.energy()[0] - E0) / abs(E0)
    st = sim.stats()
    kcfg = sim.kick_config
    sim.close()
    ms = float(np.mean(step_ms))
    inter = n * nb - nb
    return {"workload": system.name, "n_big": nb, "n_small": n - nb, "steps": steps, "warmup": warmup,
            "steps_per_s": 1e3 / ms, "ms_per_step": ms, "interactions_per_step": inter,
            "interactions_per_s": inter * 1e3 / ms, "kick_ms": float(np.mean(kick_ms)), "kick": kcfg,
            "dE_over_E": dE, "encounters_last_step": st,
            "timing": "CUDA events on the simulation's stream, L2 flushed before every step"}


def heavy_rates(seed: int, steps: int, warmup: int, flush):
    """The encounter-heavy stress workload: 131072 bodies of 1e-4 Earth
    masses between 2 and 10 au with Jupiter and Saturn, radii inflated
    tenfold, dt = 0.05 yr; mixed form, device-timed like the headline.  Its
    steps are bound by the Bulirsch-Stoer of the giants' encounter groups
    (hundreds to thousands of members, the whole-GPU kernel)."""
    from paper_2601_19654_gb300 import opal
    system = ic.encounter_heavy(seed)
    n = system.n
    sim = opal.Simulation.from_system(system, precision=1)
    E0 = sim.energy()[0]
    step_ms, kick_ms = time_steps(sim, steps, warmup, flush)
    dE = abs(sim.energy()[0] - E0) / abs(E0)
    st = sim.stats()
    sim.close()
    ms = float(np.mean(step_ms))
    return {"workload": system.name, "bodies": n, "steps": steps, "warmup": warmup, "steps_per_s": 1e3 / ms,
            "ms_per_step": ms, "interactions_per_s": n * (n - 1) * 1e3 / ms, "kick_ms": float(np.mean(kick_ms)),
            "dE_over_E": dE, "encounters_last_step": st,
            "timing": "CUDA events on the simulation's stream, L2 flushed before every step"}


def oracle_rate(system, seconds: float, max_steps: int | None = None):
    """Steps/s of the oracle on this host's cores for about `seconds`; its
    scan skips the pairs its end-point bound rules out (the same flagged set
    as its all-pairs test).  Also returns its state, to compare against."""
    import oracle
    oracle.build()
    sim = oracle.Sim.from_system(system, scan_prune=1)
    E0 = sim.energy()[0]
    t0 = time.perf_counter()
    done = 0
    while True:
        assert sim.step(1) == oracle.OK
        done += 1
        el = time.perf_counter() - t0
        if (el >= seconds and done >= 2) or (max_steps and done >= max_steps):
            break
    dE = abs(sim.energy()[0] - E0) / abs(E0)
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return done / el, done, el, threads, dE, sim


def relpos(a, b):
    """Largest relative position error of a against b (rows are bodies)."""
    return float(np.max(np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)))


def gpu_vs_oracle(system, steps: int, osim):
    """Both GPU forms over the oracle's `steps` steps from the same inputs:
    relative position error against the oracle's state and |dE/E|."""
    from paper_2601_19654_gb300 import opal
    alive = np.nonzero(osim.alive)[0]
    out = {"steps": steps}
    for name, prec in (("mixed", 1), ("fp64", 0)):
        with opal.Simulation.from_system(system, precision=prec) as sim:
            E0 = sim.energy()[0]
            sim.step(steps)
            st = sim.state()
            out[f"dE_over_E_{name}"] = abs(sim.energy()[0] - E0) / abs(E0)
            out[f"pos_err_{name}"] = (relpos(st["x"], osim.x[alive]) if st["ids"].tolist() == alive.tolist()
                                      else None)
    return out


# ---------------------------------------------------------------- main
def run_reference(args, rank, world):
    if rank != 0:
        return
    system = ic.equal_mass_disk(args.seed)
    import oracle
    oracle.build()
    sim = oracle.Sim.from_system(system, scan_prune=1)
    warm = min(args.warmup, 3)   # each oracle step of this system takes about a second
    for _ in range(warm):
        sim.step(1)
    budget = 120.0
    t0 = time.perf_counter()
    done = 0
    while done < args.steps and (time.perf_counter() - t0) < budget:
        assert sim.step(1) == oracle.OK
        done += 1
    el = time.perf_counter() - t0
    v = done / el
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": done, "warmup": warm, "ms_per_step": 1e3 / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": system.name, "bodies": system.n, "form": "FP64 serial oracle (C, OpenMP kick)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{done} full steps of the 16384-body system ({el:.1f} s; the scan "
                                       "skips pairs by its end-point bound)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "interactions_per_s": v * system.n * (system.n - 1)}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local):
    import torch
    from paper_2601_19654_gb300 import opal
    from paper_2601_19654_gb300.build import build
    if local == 0:
        build()
    barrier(world)
    system = ic.equal_mass_disk(args.seed + rank)
    n = system.n
    pairs = n * (n - 1)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    # mixed form (the headline)
    sim = opal.Simulation.from_system(system, precision=1)
    kick_cfg = sim.kick_config
    kernels_per_step = sim.graph_kernels
    E0 = sim.energy()[0]
    barrier(world)
    visible = [t for t in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if t.strip()]
    gpu_id = visible[local] if local < len(visible) else str(local)
    with ClockSampler(gpu_id) as clk:
        step_ms, kick_ms = time_steps(sim, args.steps, args.warmup, flush)
    value, total_ms = job_rate(float(np.sum(step_ms)), args.steps, world)
    dE_mixed = abs(sim.energy()[0] - E0) / abs(E0)
    last = sim.stats()
    mixed_state = sim.state()
    # the same kick kernel launched alone on the state the timed run left
    kick_alone = sim.kick_alone_ms(20)
    step_order = "overlap" if os.environ.get("OPAL_STEP_ORDER", "") != "inorder" else "inorder"
    sim.close()
    ms_per_step = total_ms / args.steps
    # the FP64 form over the same steps from the same inputs: the mixed
    # form's position error against it
    with opal.Simulation.from_system(system, precision=0) as ref64:
        ref64.step(args.warmup + args.steps)
        ref_state = ref64.state()
    pos_err_vs_fp64 = (relpos(mixed_state["x"], ref_state["x"])
                       if mixed_state["ids"].tolist() == ref_state["ids"].tolist() else None)

    # FP64 form, same workload
    sim64 = opal.Simulation.from_system(system, precision=0)
    E064 = sim64.energy()[0]
    s64, k64 = time_steps(sim64, args.fp64_steps, 3, flush)
    dE_fp64 = abs(sim64.energy()[0] - E064) / abs(E064)
    sim64.close()
    ms64 = max_over_ranks(float(np.mean(s64)), world)

    # measured ALU peaks of this device (FP32 and FP64 FMA chains, MUFU rsqrt),
    # beside the nominal FP32 peak
    try:
        alu = opal.probe_alu_peaks()
    except opal.OpalError:
        alu = None

    kick_avg = float(np.mean(kick_ms))
    kick64_avg = float(np.mean(k64))
    flops = FLOPS_PER_INTERACTION * pairs
    peak = N_SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    achieved = flops / (kick_alone * 1e-3) / 1e12
    achieved_graph = flops / (kick_avg * 1e-3) / 1e12
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": system.name, "bodies": n, "form": "mixed (FP32 pair kick, FP64 drift/BS)",
                   "dt_yr": 0.01, "rcrit_hill": 3.0, "l2": "flushed (256 MiB memset) before every timed step",
                   "replicas": world, "kick": kick_cfg},
        "interactions_per_s": value * pairs,
        "dE_over_E": {"mixed": dE_mixed, "fp64": dE_fp64,
                      "over_steps": {"mixed": args.warmup + args.steps, "fp64": 3 + args.fp64_steps}},
        "pos_err_vs_fp64": {"value": pos_err_vs_fp64, "steps": args.warmup + args.steps,
                            "note": "max relative position error of the mixed run against the FP64 GPU form "
                                    "after the same steps from the same inputs"},
        "fp64": {"value": world * 1e3 / ms64, "unit": UNIT, "ms_per_step": ms64,
                 "interactions_per_s": world * 1e3 / ms64 * pairs, "kick_ms": kick64_avg,
                 "steps": args.fp64_steps, "kick_fp64_tflops": flops / (kick64_avg * 1e-3) / 1e12,
                 "kick_frac_of_measured_fp64": (flops / (kick64_avg * 1e-3) / 1e12 / alu["fp64_tflops"]
                                                if alu else None)},
        "mixed_over_fp64": ms64 / ms_per_step,
        "encounters_last_step": last,
        "roofline": {"bound": "alu", "kernel": "kick (mixed)", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": KICK_TRAFFIC.get(kick_cfg.split(",")[0]),
                     "note": f"{FLOPS_PER_INTERACTION} FP32 flops per pair x N(N-1) pairs per launch; "
                             "peak = 152 SMs x 128 FP32 lanes x 2 x 2070 MHz (of nominal max clock); "
                             "achieved: the step's kick kernel launched alone 20 times on the state the "
                             "timed run left (CUDA events on the simulation's stream); in_graph: the same "
                             "kernel timed inside the step graph over the timed steps, where it runs "
                             "beside the encounter integrator",
                     "kick_ms": kick_alone, "measured_alu_peaks": alu,
                     "frac_of_measured_fp32": achieved / alu["fp32_tflops"] if alu else None,
                     "in_graph": {"kick_ms": kick_avg, "achieved": achieved_graph, "frac": achieved_graph / peak,
                                  "frac_of_measured_fp32": achieved_graph / alu["fp32_tflops"] if alu else None,
                                  "kick_share_of_step": kick_avg / float(np.mean(step_ms)),
                                  "step_order": step_order}},
        "gpu_launches": kernels_per_step * args.steps,
        "clocks": clocks,
    }
    if rank == 0:
        line["e2e"] = e2e_rate(system, max(300, args.steps), precision=1)
        if not args.no_ensemble:
            line["ensemble"] = ensemble_rates(args.seed, args.ensemble_steps, 3)
        if not args.no_small:
            line["small_bodies"] = small_body_rates(args.seed, args.small_steps, 5, flush)
        if not args.no_heavy:
            line["encounter_heavy"] = heavy_rates(args.seed, args.heavy_steps, 1, flush)
        if not args.no_removals:
            line["removals"] = removal_rates(system, min(args.steps, 100), 5, flush, ms_per_step)
        if not args.no_cpu_baseline:
            v, done, el, threads, dE, osim = oracle_rate(system, args.cpu_seconds)
            line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                                    "sample": f"{done} full steps of the {n}-body system ({el:.1f} s; the scan "
                                              "skips pairs by its end-point bound)",
                                    "dE_over_E": dE}
            # the FP64 oracle over those steps against both GPU forms
            cmp = gpu_vs_oracle(system, done, osim)
            cmp["dE_over_E_oracle"] = dE
            line["vs_oracle"] = cmp
        print(json.dumps(line), flush=True)


def main(argv=None):
    args = parse_args(argv)
    rank, world, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
