"""Run a seeded workload for a few steps and report what happened.

  python -m paper_2601_19654_gb300.run --workload disk --steps 20 --precision 1 --profile

Workloads (opal_ic): tiny (10 bodies), planetesimals (1000 + Jupiter),
disk (16384 equal masses), heavy (131072 + Jupiter and Saturn), embryos
(1023 embryos and Jupiter with 262144 massless planetesimals; --n sets the
planetesimal count), ensemble (256 systems of 64-4096 bodies).  Prints steps/s, the encounter counters of
the last step, |dE/E| and, with --profile, the device time of every kernel
(each launched alone); with --timeline K, the step graph's kernels as they
ran on the device (a separate build with the device timeline).
"""
from __future__ import annotations

import argparse
import os
import statistics
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import opal_ic as ic  # noqa: E402

WORKLOADS = {
    "tiny": lambda seed, n: ic.tiny(seed, n or 10),
    "planetesimals": lambda seed, n: ic.planetesimals_jupiter(seed, n or 1000),
    "disk": lambda seed, n: ic.equal_mass_disk(seed, n or 16384),
    "heavy": lambda seed, n: ic.encounter_heavy(seed, n or 131072),
    "embryos": lambda seed, n: ic.embryos_planetesimals(seed, 1024, n or 262144),
}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--workload", default="disk", choices=sorted(WORKLOADS) + ["ensemble"])
    ap.add_argument("--n", type=int, default=0, help="body count (workload default if 0)")
    ap.add_argument("--nsys", type=int, default=256, help="systems of the ensemble workload")
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--precision", type=int, default=1, choices=[0, 1])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--profile", action="store_true")
    ap.add_argument("--timeline", type=int, default=0, metavar="K",
                    help="K more steps one at a time in the timeline build: each kernel's first block start "
                         "and last block end on the device, medians over the K steps, from the step's start")
    args = ap.parse_args(argv)

    if args.timeline:
        os.environ["OPAL_TIMELINE_BUILD"] = "1"   # before the library is first loaded
    from paper_2601_19654_gb300 import opal
    from paper_2601_19654_gb300.build import build
    build(timeline=bool(args.timeline))
    if args.workload == "ensemble":
        systems = ic.ensemble(args.seed, nsys=args.nsys)
        sim = opal.Simulation.ensemble(systems, precision=args.precision)
        label = f"ensemble of {len(systems)} systems, {sum(s.n for s in systems)} bodies"
    else:
        s = WORKLOADS[args.workload](args.seed, args.n)
        sim = opal.Simulation.from_system(s, precision=args.precision)
        label = f"{s.name}, {s.n} bodies"
    E0 = sim.energy()[0]
    t0 = time.perf_counter()
    sim.step(args.steps)
    el = time.perf_counter() - t0
    E1 = sim.energy()[0]
    print(f"{label}: precision {args.precision}, {args.steps} steps, {args.steps / el:.1f} steps/s "
          f"(host clock), |dE/E| = {abs(E1 - E0) / abs(E0):.3e}")
    print(f"  kick: {sim.kick_config}; {sim.graph_kernels} kernels per step")
    print(f"  last step: {sim.stats()}")
    if args.profile:
        prof = sim.profile(max(1, min(args.steps, 10)))
        for name, ms in prof.items():
            print(f"  {name:28s} {ms * 1e3:10.1f} us")
    if args.timeline:
        spans = {}
        for _ in range(args.timeline):
            sim.timeline_reset()
            sim.step(1)
            tl = sim.timeline()
            t0 = min(a for a, _ in tl.values())
            for name, (a, b) in tl.items():
                spans.setdefault(name, []).append(((a - t0) * 1e-3, (b - t0) * 1e-3))
        print(f"  device timeline, medians over {args.timeline} steps one at a time (us from the step's start):")
        rows = sorted(((statistics.median(a for a, _ in v), statistics.median(b for _, b in v), k)
                       for k, v in spans.items()))
        for a, b, name in rows:
            print(f"  {name:16s} {a:8.1f} {b:8.1f}  ({b - a:6.1f})")
    sim.close()


if __name__ == "__main__":
    main()
