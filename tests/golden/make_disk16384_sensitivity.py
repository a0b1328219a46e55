"""Writes disk16384_oracle_sensitivity.json: how far the oracle's own
100-step run of the 16384-body equal-mass disk (seed 0, dt = 0.01 yr, the
benchmark's workload) moves when every input position is changed by one ulp.

Two oracle runs, identical except for that ulp; the per-body relative
position difference after 100 steps is summarised (maximum and quantiles).
It bounds the agreement any two correct FP64 implementations can reach on
this workload: rounding differences of the order of an ulp grow through the
encounters as this one does.  Calls only the oracle (and the seeded input
generator).  Takes a few minutes on 8 cores:

    python tests/golden/make_disk16384_sensitivity.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import opal_ic as ic  # noqa: E402

STEPS = 100


def main():
    s = ic.equal_mass_disk(0)
    a = oracle.Sim.from_system(s, scan_prune=1)
    b = oracle.Sim.from_system(s, scan_prune=1)
    b.x[:] = np.nextafter(b.x, np.inf)
    for _ in range(STEPS):
        assert a.step(1) == oracle.OK and b.step(1) == oracle.OK
    both = (a.alive > 0) & (b.alive > 0)
    err = np.linalg.norm(a.x[both] - b.x[both], axis=1) / np.linalg.norm(a.x[both], axis=1)
    out = {
        "workload": "equal_mass_disk seed 0, 16384 bodies, dt = 0.01 yr, 3 Hill radii",
        "steps": STEPS,
        "perturbation": "every input position moved by one ulp (nextafter toward +inf) in the second run",
        "max_rel_pos_change": float(err.max()),
        "quantiles": {q: float(np.quantile(err, float(q))) for q in ("0.5", "0.9", "0.99", "0.999")},
        "bodies_above_1e-12": int((err > 1e-12).sum()),
        "bodies": int(both.sum()),
        "script": "tests/golden/make_disk16384_sensitivity.py",
    }
    with open(os.path.join(HERE, "disk16384_oracle_sensitivity.json"), "w") as f:
        json.dump(out, f, indent=2)
        f.write("\n")
    print(json.dumps(out, indent=2))


if __name__ == "__main__":
    main()
