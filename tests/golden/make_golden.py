"""Write tests/golden/oracle_values.json from the FP64 CPU oracle only.

Run:  python tests/golden/make_golden.py
Values: hit count, weighted yield and the order-free checksums of single
steps of the seeded synthetic workloads.  They let the GPU tests compare
full-size steps without recomputing the oracle, and pin the oracle's FP64
results across host architectures (x86-64 here, aarch64 on the GPU host).
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1608_01125_gb300 import synth  # noqa: E402


def main():
    out = {"_about": "FP64 oracle results; written by tests/golden/make_golden.py", "cases": []}
    wl = synth.tiny_headon()
    a, b = synth.beams(wl)
    _, r = oracle.bruteforce(a, b, 0, wl.dt, wl.kappa)
    out["cases"].append({"workload": wl.name, "n": wl.a.n, "seed": wl.seed, "step": 0,
                         "method": "bruteforce", **{k: r[k] for k in ("count", "weighted")},
                         "hsum": str(r["hsum"]), "hxor": str(r["hxor"])})
    wl = synth.headon_1m()
    a, b = synth.beams(wl)
    for step in (0, 1, 7, 40):
        _, r = oracle.tree(a, b, step, wl.dt, wl.kappa, nthreads=os.cpu_count() or 1,
                           cap=1 << 22)
        out["cases"].append({"workload": wl.name, "n": wl.a.n, "seed": wl.seed, "step": step,
                             "method": "tree", **{k: r[k] for k in ("count", "weighted")},
                             "hsum": str(r["hsum"]), "hxor": str(r["hxor"])})
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_values.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path)


def crossing90(out_path=None):
    """Stored oracle values of the 90-degree crossing workload (2 x 5e7
    photons, 256 steps): three steps drawn with PCG64(0) from the window
    80..176 in which the bunches overlap.  Slow: run by hand
    (python tests/golden/make_golden.py crossing90)."""
    import numpy as np
    wl = synth.crossing90_5e7()
    a, b = synth.beams(wl)
    steps = sorted(int(s) for s in np.random.default_rng(0).choice(np.arange(80, 177), 3,
                                                                    replace=False))
    out = {"_about": "FP64 oracle (k-d tree) results; written by tests/golden/make_golden.py",
           "cases": []}
    for step in steps:
        _, r = oracle.tree(a, b, step, wl.dt, wl.kappa, nthreads=os.cpu_count() or 1,
                           cap=1 << 24)
        out["cases"].append({"workload": wl.name, "n": wl.a.n, "seed": wl.seed, "step": step,
                             "method": "tree", "count": r["count"], "weighted": r["weighted"],
                             "hsum": str(r["hsum"]), "hxor": str(r["hxor"])})
        print(out["cases"][-1], flush=True)
    path = out_path or os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                    "oracle_values_crossing90.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path)


def headon_run(out_path=None):
    """Stored oracle values of every time step of the 2 x 1,048,576 head-on run
    (64 steps of 5 fs): the per-step count, weighted yield and checksums whose
    sums over the run the captured run (trilens_run) must reproduce.  Slow: run
    by hand (python tests/golden/make_golden.py headon_run)."""
    wl = synth.headon_1m()
    a, b = synth.beams(wl)
    out = {"_about": "FP64 oracle (k-d tree) results of every time step; written by "
                     "tests/golden/make_golden.py", "workload": wl.name, "n": wl.a.n,
           "seed": wl.seed, "steps": []}
    for step in range(wl.steps):
        _, r = oracle.tree(a, b, step, wl.dt, wl.kappa, nthreads=os.cpu_count() or 1,
                           cap=1 << 22)
        out["steps"].append({"step": step, "count": r["count"], "weighted": r["weighted"],
                             "hsum": str(r["hsum"]), "hxor": str(r["hxor"])})
        print(out["steps"][-1], flush=True)
    path = out_path or os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                    "oracle_values_headon_run.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path)


if __name__ == "__main__":
    if len(sys.argv) > 1 and sys.argv[1] == "crossing90":
        crossing90()
    elif len(sys.argv) > 1 and sys.argv[1] == "headon_run":
        headon_run()
    else:
        main()

