"""Write oracle_stress_<workload>.json: the FP64 oracle's converged stress,
iteration count and rounding family for every RVE of a workload.

An RVE's rounding family is the set of stresses the oracle itself reaches
when alpha or the damping coefficient c moves by 1, 2 or 3 units in the last
place either way (12 runs beside the base run; tests/parity_util.py defines
the set). Random fiber networks carry floppy modes, and the relaxation can
settle anywhere on a family of equilibria; which one is decided by rounding.
Per RVE the file holds the base run's stress, iteration count and f_ref, the
family's largest distance from the base run ("envelope") and its diameter
(largest distance between two members, both relative to the base stress).
The GPU parity tests and the benchmark's per-RVE error report read these
files; every value in them comes from oracle/ alone.

Usage: python tests/golden/make_oracle_stress.py WORKLOAD [threads]
  WORKLOAD: rve5000x64 (all 64 RVEs), uneven1k33k (64 RVEs of the
  1024 x log-U(1k,33k) workload, stratified by size), uneven500_20k (64 RVEs
  of the 4096 x log-U(500,20k) workload, stratified by size)
"""
import json
import os
import sys
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402
import rve_inputs as ri  # noqa: E402
from parity_util import family_diameter, perturbations  # noqa: E402

ALPHA = 0.9


def rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a - b))


def workload(name):
    if name == "rve5000x64":
        return ri.equal_rves(64, 5000), list(range(64)), "all 64 RVEs"
    if name == "rve512x1":
        return ri.single_rve_512(), [0], "the single 512-node RVE"
    if name == "uneven1k33k":
        sizes = ri.uneven_sizes(1024, 1000, 33000, 3)
        idx = ri.stratified_idx(sizes, 64)
        return ri.uneven_subset(1024, 1000, 33000, 3, idx), idx, \
            "64 of 1024 RVEs, stratified by node count"
    if name == "uneven500_20k":
        sizes = ri.uneven_sizes(4096, 500, 20000, 4)
        idx = ri.stratified_idx(sizes, 64)
        return ri.uneven_subset(4096, 500, 20000, 4, idx), idx, \
            "64 of 4096 RVEs, stratified by node count"
    raise SystemExit(f"unknown workload {name}")


def main():
    name = sys.argv[1]
    threads = int(sys.argv[2]) if len(sys.argv) > 2 else (os.cpu_count() or 1)
    w, idx, what = workload(name)
    t0 = time.time()
    # one job per (RVE, run); the largest RVEs first
    jobs = []
    for p in sorted(range(w.n_rve), key=lambda p: -w.nets[p].n_nodes):
        jobs.append((p, ALPHA, float(w.damping[p])))
        jobs += [(p, a, cc) for a, cc in perturbations(ALPHA, float(w.damping[p]))]

    def run(j):
        p, a, cc = j
        return oracle.solve(w.nets[p], w.F[p], cc, tol=1e-8, alpha=a, init=1)

    runs = {}
    with ThreadPoolExecutor(max_workers=threads) as ex:
        for j, r in zip(jobs, ex.map(run, jobs)):
            runs.setdefault(j[0], []).append(r)
            if len(runs[j[0]]) == 13:
                print(f"RVE {idx[j[0]]}: done ({time.time() - t0:.0f} s)", flush=True)
    res = []
    for p in range(w.n_rve):
        base, rest = runs[p][0], runs[p][1:]
        sig = [base["sigma"]] + [r["sigma"] for r in rest]
        res.append({"sigma": base["sigma"].reshape(-1).tolist(), "iters": int(base["iters"]),
                    "status": base["status"], "f_ref": float(base["f_ref"]),
                    "n_nodes": int(w.nets[p].n_nodes),
                    "envelope": max(rel(s, base["sigma"]) for s in sig[1:]),
                    "diameter": family_diameter(sig, base["sigma"]),
                    "family_iters": [int(r["iters"]) for r in rest],
                    "family_status": sorted({r["status"] for r in rest})})
        print(f"RVE {idx[p]}: n={res[-1]['n_nodes']} iters={res[-1]['iters']} "
              f"env={res[-1]['envelope']:.2e} diam={res[-1]['diameter']:.2e}", flush=True)
    out = {"_source": "FP64 oracle (oracle/dr_oracle.c), tol 1e-8, affine start, damping "
                      "0.002 (512/n)^(1/3); family = base run plus alpha or c moved by 1..3 "
                      "ulps either way; envelope = largest relative stress change from the "
                      "base run, diameter = largest relative difference between two family "
                      "members; generated by make_oracle_stress.py",
           "workload": name, "rves": idx, "what": what,
           "seconds": round(time.time() - t0, 1), "threads": threads, "results": res}
    with open(os.path.join(os.path.dirname(__file__), f"oracle_stress_{name}.json"), "w") as f:
        json.dump(out, f, indent=0)


if __name__ == "__main__":
    main()
