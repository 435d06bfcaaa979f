"""Write oracle_stress_<workload>.json: the FP64 oracle's converged stress,
iteration count and rounding envelope for every RVE of a workload.

The envelope of an RVE is the largest relative (Frobenius) stress change of
the oracle itself when one input of the iteration moves by one unit in the
last place: the time-step factor alpha either way, and the damping
coefficient c either way. Random fiber networks pass bifurcations, and an
RVE whose equilibrium is picked by rounding shows a large envelope; no
implementation with a different rounding order can be held closer to the
oracle than that. The GPU parity tests and the benchmark's per-RVE error
report read these files; every value in them comes from oracle/ alone.

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

import oracle  # noqa: E402
import rve_inputs as ri  # noqa: E402


def rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a - b))


def stratified(sizes, k):
    """k RVE indices spread evenly over the size order (smallest to largest)."""
    order = np.argsort(sizes, kind="stable")
    pick = np.rint(np.linspace(0, len(order) - 1, k)).astype(int)
    return sorted(int(order[i]) for i in pick)


def workload(name):
    if name == "rve5000x64":
        return ri.equal_rves(64, 5000), list(range(64)), "all 64 RVEs"
    if name == "uneven1k33k":
        sizes = ri.uneven_sizes(1024, 1000, 33000, 3)
        idx = stratified(sizes, 64)
        return ri.uneven_subset(1024, 1000, 33000, 3, idx), idx, \
            "64 of 1024 RVEs, stratified by node count"
    if name == "uneven500_20k":
        sizes = ri.uneven_sizes(4096, 500, 20000, 4)
        idx = stratified(sizes, 64)
        return ri.uneven_subset(4096, 500, 20000, 4, idx), idx, \
            "64 of 4096 RVEs, stratified by node count"
    raise SystemExit(f"unknown workload {name}")


def one(w, p, alpha=0.9):
    net, F, c = w.nets[p], w.F[p], w.damping[p]
    base = oracle.solve(net, F, c, tol=1e-8, alpha=alpha, init=1)
    runs = [oracle.solve(net, F, c, tol=1e-8, alpha=a, init=1)
            for a in (np.nextafter(alpha, 1.0), np.nextafter(alpha, 0.0))]
    runs += [oracle.solve(net, F, cc, tol=1e-8, alpha=alpha, init=1)
             for cc in (np.nextafter(c, 1.0), np.nextafter(c, 0.0))]
    env_alpha = max(rel(r["sigma"], base["sigma"]) for r in runs[:2])
    env = max(rel(r["sigma"], base["sigma"]) for r in runs)
    return {"sigma": base["sigma"].reshape(-1).tolist(), "iters": int(base["iters"]),
            "status": base["status"], "f_ref": float(base["f_ref"]),
            "n_nodes": int(net.n_nodes), "envelope_alpha": env_alpha, "envelope": env}


def main():
    name = sys.argv[1]
    threads = int(sys.argv[2]) if len(sys.argv) > 2 else (os.cpu_count() or 1)
    w, idx, what = workload(name)
    t0 = time.time()
    order = sorted(range(w.n_rve), key=lambda p: -w.nets[p].n_nodes)
    res = [None] * w.n_rve
    with ThreadPoolExecutor(max_workers=threads) as ex:
        for p, r in zip(order, ex.map(lambda p: one(w, p), order)):
            res[p] = r
            print(f"RVE {idx[p]}: n={r['n_nodes']} iters={r['iters']} env={r['envelope']:.2e}",
                  flush=True)
    out = {"_source": "FP64 oracle (oracle/dr_oracle.c), tol 1e-8, affine start, damping "
                      "0.002 (512/n)^(1/3); envelope = max relative stress change under a "
                      "one-ulp change of alpha or c; generated by make_oracle_stress.py",
           "workload": name, "rves": idx, "what": what,
           "seconds": round(time.time() - t0, 1), "threads": threads, "results": res}
    with open(os.path.join(os.path.dirname(__file__), f"oracle_stress_{name}.json"), "w") as f:
        json.dump(out, f, indent=0)


if __name__ == "__main__":
    main()
