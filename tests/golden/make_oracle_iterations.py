"""Write oracle_iterations.json: the FP64 oracle's own iteration counts to
convergence (tol 1e-8, affine start) for the benchmark workloads.

The CPU-baseline and reference legs of bench.py time the oracle on a bounded
sample (capped iterations) and turn its measured DOF-iterations/s into
solves/s with these counts. Calls only oracle/ and the input generator.
Usage: python tests/golden/make_oracle_iterations.py [threads]
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import rve_inputs as ri  # noqa: E402


def main():
    threads = int(sys.argv[1]) if len(sys.argv) > 1 else (os.cpu_count() or 1)
    out = {"_source": "FP64 oracle (oracle/dr_oracle.c), tol 1e-8, affine start, "
                      "damping 0.002 (512/n)^(1/3); generated by make_oracle_iterations.py"}
    for name, make in (("rve512x1", ri.single_rve_512), ("rve5000x64", lambda: ri.equal_rves(64, 5000))):
        w = make()
        t0 = time.time()
        res = oracle.solve_batch(w, init=1, tol=1e-8, threads=threads)
        out[name] = {"iters": [r["iters"] for r in res],
                     "status": [r["status"] for r in res],
                     "seconds": round(time.time() - t0, 1), "threads": threads}
        print(name, "done", time.time() - t0, flush=True)
    with open(os.path.join(os.path.dirname(__file__), "oracle_iterations.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
