"""CPU checks of the benchmark's own arithmetic: the per-RVE stress-error
report against stored oracle results, the FP64 ALU lower bound, the
conversion of oracle DOF-iterations into solves, and the workload registry."""
import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import rve_inputs as ri  # noqa: E402


def _args(**kw):
    a = argparse.Namespace(workload="rve5000x64", rves="")
    for k, v in kw.items():
        setattr(a, k, v)
    return a


def test_stress_errors_reproduce_the_stored_results():
    """Feeding the stored oracle stresses back gives zero error; moving one
    RVE by a known relative amount is reported as exactly that."""
    g = bench.golden("rve5000x64")
    sig = np.array([np.array(r["sigma"]).reshape(3, 3) for r in g["results"]])
    st = np.zeros(len(sig), int)
    rep = bench.stress_errors(_args(), sig, st)
    assert rep["available"] and rep["n"] == 64 and rep["max"] == 0.0 and rep["over_bound"] == 0
    moved = sig.copy()
    moved[7] *= 1.0 + 3e-3
    rep = bench.stress_errors(_args(), moved, st)
    assert abs(rep["max"] - 3e-3) < 1e-12 and rep["over_1e-5"] == 1
    assert rep["over_bound"] == int(3e-3 > max(1e-5, g["results"][7]["diameter"]))
    assert bench.stress_errors(_args(rves="1,2"), sig, st)["available"] is False


def test_stress_errors_map_subset_ids_of_the_uneven_workloads():
    """For a full uneven batch the stored subset's RVE ids index the batch."""
    g = bench.golden("uneven500_20k")
    n = 4096
    sig = np.tile(np.eye(3), (n, 1, 1))
    for k, r in enumerate(g["results"]):
        sig[g["rves"][k]] = np.array(r["sigma"]).reshape(3, 3)
    rep = bench.stress_errors(_args(workload="uneven500_20k"), sig, np.zeros(n, int))
    assert rep["n"] == 64 and rep["max"] == 0.0


def test_fp64_alu_seconds_counts_operations():
    """One free node between two fixed ones (two elements, degree 2): 26 + 34
    + 6 add/multiply, 4 + 3 divisions and 2 square roots per iteration."""
    net = ri.Network(X=np.array([[0.0, 0, 0], [0.5, 0, 0], [1.0, 0, 0]]),
                     elems=np.array([[0, 1], [1, 2]], np.int32), EA=np.ones(2),
                     fixed=np.array([1, 0, 1], np.uint8))
    t = bench.fp64_alu_seconds([net], [10], (1.0, 1.0, 1.0))
    assert t == 10 * (66 + 7 + 2)
    t = bench.fp64_alu_seconds([net], [10], (2.0, 7.0, 2.0))
    assert abs(t - 10 * (66 / 2.0 + 7 / 7.0 + 2 / 2.0)) < 1e-12


def test_oracle_dofs_per_solve_from_stored_results():
    g = bench.golden("rve5000x64")
    want = np.mean([3.0 * r["n_nodes"] * r["iters"] for r in g["results"]])
    got, src = bench.oracle_dofs_per_solve("rve5000x64")
    assert got == want and "64" in src


def test_workload_registry_names_stored_results():
    for name, (_, text, gname, ids) in bench.WORKLOADS.items():
        assert text and ids in ("same", "ids")
        assert os.path.exists(os.path.join(ROOT, "tests", "golden", f"oracle_stress_{gname}.json")), name
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "oracle_stress_uneven1k33k.json")))
    assert g["rves"] == ri.stratified_idx(ri.uneven_sizes(1024, 1000, 33000, 3), 64)
