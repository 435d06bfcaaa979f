"""Full-size checks: the 64 x 5000-node batch in the launch configuration the
benchmark times (mixed precision, default options), every RVE against the
FP64 oracle's converged stress and the diameter of its rounding family stored
in tests/golden/oracle_stress_rve5000x64.json (written by
tests/golden/make_oracle_stress.py, which runs only the oracle)."""
import json
import os

import numpy as np
import pytest

import rve_inputs as ri

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2305_07030_gb300 import Batch  # noqa: E402
from parity_util import check_equilibrium, mixed_bound, rel_err, within_family  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "oracle_stress_rve5000x64.json")


def test_rve5000x64_every_rve_against_oracle():
    """Every RVE converges, its displacement is an equilibrium by the oracle's
    force law, its stress is the oracle's stress at that displacement, and it
    is within the mixed bound (1e-5, or the diameter of the oracle's own
    rounding family where that is larger) of the oracle's converged stress."""
    with open(GOLDEN) as f:
        gold = json.load(f)["results"]
    w = ri.equal_rves(64, 5000)
    with Batch(w.nets, damping=w.damping) as b:
        b.solve(w.F)  # defaults: mixed precision, affine start, tol 1e-8
        out = b.stress()
        u = b.displacement()
        f_ref = b.diagnostics()["f_ref"]
    off = np.concatenate([[0], np.cumsum([n.n_nodes for n in w.nets])])
    assert all(s == "OK" for s in out["status"])
    assert np.all(out["rel_res"] <= 1e-8)
    rows = []
    for p in range(w.n_rve):
        res, s_at_u = check_equilibrium(w.nets[p], w.F[p], u[off[p]:off[p + 1]], f_ref[p], 1e-8)
        assert res <= 1.5e-8, (p, res)
        assert rel_err(out["sigma"][p], s_at_u) <= 1e-12
        g = gold[p]
        assert g["status"] == "OK"
        assert abs(f_ref[p] - g["f_ref"]) <= 1e-6 * g["f_ref"]
        err = rel_err(out["sigma"][p], np.array(g["sigma"]).reshape(3, 3))
        rows.append((p, err, g["diameter"], err / max(g["diameter"], 1e-300)))
    for r in rows:
        print("RVE %d: stress rel err %.2e, oracle family diameter %.2e, ratio %.2f" % r)
    # beyond the stored 13-run diameter the extended family decides; these
    # networks are multimodal (see test_uneven500_20k_subset_against_oracle),
    # so one RVE in eight may settle in an equilibrium no sampled oracle run
    # reaches; it is still an equilibrium (checked above) and is listed
    bad = []
    for p, err, diam, _ in rows:
        ok, e, bound = within_family(w.nets[p], w.F[p], w.damping[p], out["sigma"][p],
                                     np.array(gold[p]["sigma"]).reshape(3, 3), diam)
        if bound > mixed_bound(diam):
            print("RVE %d: extended family diameter %.2e (error %.2e)" % (p, bound, e))
        if not ok:
            bad.append((p, e, bound))
    print("outside the extended family:", bad)
    assert len(bad) <= len(rows) // 8, bad


GOLD_U4 = os.path.join(os.path.dirname(__file__), "golden", "oracle_stress_uneven500_20k.json")


def test_uneven500_20k_subset_against_oracle():
    """The 64 size-stratified RVEs of the 4096 x log-U(500, 20k) workload (500
    to 20,000 nodes: clusters of 1 to 16 CTAs, kernels with and without their
    shared-memory tables), default options. Every result must be an
    equilibrium of its problem by the oracle's own force law, with the
    oracle's stress at that state. Against the oracle's base run these
    networks are multimodal: an RVE whose 13-run family spans 5e-7 can still
    settle, under other rounding-level differences in the force evaluation,
    into an equilibrium 6e-4 away (one of 16 oracle runs with each element's
    EA moved by 1-4 ulps lands there), so the family check (with its
    extension) is required of seven in eight RVEs and the rest are listed."""
    with open(GOLD_U4) as f:
        gold = json.load(f)
    w = ri.uneven_subset(4096, 500, 20000, 4, gold["rves"])
    with Batch(w.nets, damping=w.damping) as b:
        b.solve(w.F)  # defaults: mixed precision, affine start, tol 1e-8
        out = b.stress()
        u = b.displacement()
        f_ref = b.diagnostics()["f_ref"]
        off = b.node_off
    assert all(s == "OK" for s in out["status"])
    outside = []
    for p, g in enumerate(gold["results"]):
        res, s_at_u = check_equilibrium(w.nets[p], w.F[p], u[off[p]:off[p + 1]], f_ref[p], 1e-8)
        assert res <= 1.5e-8, (p, res)
        assert rel_err(out["sigma"][p], s_at_u) <= 1e-12
        ok, err, bound = within_family(w.nets[p], w.F[p], w.damping[p], out["sigma"][p],
                                       np.array(g["sigma"]).reshape(3, 3), g["diameter"])
        if not ok:
            outside.append((p, g["n_nodes"], err, g["diameter"], bound))
    print("outside the extended family (p, nodes, err, 13-run diameter, extended):", outside)
    assert len(outside) <= len(gold["results"]) // 8, outside
