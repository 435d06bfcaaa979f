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
    # beyond the stored 13-run diameter: the family extended to 25 runs decides
    bad = []
    for p, err, diam, _ in rows:
        ok, e, bound = within_family(w.nets[p], w.F[p], w.damping[p], out["sigma"][p],
                                     np.array(gold[p]["sigma"]).reshape(3, 3), diam)
        if bound > mixed_bound(diam):
            print("RVE %d: extended family diameter %.2e (error %.2e)" % (p, bound, e))
        if not ok:
            bad.append((p, e, bound))
    assert not bad, bad
