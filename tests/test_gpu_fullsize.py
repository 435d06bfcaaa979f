"""Full-size checks: the 64 x 5000-node batch in the launch configuration the
benchmark times (mixed precision, default options), with sampled RVEs solved
by the FP64 oracle one by one."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
import rve_inputs as ri

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2305_07030_gb300 import Batch  # noqa: E402
from parity_util import check_equilibrium, envelope_batch, rel_err  # noqa: E402


def test_rve5000x64_sampled_against_oracle():
    """Every RVE converges; sampled RVEs (RVE 0 and the four that converge
    fastest, to bound the oracle's time) are checked against the oracle and
    its rounding envelope, and every RVE's displacement is verified as an
    equilibrium by the oracle's force law."""
    w = ri.equal_rves(64, 5000)
    with Batch(w.nets, damping=w.damping) as b:
        b.solve(w.F)  # defaults: mixed precision, affine start, tol 1e-8
        out = b.stress()
        u = b.displacement()
        f_ref = b.diagnostics()["f_ref"]
    off = np.concatenate([[0], np.cumsum([n.n_nodes for n in w.nets])])
    assert all(s == "OK" for s in out["status"])
    assert np.all(out["rel_res"] <= 1e-8)
    for p in range(w.n_rve):
        res, s_at_u = check_equilibrium(w.nets[p], w.F[p], u[off[p]:off[p + 1]], f_ref[p], 1e-8)
        assert res <= 1.5e-8, (p, res)
        assert rel_err(out["sigma"][p], s_at_u) <= 1e-12
    sample = sorted(set([0] + [int(x) for x in np.argsort(out["iters"])[:4]]))
    env = envelope_batch(w, idx=sample, threads=min(16, os.cpu_count() or 1))
    for p, (r, spread) in zip(sample, env):
        err = rel_err(out["sigma"][p], r["sigma"])
        print(f"RVE {p}: stress rel err {err:.2e}, oracle envelope {spread:.2e}, "
              f"iters {out['iters'][p]} vs oracle {r['iters']}")
        assert err <= (1e-5 if spread <= 1e-6 else 10.0 * spread)
