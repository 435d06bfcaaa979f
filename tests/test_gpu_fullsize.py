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


def test_rve5000x64_sampled_against_oracle():
    w = ri.equal_rves(64, 5000)
    with Batch(w.nets, damping=w.damping) as b:
        b.solve(w.F)  # defaults: mixed precision, affine start, tol 1e-8
        out = b.stress()
    assert all(s == "OK" for s in out["status"])
    assert np.all(out["rel_res"] <= 1e-8)
    # the four RVEs that converge fastest (bounded oracle time), plus RVE 0
    sample = sorted(set([0] + list(np.argsort(out["iters"])[:4])))
    with ThreadPoolExecutor(max_workers=len(sample)) as ex:
        refs = list(ex.map(lambda p: oracle.solve(w.nets[p], w.F[p], w.damping[p], init=1), sample))
    for p, r in zip(sample, refs):
        err = np.linalg.norm(out["sigma"][p] - r["sigma"]) / np.linalg.norm(r["sigma"])
        print(f"RVE {p}: stress rel err {err:.2e}, iters {out['iters'][p]} vs oracle {r['iters']}")
        assert err <= 1e-5
