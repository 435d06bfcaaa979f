"""The macroscale FE2 driver on the GPU batch (Section I): a 2 x 2 x 2 hex
mesh whose 64 Gauss points each solve a random fiber RVE through the C ABI.
In FP64 mode every RVE solve is the oracle's trajectory bit for bit, so the
whole macroscale loop must reproduce the oracle-driven loop (same outer
iterations, macro displacements to rounding of the stress sums)."""
import numpy as np
import pytest

import rve_inputs as ri
from test_macro import OracleRVEs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2305_07030_gb300 import macro as mc  # noqa: E402


def _nets(m):
    rng = np.random.default_rng(11)
    nets = [ri.random_network(60, rng) for _ in range(m.n_gp)]
    return nets, np.array([ri.default_damping(60) for _ in nets])


def test_fe2_loop_fp64_equals_oracle_loop():
    m = mc.HexMesh(2, 2, 2)
    nets, c = _nets(m)
    steps = [np.diag([1.0 + 0.01 * k, 1.0, 1.0]) for k in (1, 2)]
    ref = mc.FE2Driver(m, OracleRVEs(nets, c, tol=1e-7))
    gpu_rves = mc.BatchRVEs(nets, damping=c, precision="fp64", tol=1e-7)
    try:
        gpu = mc.FE2Driver(m, gpu_rves)
        assert abs(gpu.lam - ref.lam) <= 1e-10 * abs(ref.lam)
        assert abs(gpu.mu - ref.mu) <= 1e-10 * abs(ref.mu)
        for Fm in steps:
            a = ref.step(Fm, tol=1e-5)
            b = gpu.step(Fm, tol=1e-5)
            assert a["converged"] and b["converged"]
            assert a["outer"] == b["outer"]
            assert np.abs(gpu.u - ref.u).max() <= 1e-10 * np.abs(ref.u).max()
            assert np.abs(b["sigma_avg"] - a["sigma_avg"]).max() <= 1e-10 * np.abs(a["sigma_avg"]).max()
    finally:
        gpu_rves.close()


def test_fe2_loop_mixed_converges():
    m = mc.HexMesh(2, 2, 2)
    nets, c = _nets(m)
    rves = mc.BatchRVEs(nets, damping=c, precision="mixed", tol=1e-7)
    try:
        d = mc.FE2Driver(m, rves)
        for k in (1, 2, 3):
            rec = d.step(np.diag([1.0 + 0.01 * k, 1.0, 1.0]), tol=1e-5)
            assert rec["converged"], rec["residuals"]
        # warm restarts: later solves need fewer iterations than the first
        assert np.mean(rves.iters[-1]) < np.mean(rves.iters[1])
    finally:
        rves.close()
