"""GPU parity of the kinetic energy (Algorithm 1's optional energy check) and
of the mixed solver's reference and warm starts, against the FP64 oracle.

Kinetic energy KE = 1/2 sum m |v|^2 over free nodes, with the full-step
velocity of the last iteration.
* FP64 mode runs the oracle's trajectory bit for bit, so the velocities are
  the oracle's and only the sum is reassociated: 1e-12 relative.
* Mixed mode: in the double-float lead, velocities carry ~48 bits but the
  per-node products m|v|^2 are formed in FP32 and summed in double-float, so
  KE is good to a few FP32 roundings per term (~1e-6 relative): bound 1e-5.
  In the FP32 phase the element stiffness about the FP32 reference geometry
  carries a relative error of about ulp(x)/|r| ~ 1e-6 (positions ~0.5, element
  vectors ~0.1-0.5), which shifts every mode's frequency by ~5e-7. At a fixed
  iteration count n the velocity phase then lags by ~n w dt 5e-7 and KE moves
  by up to about twice that: 5e-5 after 40 iterations at w dt ~ 1.3 (the
  chain below); measured 1.2e-4 after 300. The FP32-phase check runs 40
  iterations against a bound of 1e-4. Every comparison is made at a fixed
  iteration count, where KE is far from zero.
"""
import numpy as np
import pytest

import oracle
import rve_inputs as ri

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2305_07030_gb300 import Batch  # noqa: E402
from parity_util import check_equilibrium, envelope_batch, rel_err, within_family  # noqa: E402


def _workload(sizes, seed):
    rng = np.random.default_rng(seed)
    nets = [ri.random_network(int(n), rng) for n in sizes]
    F = np.array([ri.symmetric_perturbation(rng) for _ in nets])
    c = np.array([ri.default_damping(n.n_nodes) for n in nets])
    return ri.Workload("t", nets, F, c)


def _chain():
    """Two fixed ends and one free node between them (one DOF moves)."""
    net = ri.Network(X=np.array([[0.0, 0.0, 0.0], [0.4, 0.0, 0.0], [1.0, 0.0, 0.0]]),
                     elems=np.array([[0, 1], [1, 2]], np.int32), EA=np.array([1.0, 3.0]),
                     fixed=np.array([1, 0, 1], np.uint8))
    return ri.Workload("chain", [net], np.diag([1.1, 1.0, 1.0])[None], np.array([0.05]))


def _ke(w, **opts):
    with Batch(w.nets, damping=w.damping) as b:
        b.solve(w.F, kinetic_energy=True, **opts)
        out = b.stress()
        out["ke"] = b.diagnostics()["kinetic_energy"]
    return out


def _oracle_ke(w, init=1, max_iter=10_000_000):
    return oracle.solve_batch(w, init=init, max_iter=max_iter, want_ke=True)


@pytest.mark.parametrize("max_iter", [60, 10_000_000])
def test_kinetic_energy_fp64(max_iter):
    """FP64: at a fixed iteration count (KE large) and at convergence."""
    w = _workload([37, 300, 777], seed=41)
    ref = _oracle_ke(w, max_iter=max_iter)
    out = _ke(w, precision="fp64", max_iter=max_iter)
    for p, r in enumerate(ref):
        assert out["iters"][p] == r["iters"]
        assert r["ke"] > 0.0
        assert abs(out["ke"][p] - r["ke"]) <= 1e-12 * r["ke"], (p, out["ke"][p], r["ke"])


def test_kinetic_energy_mixed_lead_and_fp32_phase():
    """Mixed: all iterations in the double-float lead, then all in FP32."""
    for w in (_chain(), _workload([150, 400], seed=42)):
        ref = _oracle_ke(w, max_iter=60)
        out = _ke(w, precision="mixed", max_iter=60, lead_tol=0.0)  # 60 lead iterations
        for p, r in enumerate(ref):
            assert out["iters"][p] == 60 and out["status"][p] == "MAXITER"
            assert abs(out["ke"][p] - r["ke"]) <= 1e-5 * r["ke"], (p, out["ke"][p], r["ke"])
        ref = _oracle_ke(w, max_iter=40)
        out = _ke(w, precision="mixed", max_iter=40, lead_iters=0)  # FP32 after one lead step
        for p, r in enumerate(ref):
            assert out["iters"][p] == 40
            assert abs(out["ke"][p] - r["ke"]) <= 1e-4 * r["ke"], (p, out["ke"][p], r["ke"])


def test_mixed_reference_start_against_oracle():
    """Algorithm 1's literal start (free nodes at u = 0), mixed precision."""
    w = _workload([150, 300, 520], seed=43)
    env = envelope_batch(w, init=0)
    with Batch(w.nets, damping=w.damping) as b:
        b.solve(w.F, precision="mixed", init="reference")
        out = b.stress()
        u = b.displacement()
        off = b.node_off
    for p, (r, spread) in enumerate(env):
        assert r["status"] == "OK" and out["status"][p] == "OK"
        res, s_at_u = check_equilibrium(w.nets[p], w.F[p], u[off[p]:off[p + 1]], r["f_ref"], 1e-8)
        assert res <= 1.5e-8, (p, res)
        assert rel_err(out["sigma"][p], s_at_u) <= 1e-12
        e = rel_err(out["sigma"][p], r["sigma"])
        print(f"reference start RVE {p}: err {e:.2e} family diameter {spread:.2e}")
        ok, e, bound = within_family(w.nets[p], w.F[p], w.damping[p], out["sigma"][p], r["sigma"],
                                     spread, init=0)
        assert ok, (p, e, bound)


def test_mixed_warm_start_against_oracle():
    """A second macro step warm-started from the first one's (mixed) result:
    the oracle restarts from the same displacement."""
    w = _workload([300, 700], seed=44)
    F2 = np.array([np.diag([1.005, 1.0, 1.0]) @ f for f in w.F])
    with Batch(w.nets, damping=w.damping) as b:
        b.solve(w.F, precision="mixed")
        first = b.stress()
        u1 = b.displacement()
        b.solve(F2, precision="mixed", init="warm")
        second = b.stress()
        u2 = b.displacement()
        off = b.node_off
    w2 = ri.Workload("t2", w.nets, F2, w.damping)
    env = envelope_batch(w2, init=2, u_warm=[u1[off[p]:off[p + 1]] for p in range(w.n_rve)])
    for p, (r, spread) in enumerate(env):
        assert first["status"][p] == second["status"][p] == r["status"] == "OK"
        res, s_at_u = check_equilibrium(w.nets[p], F2[p], u2[off[p]:off[p + 1]], r["f_ref"], 1e-8)
        assert res <= 1.5e-8, (p, res)
        assert rel_err(second["sigma"][p], s_at_u) <= 1e-12
        e = rel_err(second["sigma"][p], r["sigma"])
        print(f"warm start RVE {p}: err {e:.2e} family diameter {spread:.2e}")
        ok, e, bound = within_family(w.nets[p], F2[p], w.damping[p], second["sigma"][p], r["sigma"],
                                     spread, init=2, u_warm=u1[off[p]:off[p + 1]])
        assert ok, (p, e, bound)


@pytest.mark.parametrize("max_iter", [60, 10_000_000])
def test_energy_balance_fp64(max_iter):
    """Algorithm 1's optional energy check, all three terms (kinetic energy,
    internal work, damping work) against the oracle: FP64 mode runs the
    oracle's trajectory, so only the sums are reassociated (1e-11)."""
    from paper_2305_07030_gb300 import FE2Error
    w = _workload([37, 300, 777, 1500], seed=45)  # 1500 nodes: the cluster kernel
    ref = oracle.solve_batch(w, init=1, max_iter=max_iter, want_energy=True)
    with Batch(w.nets, damping=w.damping) as b:
        b.solve(w.F, precision="fp64", kinetic_energy="balance", max_iter=max_iter)
        out = b.stress()
        e = b.energy()
        for p, r in enumerate(ref):
            assert out["iters"][p] == r["iters"]
            assert abs(e["kinetic"][p] - r["ke"]) <= 1e-11 * r["ke"] + 1e-300
            assert abs(e["internal_work"][p] - r["wint"]) <= 1e-11 * abs(r["wint"])
            assert abs(e["external_work"][p] - r["wext"]) <= 1e-11 * abs(r["wext"])
            bal = (r["ke"] + r["wint"] - r["wext"]) / max(abs(r["wint"]), abs(r["wext"]), r["ke"])
            assert abs(e["balance"][p] - bal) <= 1e-9
        # the work terms are FP64-only; a mixed solve leaves nothing to report
        with pytest.raises(FE2Error):
            b.solve(w.F, precision="mixed", kinetic_energy="balance")
        b.solve(w.F, precision="fp64", kinetic_energy=True, max_iter=5)
        with pytest.raises(FE2Error):
            b.energy()
