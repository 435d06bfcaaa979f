"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

FP64 mode follows the oracle's operations in the oracle's order, so the
trajectory must be bit-identical: equal iteration counts and equal
displacements; only the stress sum is reassociated (1e-12 relative).
Mixed mode must stay within 1e-5 relative stress error (Frobenius norm) of
the oracle, or within the diameter of the oracle's own rounding family where
that is larger (see parity_util), and must land on a true equilibrium.
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


def _workload(sizes, seed, ea="lognormal", Fscale=0.02):
    rng = np.random.default_rng(seed)
    nets = [ri.random_network(int(n), rng, ea=ea) for n in sizes]
    F = np.array([ri.symmetric_perturbation(rng, Fscale) for _ in nets])
    c = np.array([ri.default_damping(n.n_nodes) for n in nets])
    return ri.Workload("t", nets, F, c)


def _solve(w, **opts):
    with Batch(w.nets, damping=w.damping) as b:
        b.solve(w.F, **opts)
        out = b.stress()
        out["u"] = b.displacement()
        out["node_off"] = b.node_off
    return out


@pytest.mark.parametrize("init", ["affine", "reference"])
def test_fp64_bitwise_trajectory(init):
    """Several RVEs (many nodes per thread, ragged tails, uneven sizes)."""
    w = _workload([37, 300, 777, 1500], seed=11)
    iv = {"affine": 1, "reference": 0}[init]
    ref = oracle.solve_batch(w, init=iv, tol=1e-8, max_iter=300000)
    out = _solve(w, precision="fp64", init=init, tol=1e-8, max_iter=300000)
    for p, r in enumerate(ref):
        a, b = out["node_off"][p], out["node_off"][p + 1]
        assert out["status"][p] == r["status"]
        assert out["iters"][p] == r["iters"], (p, out["iters"][p], r["iters"])
        assert np.array_equal(out["u"][a:b], r["u"]), np.abs(out["u"][a:b] - r["u"]).max()
        assert rel_err(out["sigma"][p], r["sigma"]) <= 1e-12
        assert abs(out["rel_res"][p] - r["rel_res"]) <= 1e-12 * max(r["rel_res"], 1e-300) + 1e-300


def test_fp64_global_scratch_class_and_maxiter(monkeypatch):
    """An RVE too big to stage in shared memory on one CTA runs from L2
    scratch when the cluster kernel is switched off; the trajectory is still
    the oracle's (checked after a fixed iteration cap)."""
    monkeypatch.setenv("FE2_FP64_CLUSTER", "0")
    w = _workload([10500], seed=12)
    ref = oracle.solve_batch(w, init=1, max_iter=400)
    out = _solve(w, precision="fp64", max_iter=400)
    assert out["status"][0] == "MAXITER" and ref[0]["status"] == "MAXITER"
    assert out["iters"][0] == 400
    assert np.array_equal(out["u"], ref[0]["u"])
    assert rel_err(out["sigma"][0], ref[0]["sigma"]) <= 1e-12


@pytest.mark.parametrize("max_iter", [400, 300000])
def test_fp64_cluster_kernel_bitwise_trajectory(max_iter):
    """RVEs of several parts run the FP64 cluster kernel (one part per CTA,
    neighbours through distributed shared memory, element slots per part):
    the trajectory is still the oracle's bit for bit, at a fixed iteration
    cap (2 to 16 parts; small parts keep the element table and the free-node
    state in shared memory, the 40,000-node RVE's parts neither) and to
    convergence."""
    sizes = [1500, 3000, 6000, 20000, 40000] if max_iter == 400 else [1300, 2600]
    w = _workload(sizes, seed=15)
    from paper_2305_07030_gb300 import plan
    assert sorted(set(int(x) for x in plan(w.nets)["parts"])) == \
        ([2, 4, 8, 16] if max_iter == 400 else [2, 4])
    ref = oracle.solve_batch(w, init=1, tol=1e-8, max_iter=max_iter)
    out = _solve(w, precision="fp64", init="affine", tol=1e-8, max_iter=max_iter)
    for p, r in enumerate(ref):
        a, b = out["node_off"][p], out["node_off"][p + 1]
        assert out["status"][p] == r["status"]
        assert out["iters"][p] == r["iters"], (p, out["iters"][p], r["iters"])
        assert np.array_equal(out["u"][a:b], r["u"]), np.abs(out["u"][a:b] - r["u"]).max()
        assert rel_err(out["sigma"][p], r["sigma"]) <= 1e-12
        assert abs(out["rel_res"][p] - r["rel_res"]) <= 1e-12 * max(r["rel_res"], 1e-300) + 1e-300


def test_mixed_within_tolerance_or_rounding_envelope():
    """Mixed precision against the oracle: 1e-5 relative stress where the
    oracle itself is insensitive to rounding; where a change of alpha or c by
    a few ulps already moves the oracle to another equilibrium, the mixed
    result may lie as far from the oracle as two such oracle runs lie from
    each other (the family's diameter). In every case the mixed displacement
    must be an equilibrium of the same problem by the oracle's force law, and
    the reported stress the oracle's stress at that displacement."""
    w = _workload([200, 512, 1200, 3000, 900], seed=13)
    env = envelope_batch(w)
    out = _solve(w, precision="mixed", tol=1e-8)
    rows = []
    for p, (r, spread) in enumerate(env):
        a, b = out["node_off"][p], out["node_off"][p + 1]
        res, s_at_u = check_equilibrium(w.nets[p], w.F[p], out["u"][a:b], r["f_ref"], 1e-8)
        e = rel_err(out["sigma"][p], r["sigma"])
        rows.append((p, w.nets[p].n_nodes, e, spread, res))
        assert out["status"][p] == "OK"
        assert res <= 1.5e-8, (p, res)
        assert rel_err(out["sigma"][p], s_at_u) <= 1e-12
        ok, e, bound = within_family(w.nets[p], w.F[p], w.damping[p], out["sigma"][p], r["sigma"],
                                     spread)
        assert ok, (rows, e, bound)
    print("mixed (p, n, err, oracle family diameter, oracle residual at GPU state):", rows)
    # the well-conditioned RVEs keep the oracle's equilibrium closely
    assert sum(1 for row in rows if row[3] <= 1e-6) >= 2


def test_mixed_unstaged_fallback():
    """Parts too large for the kernels' shared-memory element tables run the
    fallback that re-reads the CSR rows every iteration: with the cluster size
    of the 1024-2047-node bucket fixed at two, a 2000-node RVE runs as two
    parts of 1000 nodes, whose tables do not fit (a 700-node RVE, one part,
    runs staged beside it)."""
    from paper_2305_07030_gb300 import plan, tuning_set
    w = _workload([2000, 700], seed=20)
    env = envelope_batch(w)
    tuning_set({10: (2, 0, 0)})
    try:
        P = plan(w.nets)
        assert P["parts"].tolist() == [2, 1]
        assert P["staged"].tolist() == [[0, 0], [1, 1]]
        with Batch(w.nets, damping=w.damping) as b:
            assert list(b.parts()) == [2, 1]
            b.solve(w.F, precision="mixed", tol=1e-8)
            out = b.stress()
            u = b.displacement()
            off = b.node_off
    finally:
        tuning_set(None)
    for p, (r, spread) in enumerate(env):
        res, s_at_u = check_equilibrium(w.nets[p], w.F[p], u[off[p]:off[p + 1]], r["f_ref"], 1e-8)
        e = rel_err(out["sigma"][p], r["sigma"])
        assert out["status"][p] == "OK"
        assert res <= 1.5e-8, (p, res)
        assert rel_err(out["sigma"][p], s_at_u) <= 1e-12
        ok, e, bound = within_family(w.nets[p], w.F[p], w.damping[p], out["sigma"][p], r["sigma"],
                                     spread)
        assert ok, (p, e, bound)


def test_single_512_node_rve_both_modes():
    """The 512-node RVE with EA = 1 and F = diag(1.05, 1, 1)."""
    w = ri.single_rve_512()
    ref = oracle.solve_batch(w, init=1)[0]
    out = _solve(w, precision="fp64")
    assert out["iters"][0] == ref["iters"]
    assert np.array_equal(out["u"], ref["u"])
    assert rel_err(out["sigma"][0], ref["sigma"]) <= 1e-12
    out = _solve(w, precision="mixed")
    e = rel_err(out["sigma"][0], ref["sigma"])
    print("512-node mixed error", e, out["iters"][0], ref["iters"])
    assert out["status"][0] == "OK" and e <= 1e-5  # this RVE is well-conditioned


def test_edge_cases():
    rng = np.random.default_rng(14)
    base = ri.random_network(80, rng)
    # isolated free node (treated as fixed) and an RVE without elements
    X = np.vstack([base.X, [[0.5, 0.5, 0.5]]])
    iso = ri.Network(X=X, elems=base.elems, EA=base.EA,
                     fixed=np.append(base.fixed, 0).astype(np.uint8))
    empty = ri.Network(X=rng.random((5, 3)), elems=np.zeros((0, 2), np.int32),
                       EA=np.zeros(0), fixed=np.zeros(5, np.uint8))
    chain = ri.Network(X=np.array([[0, 0, 0], [0.5, 0, 0], [1.0, 0, 0]]),
                       elems=np.array([[0, 1], [1, 2]], np.int32), EA=np.array([1.0, 2.0]),
                       fixed=np.array([1, 0, 1], np.uint8))
    nets = [iso, empty, chain, base]
    F = np.array([ri.symmetric_perturbation(rng), np.eye(3), np.diag([1.1, 1, 1]), np.eye(3)])
    c = np.array([0.01, 0.01, 0.125, 0.01])
    w = ri.Workload("edge", nets, F, c)
    ref = oracle.solve_batch(w, init=1)
    out = _solve(w, precision="fp64")
    for p, r in enumerate(ref):
        a, b = out["node_off"][p], out["node_off"][p + 1]
        assert out["status"][p] == r["status"] == "OK"
        assert out["iters"][p] == r["iters"]
        assert np.array_equal(out["u"][a:b], r["u"])
    assert out["iters"][1] == 1 and np.all(out["sigma"][1] == 0)
    assert out["iters"][3] == 1 and np.all(out["sigma"][3] == 0)  # F = I
    # non-finite F is reported per RVE, not as a call failure
    F2 = F.copy()
    F2[2, 0, 0] = np.nan
    out = _solve(ri.Workload("nan", nets, F2, c), precision="mixed", max_iter=50)
    assert out["status"][2] == "NAN"
    assert out["status"][1] == "OK" and out["status"][3] == "OK"
    assert out["status"][0] in ("OK", "MAXITER")


def test_alone_equals_in_the_mix():
    """Batching does not change any RVE's result (FP64: bitwise)."""
    w = _workload([60, 900, 150, 2600, 400, 75], seed=15)
    mix = _solve(w, precision="fp64")
    for p in (1, 4):
        alone = _solve(w.subset([p]), precision="fp64")
        assert alone["iters"][0] == mix["iters"][p]
        assert np.array_equal(alone["sigma"][0], mix["sigma"][p])
    mixm = _solve(w, precision="mixed")
    alone = _solve(w.subset([3]), precision="mixed")
    assert alone["iters"][0] == mixm["iters"][3]
    assert np.array_equal(alone["sigma"][0], mixm["sigma"][3])


def test_warm_start_matches_oracle():
    w = _workload([400, 900], seed=16)
    with Batch(w.nets, damping=w.damping) as b:
        b.solve(w.F, precision="fp64")
        first = b.stress()
        u1 = b.displacement()
        F2 = np.array([np.diag([1.005, 1, 1]) @ f for f in w.F])
        b.solve(F2, precision="fp64", init="warm")
        second = b.stress()
        u2 = b.displacement()
    off = np.concatenate([[0], np.cumsum([n.n_nodes for n in w.nets])])
    for p, net in enumerate(w.nets):
        r = oracle.solve(net, F2[p], w.damping[p], init=2, u_warm=u1[off[p]:off[p + 1]])
        assert second["iters"][p] == r["iters"]
        assert np.array_equal(u2[off[p]:off[p + 1]], r["u"])
        assert second["status"][p] == first["status"][p] == "OK"


def test_device_entry_points():
    w = _workload([300, 500], seed=17)
    with Batch(w.nets, damping=w.damping) as b:
        F_dev = torch.tensor(w.F.reshape(-1), dtype=torch.float64, device="cuda")
        s = torch.cuda.Stream()
        b.solve_dev(F_dev, stream=s, precision="fp64")
        sig = torch.zeros(9 * w.n_rve, dtype=torch.float64, device="cuda")
        it = torch.zeros(w.n_rve, dtype=torch.int64, device="cuda")
        b.results_dev(sigma_dev=sig, iters_dev=it, stream=s)
        s.synchronize()
        host = b.stress()
        assert np.array_equal(sig.cpu().numpy().reshape(-1, 3, 3), host["sigma"])
        assert np.array_equal(it.cpu().numpy(), host["iters"])
        assert b.info()["launches"] >= 1


def test_naive_path_matches_oracle():
    """The paper's naive launch loop (atomic scatter: rounding order differs)."""
    w = _workload([150, 260], seed=18)
    ref = oracle.solve_batch(w, init=1)
    with Batch(w.nets, damping=w.damping) as b:
        b.solve_naive(w.F, init="affine")
        out = b.stress()
    for p, r in enumerate(ref):
        assert out["status"][p] == "OK"
        assert abs(out["iters"][p] - r["iters"]) <= 0.05 * r["iters"] + 2
        assert rel_err(out["sigma"][p], r["sigma"]) <= 1e-6


def test_invalid_inputs_rejected():
    from paper_2305_07030_gb300 import FE2Error
    rng = np.random.default_rng(19)
    net = ri.random_network(30, rng)
    bad = ri.Network(X=net.X, elems=np.vstack([net.elems, net.elems[:1]]),
                     EA=np.append(net.EA, 1.0), fixed=net.fixed)
    with pytest.raises(FE2Error, match="repeats"):
        Batch([bad])
    bad = ri.Network(X=net.X, elems=np.array([[0, 0]], np.int32), EA=np.ones(1), fixed=net.fixed)
    with pytest.raises(FE2Error, match="itself"):
        Batch([bad])
    bad = ri.Network(X=net.X, elems=net.elems, EA=-net.EA, fixed=net.fixed)
    with pytest.raises(FE2Error, match="EA"):
        Batch([bad])
    bad = ri.Network(X=net.X, elems=np.array([[0, 99]], np.int32), EA=np.ones(1), fixed=net.fixed)
    with pytest.raises(FE2Error, match="range"):
        Batch([bad])
    with Batch([net]) as b:
        with pytest.raises(FE2Error):
            b.solve(np.eye(3)[None], max_iter=0)


def test_stall_hand_back_resumes_in_double_float():
    """An RVE whose FP32 residual stops falling goes back to the double-float
    kernel, which runs it to convergence. With a stall window of one FP32
    evaluation every RVE is handed back at once: all still converge to an
    oracle-verified equilibrium within the mixed bound, and nearly all of
    their iterations run in double-float; with the default window none is
    handed back on these well-behaved RVEs."""
    w = _workload([200, 512, 900], seed=14)
    env = envelope_batch(w)
    with Batch(w.nets, damping=w.damping) as b:
        b.solve(w.F, precision="mixed", stall_window=1)
        out = b.stress()
        lead = b.diagnostics()["lead_iters"]
        u = b.displacement()
        off = b.node_off
        b.solve(w.F, precision="mixed")
        plain = b.stress()
        lead_plain = b.diagnostics()["lead_iters"]
    for p, (r, diam) in enumerate(env):
        assert out["status"][p] == "OK" and plain["status"][p] == "OK"
        res, s_at_u = check_equilibrium(w.nets[p], w.F[p], u[off[p]:off[p + 1]], r["f_ref"], 1e-8)
        assert res <= 1.5e-8, (p, res)
        assert rel_err(out["sigma"][p], s_at_u) <= 1e-12
        ok, e, bound = within_family(w.nets[p], w.F[p], w.damping[p], out["sigma"][p], r["sigma"],
                                     diam)
        assert ok, (p, e, bound)
        # handed back after a few FP32 evaluations: the rest ran in double-float
        assert out["iters"][p] - lead[p] <= 8, (p, out["iters"][p], lead[p])
        assert plain["iters"][p] - lead_plain[p] > 8
