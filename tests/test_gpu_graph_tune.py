"""GPU tests of the batch runtime: the batched solve replayed as a CUDA graph,
the per-size-bucket autotuner, and the largest RVEs of the mixed path.

Results must not depend on how the launches reach the GPU: the graph replay
of a solve is bit-identical to the same launches issued on streams, and a
tuned configuration keeps every RVE's result independent of the batch it is
in. The largest RVEs of the uneven workloads (up to ~33,000 nodes) run the
mixed path without element tables (velocity and acceleration in global
memory); the oracle would need tens of minutes for one of them, so their
converged state is checked by properties that hold at any size: it is an
equilibrium by the oracle's own force law, and the reported stress is the
oracle's stress at that state.
"""
import json
import os

import numpy as np
import pytest

import rve_inputs as ri

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2305_07030_gb300 as fe2  # noqa: E402
from paper_2305_07030_gb300 import Batch  # noqa: E402
from parity_util import check_equilibrium, rel_err  # noqa: E402


def _workload(sizes, seed):
    rng = np.random.default_rng(seed)
    nets = [ri.random_network(int(n), rng) for n in sizes]
    F = np.array([ri.symmetric_perturbation(rng) for _ in nets])
    c = np.array([ri.default_damping(n.n_nodes) for n in nets])
    return ri.Workload("g", nets, F, c)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_replay_equals_stream_launches(precision):
    """Several size classes (concurrent launches): the first graph solve
    captures, the second replays; both equal plain stream launches."""
    w = _workload([60, 700, 2500, 5200, 300, 9000], seed=51)
    runs = []
    with Batch(w.nets, damping=w.damping) as b:
        for launch in ("stream", "graph", "graph"):
            b.solve(w.F, precision=precision, launch=launch)
            out = b.stress()
            out["u"] = b.displacement()
            out["launches"] = b.info()["launches"]
            out["times"] = b.kernel_times_ms()
            runs.append(out)
    ref = runs[0]
    for out in runs[1:]:
        assert np.array_equal(out["iters"], ref["iters"])
        assert np.array_equal(out["sigma"], ref["sigma"])
        assert np.array_equal(out["u"], ref["u"])
        assert out["launches"] == ref["launches"] >= 1
        assert len(out["times"]) == len(ref["times"]) and all(t > 0 for t in out["times"])
    assert all(s == "OK" for s in ref["status"])


def test_autotune_writes_loads_and_keeps_results_batch_independent(tmp_path):
    """The autotuner picks a configuration per size bucket, writes it as JSON
    and sets it; loading the file restores it; under the tuned configuration
    an RVE gives the same result alone and in a mixed batch."""
    w = _workload([700, 900, 3000, 3500, 6000], seed=52)
    path = str(tmp_path / "tune.json")
    try:
        tuned = fe2.autotune(w.nets, w.F, w.damping, trial_iters=400, json_path=path)
        assert tuned, "no bucket tuned"
        with open(path) as f:
            doc = json.load(f)
        assert doc["precision"] == "mixed" and doc["sm_count"] == torch.cuda.get_device_properties(0).multi_processor_count
        got = {e["bucket"]: (e["parts"], e["block_fp32"]) for e in doc["buckets"]}
        assert got == {b: v[:2] for b, v in tuned.items()}
        for e in doc["buckets"]:
            assert e["node_iters_per_s_per_sm"] > 0 and len(e["tried"]) >= 1
        fe2.tuning_set(None)
        fe2.tuning_load(path)
        assert fe2.tuning_get() == tuned
        with Batch(w.nets, damping=w.damping) as b:
            b.solve(w.F)
            mix = b.stress()
            parts = b.parts()
        for p in (1, 3):
            with Batch([w.nets[p]], damping=w.damping[[p]]) as b:
                b.solve(w.F[[p]])
                alone = b.stress()
                assert b.parts()[0] == parts[p]
            assert alone["iters"][0] == mix["iters"][p]
            assert np.array_equal(alone["sigma"][0], mix["sigma"][p])
        bk = {int(np.floor(np.log2(n.n_nodes))) for n in w.nets}
        for p, n in enumerate(w.nets):
            b_ = int(np.floor(np.log2(n.n_nodes)))
            if b_ in tuned:
                assert parts[p] == tuned[b_][0]
        assert bk >= set(tuned)
    finally:
        fe2.tuning_set(None)


def test_largest_mixed_rves_reach_equilibrium():
    """RVEs at and above the old 28,800-node limit of the mixed path (the
    largest of the 1024 x log-U(1k, 33k) workload is 32,918 nodes)."""
    rng = np.random.default_rng(53)
    nets = [ri.random_network(n, rng) for n in (29_500, 32_918)]
    F = np.array([ri.symmetric_perturbation(rng) for _ in nets])
    c = np.array([ri.default_damping(n.n_nodes) for n in nets])
    with Batch(nets, damping=c) as b:
        assert list(b.parts()) == [16, 16]
        b.solve(F, precision="mixed")
        out = b.stress()
        u = b.displacement()
        f_ref = b.diagnostics()["f_ref"]
        off = b.node_off
    for p, net in enumerate(nets):
        assert out["status"][p] == "OK", out
        res, s_at_u = check_equilibrium(net, F[p], u[off[p]:off[p + 1]], f_ref[p], 1e-8)
        print(f"{net.n_nodes} nodes: {out['iters'][p]} iterations, oracle residual at GPU state {res:.2e}")
        assert res <= 1.5e-8
        assert rel_err(out["sigma"][p], s_at_u) <= 1e-12


def test_mixed_rejects_rves_beyond_shared_memory():
    from paper_2305_07030_gb300 import FE2Error
    rng = np.random.default_rng(54)
    net = ri.random_network(37_000, rng)
    with Batch([net]) as b:
        with pytest.raises(FE2Error, match="FE2_PREC_FP64"):
            b.solve(np.eye(3)[None], precision="mixed")
        b.solve(np.eye(3)[None], precision="fp64", max_iter=3)  # FP64 takes any size
        assert b.stress()["iters"][0] == 1  # F = I: converged at once
