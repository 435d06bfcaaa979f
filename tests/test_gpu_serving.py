"""Serving (continuous micro-batching) on the GPU: submissions that overlap on
the device give each RVE exactly the result it gets alone, and the timed
request loop with warm restarts reproduces a sequential replay."""
import time

import numpy as np
import pytest

import rve_inputs as ri

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2305_07030_gb300 import Batch  # noqa: E402


def _workload(sizes, seed):
    rng = np.random.default_rng(seed)
    nets = [ri.random_network(int(n), rng) for n in sizes]
    F = np.array([ri.symmetric_perturbation(rng) for _ in nets])
    c = np.array([ri.default_damping(n.n_nodes) for n in nets])
    return ri.Workload("s", nets, F, c)


def _drain(b, want):
    got = {}
    t0 = time.time()
    while len(got) < want:
        r = b.poll()
        for k, p in enumerate(r["ids"]):
            got[int(p)] = (r["sigma"][k].copy(), int(r["iters"][k]), r["status"][k])
        assert time.time() - t0 < 600
        time.sleep(0.001)
    return got


def test_overlapping_submissions_equal_alone():
    w = _workload([300, 1200, 450, 2600, 800, 150, 1900, 600], seed=31)
    with Batch(w.nets, damping=w.damping) as b:
        a = b.submit([0, 1, 2, 3], w.F[[0, 1, 2, 3]])
        c = b.submit([4, 5, 6, 7], w.F[[4, 5, 6, 7]])  # overlaps the first on the device
        assert a is not None and c is not None and a != c
        mix = _drain(b, 8)
        alone = {}
        for p in range(w.n_rve):
            assert b.submit([p], w.F[[p]]) is not None
            alone.update(_drain(b, 1))
    for p in range(w.n_rve):
        assert mix[p][2] == alone[p][2] == "OK"
        assert mix[p][1] == alone[p][1]
        assert np.array_equal(mix[p][0], alone[p][0])


def test_submit_rejects_in_flight_and_bad_ids():
    from paper_2305_07030_gb300 import FE2Error
    w = _workload([200, 300], seed=32)
    with Batch(w.nets, damping=w.damping) as b:
        assert b.submit([0], w.F[[0]]) is not None
        with pytest.raises(FE2Error, match="in flight"):
            b.submit([0, 1], w.F[[0, 1]])
        with pytest.raises(FE2Error, match="range"):
            b.submit([5], w.F[[0]])
        _drain(b, 1)


def test_request_loop_with_warm_restarts_matches_replay():
    w = _workload([250, 700, 400, 1100, 180], seed=33)
    steps = 3
    rng = np.random.default_rng(34)
    # request r: RVE p, step k; F grows by 0.5 % stretch per step
    reqs = [(p, k) for k in range(steps) for p in range(w.n_rve)]
    t_arr = np.sort(rng.uniform(0.0, 0.05, size=len(reqs)))
    rve = np.array([p for p, _ in reqs], np.int32)
    F = np.array([np.diag([1.0 + 0.005 * k, 1.0, 1.0]) @ w.F[p] for p, k in reqs])
    with Batch(w.nets, damping=w.damping) as b:
        out = b.serve(rve, t_arr, F, max_batch=4)
    assert np.all(out["status"] == 0)
    assert np.all(out["t_done"] >= t_arr)
    # replay: each RVE's chain alone, in order, on a fresh batch
    with Batch(w.nets, damping=w.damping) as b2:
        for p in range(w.n_rve):
            for r in [i for i, (q, _) in enumerate(reqs) if q == p]:
                init = "affine" if reqs[r][1] == 0 else "warm"
                assert b2.submit([p], F[[r]], init=init) is not None
                res = _drain(b2, 1)[p]
                assert res[1] == out["iters"][r]
                assert np.array_equal(res[0], out["sigma"][r])


def test_batched_and_served_calls_are_ordered():
    """A warm submission issued right after an asynchronous batched solve
    starts from that solve's result, and a batched solve issued while
    submissions are in flight starts after them: both give exactly the
    serialised results."""
    w = _workload([300, 900, 500], seed=35)
    F2 = np.array([np.diag([1.005, 1.0, 1.0]) @ f for f in w.F])
    # serialised order
    with Batch(w.nets, damping=w.damping) as b:
        b.solve(w.F, precision="fp64")
        b.stress()  # waits
        assert b.submit([1], F2[[1]], precision="fp64", init="warm") is not None
        ser_warm = _drain(b, 1)[1]
        assert b.submit([0, 2], w.F[[0, 2]], precision="fp64") is not None
        _drain(b, 2)
        b.solve(F2, precision="fp64", init="warm")
        ser_batch = b.stress()
    # the same calls without waiting in between
    with Batch(w.nets, damping=w.damping) as b:
        b.solve(w.F, precision="fp64")
        assert b.submit([1], F2[[1]], precision="fp64", init="warm") is not None
        got_warm = _drain(b, 1)[1]
        assert b.submit([0, 2], w.F[[0, 2]], precision="fp64") is not None
        b.solve(F2, precision="fp64", init="warm")  # while [0, 2] may be in flight
        got_batch = b.stress()
        _drain(b, 2)
    assert got_warm[1] == ser_warm[1] and np.array_equal(got_warm[0], ser_warm[0])
    assert np.array_equal(got_batch["iters"], ser_batch["iters"])
    assert np.array_equal(got_batch["sigma"], ser_batch["sigma"])
