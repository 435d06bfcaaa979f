"""Sharding a batch over ranks (host logic; CPU, gloo, world_size 2).

The partition is longest-processing-time-first by estimated cost; the
gathered per-RVE results must equal a one-process solve bit for bit, with
every RVE solved by exactly one rank.
"""
import os
import socket
import tempfile

import numpy as np
import pytest

import rve_inputs as ri


def test_shard_plan_is_lpt_and_deterministic():
    import paper_2305_07030_gb300 as m
    rng = np.random.default_rng(61)
    counts = ri.log_uniform_sizes(rng, 97, 500, 20000)
    for ranks in (1, 2, 3, 8):
        r1, cost = m.shard_plan(counts, ranks)
        r2, _ = m.shard_plan(counts, ranks)
        assert np.array_equal(r1, r2)
        assert r1.min() >= 0 and r1.max() < ranks
        c = counts.astype(float) ** 1.5
        assert np.allclose(np.bincount(r1, weights=c, minlength=ranks), cost)
        # LPT: no rank exceeds the mean load by more than the largest job
        assert cost.max() <= c.sum() / ranks + c.max() + 1e-6
        # and its own greedy rule: the last job placed on the busiest rank
        # went to a least-loaded rank at that time
    it = rng.integers(1000, 100000, size=97)
    r3, cost3 = m.shard_plan(counts, 4, iters=it)
    assert np.allclose(np.bincount(r3, weights=counts * it.astype(float), minlength=4), cost3)
    with pytest.raises(m.FE2Error):
        m.shard_plan(counts, 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_sharded_solve_gathers_bit_identical_results_world2():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    import shard_worker
    sizes, seed = [60, 250, 90, 400, 130, 75, 310], 62
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "gathered.npz")
        mp.spawn(shard_worker.run, args=(2, _free_port(), out, sizes, seed), nprocs=2, join=True)
        got = np.load(out)
    rng = np.random.default_rng(seed)
    nets = [ri.random_network(int(n), rng) for n in sizes]
    F = np.array([ri.symmetric_perturbation(rng) for _ in nets])
    c = np.array([ri.default_damping(n.n_nodes) for n in nets])
    sig, it, st = shard_worker._oracle_solve(nets, F, c, max_iter=3000)
    assert np.array_equal(got["sigma"], sig)
    assert np.array_equal(got["iters"], it)
    assert np.array_equal(got["status"], st)
    assert set(got["rank_of"].tolist()) == {0, 1}
    import paper_2305_07030_gb300 as m
    assert np.array_equal(got["rank_of"], m.shard_plan(sizes, 2)[0])
