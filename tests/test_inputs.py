"""Seeded workload generator: kNN networks, boundary band, sizes, packing."""
import numpy as np

import rve_inputs as ri


def test_knn_matches_brute_force():
    rng = np.random.default_rng(0)
    X = rng.random((300, 3))
    el = ri.knn_edges(X, 4)
    d2 = ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(d2, np.inf)
    ref = set()
    for i in range(300):
        order = np.lexsort((np.arange(300), d2[i]))[:4]
        for j in order:
            ref.add((min(i, j), max(i, j)))
    assert set(map(tuple, el.tolist())) == ref
    assert np.all(el[:, 0] < el[:, 1])
    key = el[:, 0].astype(np.int64) * 300 + el[:, 1]
    assert np.all(np.diff(key) > 0)  # sorted, unique


def test_boundary_band_and_degrees():
    w = ri.single_rve_512()
    net = w.nets[0]
    dist = np.minimum(net.X, 1 - net.X).min(1)
    assert np.array_equal(net.fixed.astype(bool), dist <= 0.05)
    deg = np.bincount(net.elems.ravel(), minlength=net.n_nodes)
    assert deg.min() >= 4
    assert 1150 < net.n_elems < 1400
    assert np.all(net.EA == 1.0)
    assert np.allclose(w.F[0], np.diag([1.05, 1, 1]))


def test_deterministic_and_sizes():
    a = ri.uneven_rves(8, 500, 20000, workload=4, stop=2)
    b = ri.uneven_rves(8, 500, 20000, workload=4, stop=2)
    for na, nb in zip(a.nets, b.nets):
        assert np.array_equal(na.X, nb.X) and np.array_equal(na.elems, nb.elems)
        assert np.array_equal(na.EA, nb.EA)
    assert np.array_equal(a.F, b.F)
    sizes = ri.uneven_sizes(4096, 500, 20000, 4)
    assert sizes.min() >= 500 and sizes.max() <= 20000
    assert abs(np.log(sizes).mean() - 0.5 * (np.log(500) + np.log(20000))) < 0.1
    F = a.F[0]
    assert np.allclose(F, F.T)


def test_pack_offsets():
    w = ri.uneven_rves(3, 50, 80, workload=3)
    pk = ri.pack(w.nets)
    assert pk["node_off"][-1] == sum(n.n_nodes for n in w.nets)
    assert pk["elem_off"][-1] == sum(n.n_elems for n in w.nets)
    assert pk["X"].shape == (3 * pk["node_off"][-1],)
    assert pk["conn"].shape == (2 * pk["elem_off"][-1],)
