"""Seeded synthetic RVE workloads: fiber networks, deformation gradients, damping.

This module only *draws* inputs. It holds none of the dynamic-relaxation
arithmetic (no forces, masses, time steps or stresses), so the FP64 oracle and
the CUDA path can both consume its output without sharing method code.

The paper's RVEs are collagen networks that are not published (Section II
names them but gives no data), so seeded stand-ins are drawn here:

* node positions uniform in the unit cube;
* each node linked to its k=4 nearest neighbours (Euclidean, non-periodic,
  self excluded, ties to the lower index), undirected and deduplicated, so an
  element is a pair (a, b) with a < b, elements sorted lexicographically;
* axial rigidity EA = 1, or lognormal(0, 0.3) per element;
* nodes with min(x, 1-x, y, 1-y, z, 1-z) <= 0.05 carry prescribed
  displacements ("fixed");
* one macroscale deformation gradient F per RVE.

Seeds: a workload with index ``w`` (1..5) uses base seed ``230507030 + w``;
RVE ``p`` of it draws from ``PCG64(base * 1000 + p)`` in the order positions,
EA, F. Node counts of uneven workloads come from ``PCG64(base)``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 230507030
BAND = 0.05


@dataclass
class Network:
    """One RVE: reference coordinates, truss elements and boundary flags."""

    X: np.ndarray            # (n, 3) float64, reference positions
    elems: np.ndarray        # (E, 2) int32, a < b, lexicographically sorted
    EA: np.ndarray           # (E,) float64, axial rigidity per element
    fixed: np.ndarray        # (n,) uint8, 1 = prescribed displacement
    V0: float = 1.0          # reference volume of the RVE (unit cube)

    @property
    def n_nodes(self) -> int:
        return int(self.X.shape[0])

    @property
    def n_elems(self) -> int:
        return int(self.elems.shape[0])


@dataclass
class Workload:
    """A batch of RVEs with one F and one damping coefficient each."""

    name: str
    nets: list
    F: np.ndarray                    # (P, 3, 3) float64
    damping: np.ndarray              # (P,) float64
    meta: dict = field(default_factory=dict)

    @property
    def n_rve(self) -> int:
        return len(self.nets)

    def total_nodes(self) -> int:
        return sum(n.n_nodes for n in self.nets)

    def subset(self, idx) -> "Workload":
        idx = list(idx)
        return Workload(self.name + f"[{len(idx)}]", [self.nets[i] for i in idx],
                        self.F[idx].copy(), self.damping[idx].copy(), dict(self.meta))


# ----------------------------------------------------------------------------
# network construction
# ----------------------------------------------------------------------------

def knn_edges(X: np.ndarray, k: int = 4) -> np.ndarray:
    """Undirected, deduplicated k-nearest-neighbour edges of point set ``X``.

    Candidates come from a k-d tree (k+3 per point); they are re-ranked by the
    exact squared distance computed here, ties broken by the lower index, so
    the result does not depend on the tree's own tie order.
    """
    n = X.shape[0]
    if n < 2:
        return np.zeros((0, 2), dtype=np.int32)
    kk = min(k, n - 1)
    q = min(kk + 3, n)
    try:
        from scipy.spatial import cKDTree
        _, cand = cKDTree(X).query(X, k=q)
        cand = np.asarray(cand, dtype=np.int64).reshape(n, q)
    except ImportError:  # pragma: no cover - scipy is present on both machines
        cand = np.empty((n, q), dtype=np.int64)
        for s in range(0, n, 512):
            d2 = ((X[s:s + 512, None, :] - X[None, :, :]) ** 2).sum(-1)
            cand[s:s + 512] = np.argsort(d2, axis=1, kind="stable")[:, :q]
    rows = np.repeat(np.arange(n), q)
    cols = cand.reshape(-1)
    diff = X[rows] - X[cols]
    d2 = diff[:, 0] * diff[:, 0] + diff[:, 1] * diff[:, 1] + diff[:, 2] * diff[:, 2]
    d2 = np.where(cols == rows, np.inf, d2).reshape(n, q)
    colsm = cols.reshape(n, q)
    order = np.lexsort((colsm, d2), axis=1)[:, :kk]
    nbr = np.take_along_axis(colsm, order, axis=1)
    a = np.repeat(np.arange(n), kk)
    b = nbr.reshape(-1)
    lo = np.minimum(a, b)
    hi = np.maximum(a, b)
    key = np.unique(lo * n + hi)
    return np.stack([key // n, key % n], axis=1).astype(np.int32)


def boundary_flags(X: np.ndarray, band: float = BAND) -> np.ndarray:
    """1 where a node lies within ``band`` of any face of the unit cube."""
    dist = np.minimum(X, 1.0 - X).min(axis=1)
    return (dist <= band).astype(np.uint8)


def random_network(n: int, rng: np.random.Generator, ea: str = "lognormal",
                   k: int = 4, band: float = BAND) -> Network:
    """kNN fiber network of ``n`` nodes drawn from ``rng`` (positions, then EA)."""
    X = rng.random((n, 3))
    elems = knn_edges(X, k)
    if ea == "unit":
        EA = np.ones(elems.shape[0])
    elif ea == "lognormal":
        EA = rng.lognormal(0.0, 0.3, size=elems.shape[0])
    else:
        raise ValueError(ea)
    return Network(X=X, elems=elems, EA=EA, fixed=boundary_flags(X, band))


def symmetric_perturbation(rng: np.random.Generator, scale: float = 0.02) -> np.ndarray:
    """F = I + scale * (G + G^T) / 2 with G i.i.d. standard normal."""
    G = rng.standard_normal((3, 3))
    return np.eye(3) + scale * 0.5 * (G + G.T)


def default_damping(n_nodes: int) -> float:
    """Damping coefficient c for an RVE of ``n_nodes`` nodes.

    The paper leaves c open. Its lowest mode frequency falls like the inverse
    linear size of the network, so c is scaled by (512/n)^(1/3) from 0.002 at
    512 nodes.
    """
    return 0.002 * (512.0 / float(n_nodes)) ** (1.0 / 3.0)


def log_uniform_sizes(rng: np.random.Generator, count: int, lo: int, hi: int) -> np.ndarray:
    """round(exp(U(ln lo, ln hi))) node counts."""
    return np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))).astype(np.int64)


# ----------------------------------------------------------------------------
# regular lattices (closed-form cases)
# ----------------------------------------------------------------------------

def cubic_lattice(m: int, bars: str = "xyz", EA_x=None) -> Network:
    """Regular m x m x m lattice of the unit cube, spacing h = 1/(m-1).

    ``bars`` picks the axis-aligned bar families ("xyz" or "x"). ``EA_x``
    (length m-1) gives every x-bar starting at x-index i the rigidity
    ``EA_x[i]``; other bars get EA = 1. Nodes are numbered i + m*(j + m*k).
    """
    h = 1.0 / (m - 1)
    idx = np.arange(m)
    I, J, K = np.meshgrid(idx, idx, idx, indexing="ij")
    I, J, K = I.ravel(order="F"), J.ravel(order="F"), K.ravel(order="F")
    node = I + m * (J + m * K)
    X = np.zeros((m ** 3, 3))
    X[node, 0] = I * h
    X[node, 1] = J * h
    X[node, 2] = K * h
    el, ea = [], []
    for axis, name in enumerate("xyz"):
        if name not in bars:
            continue
        step = [1, m, m * m][axis]
        for a in range(m ** 3):
            ijk = [a % m, (a // m) % m, a // (m * m)]
            if ijk[axis] == m - 1:
                continue
            el.append((a, a + step))
            if axis == 0 and EA_x is not None:
                ea.append(float(EA_x[ijk[0]]))
            else:
                ea.append(1.0)
    elems = np.array(el, dtype=np.int32)
    EA = np.array(ea)
    order = np.lexsort((elems[:, 1], elems[:, 0]))
    return Network(X=X, elems=elems[order], EA=EA[order], fixed=boundary_flags(X))


def braced_lattice(m: int) -> Network:
    """m^3 lattice with axis bars plus one face diagonal per square (a rigid truss).

    Every node within 0.05 of a face is fixed; interior nodes are free.
    """
    base = cubic_lattice(m)
    el = [tuple(e) for e in base.elems]
    for a in range(m ** 3):
        i, j, k = a % m, (a // m) % m, a // (m * m)
        if i < m - 1 and j < m - 1:
            el.append((a, a + 1 + m))
        if j < m - 1 and k < m - 1:
            el.append((a, a + m + m * m))
        if i < m - 1 and k < m - 1:
            el.append((a, a + 1 + m * m))
        if i < m - 1 and j < m - 1 and k < m - 1:
            el.append((a, a + 1 + m + m * m))
    elems = np.array(sorted(set((min(a, b), max(a, b)) for a, b in el)), dtype=np.int32)
    return Network(X=base.X, elems=elems, EA=np.ones(elems.shape[0]), fixed=base.fixed)


# ----------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------

def _rve_rng(workload: int, p: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64((SEED_BASE + workload) * 1000 + p))


def single_rve_512() -> Workload:
    """One 512-node RVE, EA = 1, F = diag(1.05, 1, 1)."""
    rng = _rve_rng(1, 0)
    net = random_network(512, rng, ea="unit")
    F = np.diag([1.05, 1.0, 1.0])[None]
    return Workload("rve512x1", [net], F, np.array([default_damping(512)]),
                    {"nodes": "512", "EA": "1", "F": "diag(1.05,1,1)"})


def equal_rves(count: int = 64, n: int = 5000) -> Workload:
    """``count`` RVEs of ``n`` nodes, lognormal EA, symmetric-perturbed F."""
    nets, Fs = [], []
    for p in range(count):
        rng = _rve_rng(2, p)
        nets.append(random_network(n, rng))
        Fs.append(symmetric_perturbation(rng))
    return Workload(f"rve{n}x{count}", nets, np.array(Fs),
                    np.array([default_damping(n)] * count),
                    {"nodes": str(n), "EA": "lognormal(0,0.3)", "F": "I+0.02 sym(N(0,1))"})


def uneven_rves(count: int, lo: int, hi: int, workload: int, first: int = 0,
                stop: int | None = None) -> Workload:
    """RVEs with log-uniform node counts in [lo, hi]; generates RVEs first..stop-1."""
    sizes = log_uniform_sizes(np.random.Generator(np.random.PCG64(SEED_BASE + workload)),
                              count, lo, hi)
    stop = count if stop is None else stop
    nets, Fs, cs = [], [], []
    for p in range(first, stop):
        rng = _rve_rng(workload, p)
        nets.append(random_network(int(sizes[p]), rng))
        Fs.append(symmetric_perturbation(rng))
        cs.append(default_damping(int(sizes[p])))
    return Workload(f"uneven{lo}-{hi}x{count}", nets, np.array(Fs).reshape(-1, 3, 3),
                    np.array(cs), {"sizes": sizes, "lo": lo, "hi": hi})


def uneven_subset(count: int, lo: int, hi: int, workload: int, idx) -> Workload:
    """The RVEs ``idx`` of the uneven workload (same draws as uneven_rves)."""
    sizes = log_uniform_sizes(np.random.Generator(np.random.PCG64(SEED_BASE + workload)),
                              count, lo, hi)
    nets, Fs, cs = [], [], []
    for p in idx:
        rng = _rve_rng(workload, int(p))
        nets.append(random_network(int(sizes[p]), rng))
        Fs.append(symmetric_perturbation(rng))
        cs.append(default_damping(int(sizes[p])))
    return Workload(f"uneven{lo}-{hi}x{count}[{len(nets)}]", nets,
                    np.array(Fs).reshape(-1, 3, 3), np.array(cs),
                    {"sizes": sizes, "lo": lo, "hi": hi, "idx": list(idx)})


def uneven_sizes(count: int, lo: int, hi: int, workload: int) -> np.ndarray:
    return log_uniform_sizes(np.random.Generator(np.random.PCG64(SEED_BASE + workload)),
                             count, lo, hi)


def stratified_idx(sizes, k: int) -> list:
    """k RVE indices spread evenly over the size order (smallest to largest):
    the seeded, size-stratified subset on which the oracle checks and times
    the uneven workloads."""
    order = np.argsort(np.asarray(sizes), kind="stable")
    pick = np.rint(np.linspace(0, len(order) - 1, k)).astype(int)
    return sorted(int(order[i]) for i in pick)


def serving_F(S: np.ndarray, step: int) -> np.ndarray:
    """F of a Gauss point at macro step ``step``: diag(1+0.005 step,1,1)(I+0.02 S)."""
    return np.diag([1.0 + 0.005 * step, 1.0, 1.0]) @ (np.eye(3) + 0.02 * S)


def serving_requests(n_points: int, n_steps: int, lo: int, hi: int, rate: float,
                     seed_workload: int = 5):
    """Macro-step request stream: per Gauss point a size, a symmetric S and
    Poisson arrival times (rate per second) for each step."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + seed_workload))
    sizes = log_uniform_sizes(rng, n_points, lo, hi)
    G = rng.standard_normal((n_points, 3, 3))
    S = 0.5 * (G + np.transpose(G, (0, 2, 1)))
    gaps = rng.exponential(1.0 / rate, size=n_points * n_steps)
    arrivals = np.cumsum(gaps).reshape(n_steps, n_points)
    return sizes, S, arrivals


# ----------------------------------------------------------------------------
# packing (caller-side, CRS-like; the library copies it at create time)
# ----------------------------------------------------------------------------

def pack(nets) -> dict:
    """Concatenate networks into the packed arrays the C ABI takes.

    node_off/elem_off are prefix sums (length P+1); conn holds RVE-local node
    ids; X is xyz-interleaved.
    """
    P = len(nets)
    node_off = np.zeros(P + 1, dtype=np.int64)
    elem_off = np.zeros(P + 1, dtype=np.int64)
    for p, net in enumerate(nets):
        node_off[p + 1] = node_off[p] + net.n_nodes
        elem_off[p + 1] = elem_off[p] + net.n_elems
    X = np.concatenate([n.X for n in nets]).astype(np.float64) if P else np.zeros((0, 3))
    conn = (np.concatenate([n.elems for n in nets]).astype(np.int32) if P
            else np.zeros((0, 2), np.int32))
    EA = np.concatenate([n.EA for n in nets]).astype(np.float64) if P else np.zeros(0)
    fixed = np.concatenate([n.fixed for n in nets]).astype(np.uint8) if P else np.zeros(0, np.uint8)
    V0 = np.array([n.V0 for n in nets], dtype=np.float64)
    return {
        "n_rve": P,
        "node_off": np.ascontiguousarray(node_off),
        "X": np.ascontiguousarray(X.reshape(-1)),
        "elem_off": np.ascontiguousarray(elem_off),
        "conn": np.ascontiguousarray(conn.reshape(-1)),
        "EA": np.ascontiguousarray(EA),
        "fixed": np.ascontiguousarray(fixed),
        "V0": V0,
    }
