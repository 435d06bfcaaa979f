"""Parity helpers shared by the GPU tests (test-only; uses the oracle)."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np

import oracle


def rel_err(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a - b)


def oracle_with_envelope(net, F, c, tol=1e-8, alpha=0.9):
    """The oracle's solve plus its rounding envelope: the largest stress
    change when the time-step factor moves by one unit in the last place
    either way. Networks that pass a bifurcation settle into an equilibrium
    picked by rounding; for them the envelope is large and no implementation
    with different rounding can be closer than that."""
    runs = [oracle.solve(net, F, c, tol=tol, alpha=a, init=1)
            for a in (alpha, np.nextafter(alpha, 1.0), np.nextafter(alpha, 0.0))]
    spread = max(rel_err(r["sigma"], runs[0]["sigma"]) for r in runs[1:])
    return runs[0], spread


def envelope_batch(w, tol=1e-8, idx=None, threads=None):
    idx = list(range(w.n_rve)) if idx is None else list(idx)
    with ThreadPoolExecutor(max_workers=threads or len(idx)) as ex:
        return list(ex.map(lambda p: oracle_with_envelope(w.nets[p], w.F[p], w.damping[p], tol), idx))


def check_equilibrium(net, F, u, f_ref, tol):
    """The displacement is an equilibrium of the same problem by the oracle's
    own force law; returns the oracle-evaluated relative residual and the
    oracle's stress at that state."""
    L = oracle.ref_lengths(net.X, net.elems)
    x = net.X + u
    g = oracle.internal_forces(x, net.elems, net.EA, L)
    res = np.linalg.norm(g[net.fixed == 0]) / f_ref if f_ref > 0 else 0.0
    return res, oracle.stress_virial(x, net.elems, net.EA, L, F, net.V0)
