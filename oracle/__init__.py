"""FP64 CPU oracle for batched dynamic relaxation (TEST INFRASTRUCTURE).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The GPU library never loads it and
shares no code with it: ``dr_oracle.c`` is a separate, plain C statement of
Algorithm 1 of Merson & Shephard (damped dynamic relaxation, Section III).

Parity status of each function (what pins it, see tests/test_oracle.py):
  ref_lengths, masses, time_step   closed forms (lattice, hand sums)
  internal_forces                  finite-difference energy gradient,
                                   action-reaction, lattice closed form
  stress_virial / stress_boundary  lattice closed forms, agreement at
                                   equilibrium, symmetry
  solve                            F = I, lattice and series-chain closed
                                   forms, exact rational trajectory of a
                                   one-DOF chain, Newton equilibrium on rigid
                                   trusses, objectivity
  newton                           lattice closed form, quadratic convergence
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

STATUS = {0: "OK", 1: "MAXITER", 2: "NAN"}


def build(force: bool = False) -> str:
    """Compile dr_oracle.c with gcc. FMA contraction is off so that x86 and
    Arm hosts round every operation the same way."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # FE2_ORACLE_LIB points the wrapper at another build of dr_oracle.c
            # (the mutation tests load deliberately broken copies this way).
            path = os.environ.get("FE2_ORACLE_LIB") or build()
            lib = C.CDLL(path)
            D, I64, P = C.c_double, C.c_int64, C.c_void_p
            lib.oracle_ref_lengths.argtypes = [I64, P, P, P]
            lib.oracle_masses.argtypes = [I64, I64, P, P, P, P]
            lib.oracle_time_step.argtypes = [I64, P, P, D]
            lib.oracle_time_step.restype = D
            lib.oracle_internal_forces.argtypes = [I64, P, I64, P, P, P, P]
            lib.oracle_strain_energy.argtypes = [I64, P, I64, P, P, P]
            lib.oracle_strain_energy.restype = D
            lib.oracle_stress_virial.argtypes = [I64, P, I64, P, P, P, P, D, P]
            lib.oracle_stress_boundary.argtypes = [I64, P, P, P, P, D, P]
            lib.oracle_dr_solve.argtypes = [I64, P, I64, P, P, P, P, D, D, I64, D, C.c_int, P, D,
                                            C.c_int, P, P, P, P, P, P, P, P]
            lib.oracle_dr_solve.restype = C.c_int
            lib.oracle_newton.argtypes = [I64, P, I64, P, P, P, P, C.c_int, D, P]
            lib.oracle_newton.restype = C.c_int
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


def ref_lengths(X, elems):
    X, el = _f64(X), _i32(elems)
    L = np.zeros(el.shape[0])
    _load().oracle_ref_lengths(el.shape[0], _p(X), _p(el), _p(L))
    return L


def masses(n, elems, EA, L):
    el, EA, L = _i32(elems), _f64(EA), _f64(L)
    m = np.zeros(n)
    _load().oracle_masses(n, el.shape[0], _p(el), _p(EA), _p(L), _p(m))
    return m


def time_step(EA, L, alpha=0.9):
    EA, L = _f64(EA), _f64(L)
    return _load().oracle_time_step(EA.shape[0], _p(EA), _p(L), alpha)


def internal_forces(x, elems, EA, L):
    x, el, EA, L = _f64(x), _i32(elems), _f64(EA), _f64(L)
    g = np.zeros_like(x)
    _load().oracle_internal_forces(x.shape[0], _p(x), el.shape[0], _p(el), _p(EA), _p(L), _p(g))
    return g


def strain_energy(x, elems, EA, L):
    x, el, EA, L = _f64(x), _i32(elems), _f64(EA), _f64(L)
    return _load().oracle_strain_energy(x.shape[0], _p(x), el.shape[0], _p(el), _p(EA), _p(L))


def stress_virial(x, elems, EA, L, F, V0=1.0):
    x, el, EA, L, F = _f64(x), _i32(elems), _f64(EA), _f64(L), _f64(F)
    s = np.zeros(9)
    _load().oracle_stress_virial(x.shape[0], _p(x), el.shape[0], _p(el), _p(EA), _p(L), _p(F),
                                 V0, _p(s))
    return s.reshape(3, 3)


def stress_boundary(x, g, fixed, F, V0=1.0):
    x, g, fx, F = _f64(x), _f64(g), _u8(fixed), _f64(F)
    s = np.zeros(9)
    _load().oracle_stress_boundary(x.shape[0], _p(x), _p(g), _p(fx), _p(F), V0, _p(s))
    return s.reshape(3, 3)


def solve(net, F, c, tol=1e-8, max_iter=10_000_000, alpha=0.9, init=0, u_warm=None,
          want_ke=False, want_energy=False):
    """Run Algorithm 1 on one network. Returns a dict with u (n,3), sigma (3,3),
    iters, rel_res, f_ref, ke, wint, wext and status ("OK", "MAXITER", "NAN").
    want_energy also tracks the internal and external work of the energy
    balance check (and the kinetic energy)."""
    X, el, EA, fx = _f64(net.X), _i32(net.elems), _f64(net.EA), _u8(net.fixed)
    F = _f64(F)
    n = X.shape[0]
    uw = _f64(u_warm) if u_warm is not None else np.zeros((n, 3))
    u = np.zeros((n, 3))
    sig = np.zeros(9)
    iters = C.c_int64(0)
    rr, fr, ke = C.c_double(0), C.c_double(0), C.c_double(0)
    wi, we = C.c_double(0), C.c_double(0)
    mode = 2 if want_energy else int(bool(want_ke))
    st = _load().oracle_dr_solve(n, _p(X), el.shape[0], _p(el), _p(EA), _p(fx), _p(F), float(c),
                                 float(tol), int(max_iter), float(alpha), int(init), _p(uw),
                                 float(net.V0), mode, _p(u), _p(sig),
                                 C.byref(iters), C.byref(rr), C.byref(fr), C.byref(ke),
                                 C.byref(wi), C.byref(we))
    if st < 0:
        raise ValueError(f"oracle_dr_solve failed with {st}")
    return {"u": u, "sigma": sig.reshape(3, 3), "iters": iters.value, "rel_res": rr.value,
            "f_ref": fr.value, "ke": ke.value, "wint": wi.value, "wext": we.value,
            "status": STATUS[st]}


def solve_batch(workload, tol=1e-8, max_iter=10_000_000, alpha=0.9, init=0, u_warm=None,
                threads=None, want_ke=False, want_energy=False):
    """Solve every RVE of a workload, one RVE per host thread (ctypes drops
    the GIL while the C solver runs)."""
    threads = threads or os.cpu_count() or 1
    uw = u_warm if u_warm is not None else [None] * workload.n_rve

    def one(p):
        return solve(workload.nets[p], workload.F[p], workload.damping[p], tol, max_iter, alpha,
                     init, uw[p], want_ke, want_energy)

    order = sorted(range(workload.n_rve), key=lambda p: -workload.nets[p].n_nodes)
    out = [None] * workload.n_rve
    with ThreadPoolExecutor(max_workers=threads) as ex:
        for p, r in zip(order, ex.map(one, order)):
            out[p] = r
    return out


def newton(net, u0, max_it=50, step_tol=1e-13):
    """Newton's method on g_free(x) = 0 from u0; returns (u, iterations, last step)."""
    X, el, EA, fx = _f64(net.X), _i32(net.elems), _f64(net.EA), _u8(net.fixed)
    u = _f64(u0).copy()
    last = C.c_double(0)
    it = _load().oracle_newton(X.shape[0], _p(X), el.shape[0], _p(el), _p(EA), _p(fx), _p(u),
                               max_it, step_tol, C.byref(last))
    if it < 0:
        raise np.linalg.LinAlgError("singular tangent")
    return u, it, last.value
