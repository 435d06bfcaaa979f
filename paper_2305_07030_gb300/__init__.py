"""Python binding of the fe2 C ABI (include/fe2.h): argument marshalling only.

Every step of the dynamic-relaxation path runs in the CUDA library
``libfe2gb300.so`` built from ``csrc/``; this module converts numpy arrays and
torch tensors to pointers and back. There is no CPU fallback: importing fails
loudly if the library cannot be built or loaded.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

__all__ = ["Batch", "Opts", "Tuning", "last_error", "FE2Error", "LIB_PATH", "RVE_STATUS",
           "tuning_get", "tuning_set", "tuning_load", "autotune", "shard_plan"]

LIB_PATH = _build.LIB
RVE_STATUS = {0: "OK", 1: "MAXITER", 2: "NAN", 3: "PENDING"}
_STATUS = {0: "FE2_OK", 1: "FE2_EINVAL", 2: "FE2_ENOMEM", 3: "FE2_ECUDA", 4: "FE2_ESTATE",
           5: "FE2_ETIMEOUT", 6: "FE2_ENODEV", 7: "FE2_EBUSY"}


class FE2Error(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


class Tuning(C.Structure):
    """fe2_tuning: per size bucket b (2^b <= nodes < 2^(b+1)) the mixed
    solver's cluster size and CTA sizes; zero = automatic."""
    _fields_ = [("parts", C.c_int32 * 32), ("block_fp32", C.c_int32 * 32),
                ("block_lead", C.c_int32 * 32)]


class Opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int64), ("dt_safety", C.c_double),
                ("precision", C.c_int32), ("init", C.c_int32), ("kinetic_energy", C.c_int32),
                ("block_threads", C.c_int32), ("lead_iters", C.c_int64),
                ("rebase_every", C.c_int32), ("launch", C.c_int32), ("lead_tol", C.c_double),
                ("stall_window", C.c_int64)]


def _load():
    # rebuilt when missing or older than any of its sources (a no-op otherwise)
    path = _build.build(force=bool(os.environ.get("FE2_REBUILD")))
    lib = C.CDLL(path)
    P, I32, I64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    lib.fe2_opts_default.argtypes = [C.POINTER(Opts)]
    lib.fe2_opts_default.restype = None
    lib.fe2_batch_create.argtypes = [I32, P, P, P, P, P, P, P, P, P, C.POINTER(P)]
    lib.fe2_batch_solve.argtypes = [P, P, C.POINTER(Opts), P]
    lib.fe2_batch_solve_dev.argtypes = [P, P, C.POINTER(Opts), P]
    lib.fe2_batch_solve_naive.argtypes = [P, P, C.POINTER(Opts), P]
    lib.fe2_batch_stress.argtypes = [P, P, P, P, P]
    lib.fe2_batch_results_dev.argtypes = [P, P, P, P, P, P]
    lib.fe2_batch_get_displacement.argtypes = [P, P]
    lib.fe2_batch_set_displacement.argtypes = [P, P]
    lib.fe2_batch_destroy.argtypes = [P]
    lib.fe2_batch_info.argtypes = [P, P, P, P, P]
    lib.fe2_batch_kernel_times.argtypes = [P, P, I32, P]
    lib.fe2_batch_diagnostics.argtypes = [P, P, P, P]
    lib.fe2_batch_submit.argtypes = [P, I32, P, P, C.POINTER(Opts), P]
    lib.fe2_batch_poll.argtypes = [P, I32, P, P, P, P, P, P]
    lib.fe2_serve.argtypes = [P, I32, P, P, P, C.POINTER(Opts), C.POINTER(Opts), I32, D, P, P, P, P]
    lib.fe2_batch_parts.argtypes = [P, P]
    lib.fe2_batch_layout.argtypes = [I32, P, P, P, P, P, P, I64, I32, P, P, P, P, P, P]
    lib.fe2_batch_plan.argtypes = [I32, P, P, P, P, P, P, I64, I32, I32, P, P, P, P, P, P, P]
    lib.fe2_probe_smem_bandwidth.argtypes = [P, P]
    lib.fe2_probe_smem_bandwidth.restype = C.c_int
    lib.fe2_probe_fp64_rates.argtypes = [P, P, P]
    lib.fe2_probe_fp64_rates.restype = C.c_int
    lib.fe2_rve_solve_noalloc.argtypes = [I32, I32, P, P, P, P, P, D, D, C.POINTER(Opts), P, P, P,
                                          P, P, P]
    lib.fe2_rve_solve_noalloc.restype = C.c_int
    lib.fe2_noalloc_scratch_bytes.argtypes = []
    lib.fe2_noalloc_scratch_bytes.restype = C.c_size_t
    lib.fe2_noalloc_last_error.argtypes = []
    lib.fe2_noalloc_last_error.restype = C.c_char_p
    lib.fe2_tuning_set.argtypes = [C.POINTER(Tuning)]
    lib.fe2_tuning_get.argtypes = [C.POINTER(Tuning)]
    lib.fe2_tuning_load.argtypes = [C.c_char_p]
    lib.fe2_autotune.argtypes = [I32, P, P, P, P, P, P, P, P, I64, C.c_char_p, C.POINTER(Tuning)]
    lib.fe2_shard_plan.argtypes = [I32, P, P, I32, P, P]
    lib.fe2_batch_energy.argtypes = [P, P, P, P, P]
    lib.fe2_batch_fp64_slots.argtypes = [I32, P, P, P, P, P, P, I64, I32, I64, P, P, P, P, P]
    lib.fe2_last_error.argtypes = []
    lib.fe2_last_error.restype = C.c_char_p
    for name in ("fe2_batch_create", "fe2_batch_solve", "fe2_batch_solve_dev",
                 "fe2_batch_solve_naive", "fe2_batch_stress", "fe2_batch_results_dev",
                 "fe2_batch_get_displacement", "fe2_batch_set_displacement",
                 "fe2_batch_destroy", "fe2_batch_info", "fe2_batch_kernel_times",
                 "fe2_batch_diagnostics", "fe2_batch_parts", "fe2_batch_submit",
                 "fe2_batch_poll", "fe2_serve", "fe2_batch_layout", "fe2_batch_plan",
                 "fe2_tuning_set", "fe2_tuning_get", "fe2_tuning_load", "fe2_autotune",
                 "fe2_shard_plan", "fe2_batch_energy", "fe2_batch_fp64_slots"):
        getattr(lib, name).restype = C.c_int
    return lib


_lib = _load()


def probe_smem_bandwidth():
    """Measured aggregate shared-memory read bandwidth (GB/s) and max SM clock (MHz)."""
    g, c = C.c_double(), C.c_double()
    rc = _lib.fe2_probe_smem_bandwidth(C.byref(g), C.byref(c))
    if rc != 0:
        raise FE2Error(3, f"smem probe failed ({rc})")
    return g.value, c.value


def probe_fp64_rates():
    """Measured aggregate FP64 throughput (operations/s) of fused multiply-add,
    correctly rounded division and square root: (fma, div, sqrt)."""
    f, d, q = C.c_double(), C.c_double(), C.c_double()
    rc = _lib.fe2_probe_fp64_rates(C.byref(f), C.byref(d), C.byref(q))
    if rc != 0:
        raise FE2Error(3, f"fp64 probe failed ({rc})")
    return f.value, d.value, q.value


def rve_solve_noalloc(n_nodes, n_elems, X_dev, conn_dev, EA_dev, fixed_dev, F_dev, u_dev,
                      sigma_dev, iters_dev, rel_res_dev, status_dev, damping=-1.0, V0=1.0,
                      stream=None, **opts):
    """fe2_rve_solve_noalloc on CUDA tensors (all device buffers are the
    caller's; the library allocates nothing). Asynchronous on `stream`."""
    o = make_opts(**opts)
    dp = lambda t: C.c_void_p(t.data_ptr())  # noqa: E731
    rc = _lib.fe2_rve_solve_noalloc(int(n_nodes), int(n_elems), dp(X_dev), dp(conn_dev),
                                    dp(EA_dev), dp(fixed_dev), dp(F_dev), float(damping),
                                    float(V0), C.byref(o), dp(u_dev), dp(sigma_dev),
                                    dp(iters_dev), dp(rel_res_dev), dp(status_dev),
                                    _stream_handle(stream))
    if rc != 0:
        raise FE2Error(rc, _lib.fe2_noalloc_last_error().decode())


def tuning_get() -> dict:
    """The process-wide launch tuning as {bucket: (parts, block_fp32, block_lead)}
    for the buckets with a non-zero entry."""
    t = Tuning()
    _check(_lib.fe2_tuning_get(C.byref(t)))
    return {b: (t.parts[b], t.block_fp32[b], t.block_lead[b]) for b in range(32)
            if t.parts[b] or t.block_fp32[b] or t.block_lead[b]}


def tuning_set(entries=None):
    """Set the tuning from {bucket: (parts, block_fp32[, block_lead])};
    None resets every entry to automatic."""
    if entries is None:
        _check(_lib.fe2_tuning_set(None))
        return
    t = Tuning()
    for b, v in entries.items():
        t.parts[b] = int(v[0])
        t.block_fp32[b] = int(v[1]) if len(v) > 1 else 0
        t.block_lead[b] = int(v[2]) if len(v) > 2 else 0
    _check(_lib.fe2_tuning_set(C.byref(t)))


def tuning_load(path):
    _check(_lib.fe2_tuning_load(os.fsencode(path)))


def autotune(nets, F, damping=None, trial_iters=2000, json_path=None):
    """Run fe2_autotune on sample RVEs; returns the chosen tuning (also set
    process-wide and, with json_path, written as JSON)."""
    node_off, X, elem_off, conn, EA, fixed = _pack_inputs(nets)
    Fh = np.ascontiguousarray(F, np.float64).reshape(len(nets), 9)
    damp = None if damping is None else np.ascontiguousarray(damping, np.float64)
    t = Tuning()
    _check(_lib.fe2_autotune(len(nets), _ptr(node_off), _ptr(X), _ptr(elem_off), _ptr(conn),
                             _ptr(EA), _ptr(fixed), _ptr(damp), _ptr(Fh), int(trial_iters),
                             None if json_path is None else os.fsencode(json_path), C.byref(t)))
    return tuning_get()


def shard_plan(node_counts, n_ranks, iters=None):
    """fe2_shard_plan: the rank of every RVE (LPT by estimated cost) and the
    summed cost per rank."""
    counts = np.asarray(node_counts, np.int64)
    node_off = np.ascontiguousarray(np.concatenate([[0], np.cumsum(counts)]), np.int64)
    it = None if iters is None else np.ascontiguousarray(iters, np.int64)
    rank_of = np.zeros(len(counts), np.int32)
    cost = np.zeros(int(n_ranks))
    _check(_lib.fe2_shard_plan(len(counts), _ptr(node_off), _ptr(it), int(n_ranks), _ptr(rank_of),
                               _ptr(cost)))
    return rank_of, cost


def last_error() -> str:
    return _lib.fe2_last_error().decode()


def _check(code):
    if code != 0:
        raise FE2Error(code, last_error())


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


_PREC = {"fp64": 0, "mixed": 1}
_INIT = {"reference": 0, "affine": 1, "warm": 2}


def make_opts(tol=1e-8, max_iter=10_000_000, dt_safety=0.9, precision="mixed", init="affine",
              kinetic_energy=False, block_threads=0, lead_iters=-1, rebase_every=0,
              lead_tol=1e-2, launch="graph", stall_window=0) -> Opts:
    o = Opts()
    _lib.fe2_opts_default(C.byref(o))
    o.tol = float(tol)
    o.max_iter = int(max_iter)
    o.dt_safety = float(dt_safety)
    o.precision = _PREC[precision] if isinstance(precision, str) else int(precision)
    o.init = _INIT[init] if isinstance(init, str) else int(init)
    # True / 1: kinetic energy; "balance" / 2: also the energy-balance work terms
    o.kinetic_energy = 2 if kinetic_energy in ("balance", 2) else int(bool(kinetic_energy))
    o.block_threads = int(block_threads)
    o.lead_iters = int(lead_iters)
    o.rebase_every = int(rebase_every)
    o.lead_tol = float(lead_tol)
    o.launch = {"graph": 0, "stream": 1}[launch] if isinstance(launch, str) else int(launch)
    o.stall_window = int(stall_window)
    return o


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


def layout(nets, smem_optin=232448, nodes_per_cta=0):
    """The internal packing that ``Batch(nets)`` would use, computed on the
    host without a device (``fe2_batch_layout``): parts per RVE, the node
    permutation, CSR rows and columns, and part offsets."""
    n_rve = len(nets)
    node_off = np.zeros(n_rve + 1, np.int64)
    elem_off = np.zeros(n_rve + 1, np.int64)
    for p, net in enumerate(nets):
        node_off[p + 1] = node_off[p] + net.X.shape[0]
        elem_off[p + 1] = elem_off[p] + net.elems.shape[0]
    X = np.ascontiguousarray(np.concatenate([n.X for n in nets]), np.float64)
    conn = np.ascontiguousarray(np.concatenate([n.elems for n in nets]), np.int32)
    EA = np.ascontiguousarray(np.concatenate([n.EA for n in nets]), np.float64)
    fixed = np.ascontiguousarray(np.concatenate([n.fixed for n in nets]), np.uint8)
    N, E = int(node_off[-1]), int(elem_off[-1])
    out = {"parts": np.zeros(n_rve, np.int32), "perm": np.zeros(N, np.int64),
           "rowptr": np.zeros(N + n_rve, np.int32), "col": np.zeros(2 * E, np.int32),
           "col_part": np.zeros(2 * E, np.int32), "part_off": np.zeros(n_rve * 34, np.int32)}
    _check(_lib.fe2_batch_layout(n_rve, _ptr(node_off), _ptr(X), _ptr(elem_off), _ptr(conn),
                                 _ptr(EA), _ptr(fixed), int(smem_optin), int(nodes_per_cta),
                                 _ptr(out["parts"]), _ptr(out["perm"]), _ptr(out["rowptr"]),
                                 _ptr(out["col"]), _ptr(out["col_part"]), _ptr(out["part_off"])))
    out["node_off"] = node_off
    out["elem_off"] = elem_off
    out["part_off"] = out["part_off"].reshape(n_rve, 2, 17)
    return out


def _pack_inputs(nets):
    n_rve = len(nets)
    node_off = np.zeros(n_rve + 1, np.int64)
    elem_off = np.zeros(n_rve + 1, np.int64)
    for p, net in enumerate(nets):
        node_off[p + 1] = node_off[p] + net.X.shape[0]
        elem_off[p + 1] = elem_off[p] + net.elems.shape[0]
    X = np.ascontiguousarray(np.concatenate([n.X for n in nets]), np.float64)
    conn = np.ascontiguousarray(np.concatenate([n.elems for n in nets]), np.int32)
    EA = np.ascontiguousarray(np.concatenate([n.EA for n in nets]), np.float64)
    fixed = np.ascontiguousarray(np.concatenate([n.fixed for n in nets]), np.uint8)
    return node_off, X, elem_off, conn, EA, fixed


def plan(nets, smem_optin=232448, nodes_per_cta=0):
    """The mixed solver's launch plan for ``Batch(nets)``, computed on the host
    without a device (``fe2_batch_plan``): per RVE its class; per class the
    cluster size, RVE count, and per kernel (lead, FP32) the shared memory per
    CTA, whether the element table is staged in it, and the CTA size."""
    n_rve = len(nets)
    node_off, X, elem_off, conn, EA, fixed = _pack_inputs(nets)
    m = max(8, n_rve)  # classes never outnumber RVEs
    ncls = C.c_int32()
    out = {"rve_class": np.zeros(n_rve, np.int32), "parts": np.zeros(m, np.int32),
           "rves": np.zeros(m, np.int32), "smem": np.zeros(2 * m, np.int64),
           "staged": np.zeros(2 * m, np.int32), "block": np.zeros(2 * m, np.int32)}
    _check(_lib.fe2_batch_plan(n_rve, _ptr(node_off), _ptr(X), _ptr(elem_off), _ptr(conn), _ptr(EA),
                               _ptr(fixed), int(smem_optin), int(nodes_per_cta), m, C.byref(ncls),
                               _ptr(out["rve_class"]), _ptr(out["parts"]), _ptr(out["rves"]),
                               _ptr(out["smem"]), _ptr(out["staged"]), _ptr(out["block"])))
    k = ncls.value
    out["n_classes"] = k
    for key in ("parts", "rves"):
        out[key] = out[key][:k]
    for key in ("smem", "staged", "block"):
        out[key] = out[key][:2 * k].reshape(k, 2)  # columns: lead, FP32
    return out


def fp64_slots(nets, smem_optin=232448, nodes_per_cta=0):
    """The FP64 cluster kernel's element slot tables for ``Batch(nets)``,
    computed on the host (``fe2_batch_fp64_slots``)."""
    n_rve = len(nets)
    node_off, X, elem_off, conn, EA, fixed = _pack_inputs(nets)
    E = int(elem_off[-1])
    ns = C.c_int64()
    args = (n_rve, _ptr(node_off), _ptr(X), _ptr(elem_off), _ptr(conn), _ptr(EA), _ptr(fixed),
            int(smem_optin), int(nodes_per_cta))
    _check(_lib.fe2_batch_fp64_slots(*args, 0, C.byref(ns), None, None, None, None))
    out = {"slot0": np.zeros(n_rve, np.int64), "part_slot": np.zeros(n_rve * 17, np.int32),
           "slot": np.zeros(4 * max(1, ns.value), np.int32), "csr_slot": np.zeros(2 * E, np.int32)}
    _check(_lib.fe2_batch_fp64_slots(*args, ns.value, C.byref(ns), _ptr(out["slot0"]),
                                     _ptr(out["part_slot"]), _ptr(out["slot"]), _ptr(out["csr_slot"])))
    out["n_slots"] = ns.value
    out["part_slot"] = out["part_slot"].reshape(n_rve, 17)
    out["slot"] = out["slot"][:4 * ns.value].reshape(-1, 4)
    return out


class Batch:
    """A packed batch of RVEs resident on the current CUDA device.

    ``nets`` is a list of objects with ``X (n,3)``, ``elems (E,2)``, ``EA (E,)``,
    ``fixed (n,)`` and ``V0`` (e.g. ``rve_inputs.Network``).
    """

    def __init__(self, nets, damping=None, stream=None):
        n_rve = len(nets)
        node_off = np.zeros(n_rve + 1, np.int64)
        elem_off = np.zeros(n_rve + 1, np.int64)
        for p, net in enumerate(nets):
            node_off[p + 1] = node_off[p] + net.X.shape[0]
            elem_off[p + 1] = elem_off[p] + net.elems.shape[0]
        X = np.ascontiguousarray(np.concatenate([n.X for n in nets]), np.float64)
        conn = np.ascontiguousarray(np.concatenate([n.elems for n in nets]), np.int32)
        EA = np.ascontiguousarray(np.concatenate([n.EA for n in nets]), np.float64)
        fixed = np.ascontiguousarray(np.concatenate([n.fixed for n in nets]), np.uint8)
        V0 = np.ascontiguousarray([getattr(n, "V0", 1.0) for n in nets], np.float64)
        damp = None if damping is None else np.ascontiguousarray(damping, np.float64)
        h = C.c_void_p()
        _check(_lib.fe2_batch_create(n_rve, _ptr(node_off), _ptr(X), _ptr(elem_off), _ptr(conn),
                                     _ptr(EA), _ptr(fixed), _ptr(V0), _ptr(damp),
                                     _stream_handle(stream), C.byref(h)))
        self._h = h
        self.n_rve = n_rve
        self.n_nodes = int(node_off[-1])
        self.node_off = node_off

    # -- solves ---------------------------------------------------------------
    def solve(self, F, stream=None, **opts):
        """Queue a solve for host F (P,3,3); returns immediately."""
        Fh = np.ascontiguousarray(F, np.float64).reshape(self.n_rve, 9)
        o = make_opts(**opts)
        _check(_lib.fe2_batch_solve(self._h, _ptr(Fh), C.byref(o), _stream_handle(stream)))

    def solve_dev(self, F_dev, stream=None, **opts):
        """Queue a solve for F already on the device (a CUDA tensor of 9*P doubles)."""
        o = make_opts(**opts)
        _check(_lib.fe2_batch_solve_dev(self._h, C.c_void_p(F_dev.data_ptr()), C.byref(o),
                                        _stream_handle(stream)))

    def solve_naive(self, F, stream=None, **opts):
        """The paper's naive per-RVE launch loop (FP64, synchronous)."""
        Fh = np.ascontiguousarray(F, np.float64).reshape(self.n_rve, 9)
        o = make_opts(**opts)
        _check(_lib.fe2_batch_solve_naive(self._h, _ptr(Fh), C.byref(o), _stream_handle(stream)))

    # -- results --------------------------------------------------------------
    def stress(self):
        P = self.n_rve
        sig = np.zeros((P, 9))
        it = np.zeros(P, np.int64)
        rr = np.zeros(P)
        st = np.zeros(P, np.int32)
        _check(_lib.fe2_batch_stress(self._h, _ptr(sig), _ptr(it), _ptr(rr), _ptr(st)))
        return {"sigma": sig.reshape(P, 3, 3), "iters": it, "rel_res": rr,
                "status": [RVE_STATUS[int(s)] for s in st]}

    def results_dev(self, sigma_dev=None, iters_dev=None, rel_dev=None, status_dev=None,
                    stream=None):
        def dp(t):
            return None if t is None else C.c_void_p(t.data_ptr())
        _check(_lib.fe2_batch_results_dev(self._h, dp(sigma_dev), dp(iters_dev), dp(rel_dev),
                                          dp(status_dev), _stream_handle(stream)))

    def displacement(self):
        u = np.zeros((self.n_nodes, 3))
        _check(_lib.fe2_batch_get_displacement(self._h, _ptr(u)))
        return u

    def set_displacement(self, u):
        uh = np.ascontiguousarray(u, np.float64).reshape(self.n_nodes, 3)
        _check(_lib.fe2_batch_set_displacement(self._h, _ptr(uh)))

    def energy(self):
        """Energy balance of the last FP64 solve with kinetic_energy=2:
        kinetic energy, internal work, external (damping) work and the
        relative balance error, per RVE."""
        out = {k: np.zeros(self.n_rve) for k in ("kinetic", "internal_work", "external_work",
                                                 "balance")}
        _check(_lib.fe2_batch_energy(self._h, _ptr(out["kinetic"]), _ptr(out["internal_work"]),
                                     _ptr(out["external_work"]), _ptr(out["balance"])))
        return out

    def info(self):
        a, b, c, d = C.c_int32(), C.c_int64(), C.c_int64(), C.c_int32()
        _check(_lib.fe2_batch_info(self._h, C.byref(a), C.byref(b), C.byref(c), C.byref(d)))
        return {"n_rve": a.value, "n_nodes": b.value, "n_elems": c.value, "launches": d.value}

    # -- serving ---------------------------------------------------------------
    def submit(self, rve_ids, F, **opts):
        """Queue a micro-batch for the given RVEs (host arrays); returns its
        ticket, or None when every slot is busy (FE2_EBUSY)."""
        ids = np.ascontiguousarray(rve_ids, np.int32)
        Fh = np.ascontiguousarray(F, np.float64).reshape(len(ids), 9)
        o = make_opts(**opts)
        t = C.c_int32(-1)
        rc = _lib.fe2_batch_submit(self._h, len(ids), _ptr(ids), _ptr(Fh), C.byref(o), C.byref(t))
        if rc == 7:
            return None
        _check(rc)
        return t.value

    def poll(self):
        """Results of every finished micro-batch: dict of arrays keyed by field."""
        P = self.n_rve
        ids = np.zeros(P, np.int32)
        sig = np.zeros((P, 9))
        it = np.zeros(P, np.int64)
        rr = np.zeros(P)
        st = np.zeros(P, np.int32)
        n = C.c_int32(0)
        _check(_lib.fe2_batch_poll(self._h, P, _ptr(ids), _ptr(sig), _ptr(it), _ptr(rr), _ptr(st),
                                   C.byref(n)))
        k = n.value
        return {"ids": ids[:k], "sigma": sig[:k].reshape(k, 3, 3), "iters": it[:k],
                "rel_res": rr[:k], "status": [RVE_STATUS[int(x)] for x in st[:k]]}

    def serve(self, rve, t_arrive, F, max_batch=0, max_inflight_bytes=0.0, first=None, next=None):
        """Run the request loop over a timed schedule; returns per-request
        completion times (s), iterations, status codes and stresses."""
        rv = np.ascontiguousarray(rve, np.int32)
        ta = np.ascontiguousarray(t_arrive, np.float64)
        Fh = np.ascontiguousarray(F, np.float64).reshape(len(rv), 9)
        of = make_opts(**(first or {}))
        on = make_opts(**(next or dict(first or {}, init="warm")))
        n = len(rv)
        td = np.zeros(n)
        it = np.zeros(n, np.int64)
        st = np.zeros(n, np.int32)
        sig = np.zeros((n, 9))
        _check(_lib.fe2_serve(self._h, n, _ptr(rv), _ptr(ta), _ptr(Fh), C.byref(of), C.byref(on),
                              int(max_batch), float(max_inflight_bytes), _ptr(td), _ptr(it),
                              _ptr(st), _ptr(sig)))
        return {"t_done": td, "iters": it, "status": st, "sigma": sig.reshape(n, 3, 3)}

    def diagnostics(self):
        P = self.n_rve
        fr, ke, ld = np.zeros(P), np.zeros(P), np.zeros(P, np.int64)
        _check(_lib.fe2_batch_diagnostics(self._h, _ptr(fr), _ptr(ke), _ptr(ld)))
        return {"f_ref": fr, "kinetic_energy": ke, "lead_iters": ld}

    def parts(self):
        out = np.zeros(self.n_rve, np.int32)
        _check(_lib.fe2_batch_parts(self._h, _ptr(out)))
        return out

    def kernel_times_ms(self):
        """Event-timed duration of each persistent launch of the last solve."""
        buf = np.zeros(512, np.float32)
        n = C.c_int32()
        _check(_lib.fe2_batch_kernel_times(self._h, _ptr(buf), 512, C.byref(n)))
        return [float(x) for x in buf[:min(n.value, 512)]]

    def close(self):
        if getattr(self, "_h", None):
            _check(_lib.fe2_batch_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
