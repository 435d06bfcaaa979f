"""The allocation-free single-RVE entry point, called through the C ABI.

Callers that cannot allocate device memory (code running while a CUDA graph
is captured, real-time loops, frameworks that own all device memory) pass
their own device buffers; the library works in a fixed device array. Its
results must equal the batched FP64 path's on the same networks, over two
calls in a row (the second call reuses the scratch array the first one left
behind). This file sorts last so that a failing run has run everything else.
"""
import ctypes as C

import numpy as np
import pytest

import rve_inputs as ri

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2305_07030_gb300 as fe2  # noqa: E402


def _dev(a, dtype):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _noalloc(net, F, c, opts, free_check=None):
    n, E = net.n_nodes, net.n_elems
    X = _dev(net.X.reshape(-1), torch.float64)
    conn = _dev(net.elems.reshape(-1), torch.int32)
    EA = _dev(net.EA, torch.float64)
    fixed = _dev(net.fixed, torch.uint8)
    Fd = _dev(F.reshape(-1), torch.float64)
    u = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    sig = torch.zeros(9, dtype=torch.float64, device="cuda")
    it = torch.zeros(1, dtype=torch.int64, device="cuda")
    rr = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    lib = fe2._lib
    p = lambda t: C.c_void_p(t.data_ptr())  # noqa: E731
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    rc = lib.fe2_rve_solve_noalloc(n, E, p(X), p(conn), p(EA), p(fixed), p(Fd), float(c), 1.0,
                                   C.byref(opts), p(u), p(sig), p(it), p(rr), p(st), None)
    assert rc == 0, lib.fe2_noalloc_last_error().decode()
    torch.cuda.synchronize()
    if free_check:
        # nothing was allocated by the call itself
        assert torch.cuda.mem_get_info()[0] >= free_before
    return {"u": u.cpu().numpy().reshape(n, 3), "sigma": sig.cpu().numpy().reshape(3, 3),
            "iters": int(it.item()), "rel_res": float(rr.item()), "status": int(st.item())}


def test_noalloc_matches_batched_fp64_on_two_calls():
    rng = np.random.default_rng(7)
    nets = [ri.random_network(700, rng), ri.random_network(300, rng)]
    Fs = [ri.symmetric_perturbation(rng) for _ in nets]
    cs = [ri.default_damping(n.n_nodes) for n in nets]
    opts = fe2.make_opts(precision="fp64", init="affine", tol=1e-8)
    for k, (net, F, c) in enumerate(zip(nets, Fs, cs)):
        out = _noalloc(net, F, c, opts, free_check=(k > 0))
        with fe2.Batch([net], damping=[c]) as b:
            b.solve(F[None], precision="fp64", init="affine", tol=1e-8)
            ref = b.stress()
            u_ref = b.displacement()
        assert out["status"] == 0 and ref["status"][0] == "OK"
        assert out["iters"] == int(ref["iters"][0])
        assert np.array_equal(out["u"], u_ref)
        err = np.linalg.norm(out["sigma"] - ref["sigma"][0]) / np.linalg.norm(ref["sigma"][0])
        assert err <= 1e-12, err
        assert abs(out["rel_res"] - ref["rel_res"][0]) <= 1e-12 * ref["rel_res"][0]


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = fe2._lib
    opts = fe2.make_opts(precision="fp64")
    dummy = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = C.c_void_p(dummy.data_ptr())
    rc = lib.fe2_rve_solve_noalloc(4097, 10, p, p, p, p, p, -1.0, 1.0, C.byref(opts), p, p, p, p,
                                   p, None)
    assert rc == 1 and "n_nodes" in lib.fe2_noalloc_last_error().decode()
    rc = lib.fe2_rve_solve_noalloc(100, 16385, p, p, p, p, p, -1.0, 1.0, C.byref(opts), p, p, p,
                                   p, p, None)
    assert rc == 1 and "n_elems" in lib.fe2_noalloc_last_error().decode()
    mixed = fe2.make_opts(precision="mixed")
    rc = lib.fe2_rve_solve_noalloc(100, 10, p, p, p, p, p, -1.0, 1.0, C.byref(mixed), p, p, p, p,
                                   p, None)
    assert rc == 1
    assert lib.fe2_noalloc_scratch_bytes() < (4 << 20)


def _batched(net, F, c, u_warm=None, **opts):
    with fe2.Batch([net], damping=[c]) as b:
        if u_warm is not None:
            b.set_displacement(u_warm)
        b.solve(F[None], precision="fp64", **opts)
        ref = b.stress()
        ref["u"] = b.displacement()
    return ref


def _same_as_batched(out, ref):
    assert out["status"] == 0 and ref["status"][0] == "OK"
    assert out["iters"] == int(ref["iters"][0])
    assert np.array_equal(out["u"], ref["u"])
    err = np.linalg.norm(out["sigma"] - ref["sigma"][0]) / np.linalg.norm(ref["sigma"][0])
    assert err <= 1e-12, err


def test_noalloc_isolated_free_node_and_warm_start():
    """A free node that no element touches is held fixed, as on the batched
    path; a warm start reads the caller's displacement in caller order."""
    rng = np.random.default_rng(8)
    base = ri.random_network(400, rng)
    net = ri.Network(X=np.vstack([base.X, [[0.5, 0.5, 0.5]]]), elems=base.elems, EA=base.EA,
                     fixed=np.append(base.fixed, 0).astype(np.uint8))
    F = ri.symmetric_perturbation(rng)
    c = ri.default_damping(net.n_nodes)
    out = _noalloc(net, F, c, fe2.make_opts(precision="fp64", init="affine"))
    ref = _batched(net, F, c, init="affine")
    _same_as_batched(out, ref)
    # the isolated node moved affinely with the boundary and no further:
    # u = F X - X, each row summed left to right in plain double arithmetic
    X = [float(v) for v in net.X[-1]]
    Fx = [float(F[r, 0]) * X[0] + float(F[r, 1]) * X[1] + float(F[r, 2]) * X[2] for r in range(3)]
    assert out["u"][-1].tolist() == [Fx[r] - X[r] for r in range(3)]
    # warm restart under a further stretch, from the first solve's displacement
    F2 = np.diag([1.005, 1.0, 1.0]) @ F
    out2 = _noalloc_warm(net, F2, c, out["u"])
    ref2 = _batched(net, F2, c, u_warm=ref["u"], init="warm")
    _same_as_batched(out2, ref2)


def _noalloc_warm(net, F, c, u0):
    n, E = net.n_nodes, net.n_elems
    args = [_dev(net.X.reshape(-1), torch.float64), _dev(net.elems.reshape(-1), torch.int32),
            _dev(net.EA, torch.float64), _dev(net.fixed, torch.uint8),
            _dev(F.reshape(-1), torch.float64)]
    u = _dev(u0.reshape(-1), torch.float64)
    sig = torch.zeros(9, dtype=torch.float64, device="cuda")
    it = torch.zeros(1, dtype=torch.int64, device="cuda")
    rr = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    fe2.rve_solve_noalloc(n, E, *args, u, sig, it, rr, st, damping=c, precision="fp64",
                          init="warm")
    torch.cuda.synchronize()
    return {"u": u.cpu().numpy().reshape(n, 3), "sigma": sig.cpu().numpy().reshape(3, 3),
            "iters": int(it.item()), "rel_res": float(rr.item()), "status": int(st.item())}


def test_noalloc_device_side_input_checks():
    """Inputs the entry point can only see on the device are checked there
    before anything depends on them: status 4, zero iterations, no solve."""
    rng = np.random.default_rng(9)
    net = ri.random_network(60, rng)
    F = np.eye(3) * 1.01
    opts = fe2.make_opts(precision="fp64")
    bad = []
    el = net.elems.copy()
    bad.append(("repeated element", ri.Network(X=net.X, elems=np.vstack([el, el[:1]]),
                                               EA=np.append(net.EA, 1.0), fixed=net.fixed)))
    el2 = el.copy()
    el2[3] = [el2[3][0], el2[3][0]]
    bad.append(("self-loop", ri.Network(X=net.X, elems=el2, EA=net.EA, fixed=net.fixed)))
    el3 = el.copy()
    el3[5, 1] = net.n_nodes + 7
    bad.append(("id out of range", ri.Network(X=net.X, elems=el3, EA=net.EA, fixed=net.fixed)))
    X4 = net.X.copy()
    X4[10, 1] = np.nan
    bad.append(("non-finite coordinate", ri.Network(X=X4, elems=el, EA=net.EA, fixed=net.fixed)))
    X5 = net.X.copy()
    X5[el[0, 1]] = X5[el[0, 0]]
    bad.append(("zero length", ri.Network(X=X5, elems=el, EA=net.EA, fixed=net.fixed)))
    EA6 = net.EA.copy()
    EA6[2] = 0.0
    bad.append(("EA <= 0", ri.Network(X=net.X, elems=el, EA=EA6, fixed=net.fixed)))
    for what, b in bad:
        out = _noalloc(b, F, 0.01, opts)
        assert out["status"] == 4 and out["iters"] == 0, what
    # the same call with valid inputs afterwards still solves
    good = _noalloc(net, F, 0.01, opts)
    assert good["status"] == 0 and good["iters"] > 0
