"""Benchmark: converged RVE solves/s of the batched dynamic-relaxation path.

One step = one batched solve of every RVE of the workload to convergence
(relative residual 1e-8, affine start) through the C ABI. Default: mixed
precision (FP32 force and update arithmetic, FP64 residual test and stress)
on 64 RVEs of 5,000 nodes (kNN k = 4, lognormal EA, F = I + 0.02 sym(G)).
Other workloads: the single 512-node RVE, the 1024 x log-U(1k, 33k) and
4096 x log-U(500, 20k) uneven batches, and their 64-RVE size-stratified
subsets (the RVEs the oracle checks); --precision fp64 runs the FP64 mode.

Prints ONE JSON line (rank 0). Per RVE the stress error against the FP64
oracle is reported from the stored oracle results of the workload
(tests/golden/oracle_stress_*.json, written by a script that runs only the
oracle). ``--impl reference`` times the FP64 CPU oracle instead (bounded
sample on the host cores). ``--serve`` runs the serving scenario,
``--experiments`` the paper's experiment shapes. Multi-GPU (torchrun):
every rank solves its own copy of the batch (independent replicas, weak
scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import rve_inputs as ri  # noqa: E402

_FIT = "kNN k=4, EA lognormal(0,0.3), F=I+0.02 sym(N(0,1)), tol 1e-8, affine start, " \
       "c=0.002(512/n)^(1/3)"


def _stratified(count, lo, hi, wl):
    idx = ri.stratified_idx(ri.uneven_sizes(count, lo, hi, wl), 64)
    return ri.uneven_subset(count, lo, hi, wl, idx)


# name -> (generator, description, stored oracle results, oracle RVE ids -> batch ids)
WORKLOADS = {
    "rve5000x64": (lambda: ri.equal_rves(64, 5000), f"64 RVEs x 5000 nodes, {_FIT}", "rve5000x64",
                   "same"),
    "rve512x1": (ri.single_rve_512, "1 RVE x 512 nodes, kNN k=4, EA=1, F=diag(1.05,1,1), tol 1e-8, "
                                    "affine start", "rve512x1", "same"),
    "uneven1k33k": (lambda: ri.uneven_rves(1024, 1000, 33000, 3),
                    f"1024 RVEs, nodes log-U(1000,33000), {_FIT}", "uneven1k33k", "ids"),
    "uneven500_20k": (lambda: ri.uneven_rves(4096, 500, 20000, 4),
                      f"4096 RVEs, nodes log-U(500,20000), {_FIT}", "uneven500_20k", "ids"),
    "uneven1k33k_s64": (lambda: _stratified(1024, 1000, 33000, 3),
                        f"64 of the 1024 RVEs log-U(1000,33000), stratified by size, {_FIT}",
                        "uneven1k33k", "same"),
    "uneven500_20k_s64": (lambda: _stratified(4096, 500, 20000, 4),
                          f"64 of the 4096 RVEs log-U(500,20000), stratified by size, {_FIT}",
                          "uneven500_20k", "same"),
}

# Algorithmic bytes per node-iteration of the relaxation (all nodes; 2.48
# elements per node; each element's data and each node's state counted once):
# mixed 104 B (u, v read+write 48, X 12, m 4, element 16 x 2.48), FP64 188 B.
BYTES_PER_NODE_ITER = {"mixed": 104.0, "fp64": 188.0}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"fe2_clocks_{os.getpid()}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# DRAM bytes (read + write) of one dr_mixed_fp32_kernel launch, scaled from
# one ncu capture of the same kernel: a 5000-node RVE of the 64 x 5000
# workload for 30,000 iterations read 1,940,224 B and wrote 5,888 B. The
# traffic is each RVE's data and state read once; it does not grow with
# iterations, so a launch's traffic scales with its number of RVEs.
FP32_DRAM_BYTES_PER_RVE = 1_940_224 + 5_888


def fp32_dram_traffic(n_rve):
    return float(FP32_DRAM_BYTES_PER_RVE * n_rve)


def golden(name):
    path = os.path.join(ROOT, "tests", "golden", f"oracle_stress_{name}.json")
    try:
        with open(path) as f:
            return json.load(f)
    except OSError:
        return None


def stress_errors(args, sigma, status):
    """Per-RVE relative (Frobenius) stress error against the stored FP64
    oracle results of this workload, and the count above each bound."""
    _, _, gname, ids = WORKLOADS[args.workload]
    if args.rves:
        return {"available": False, "why": "RVE subset run"}
    g = golden(gname)
    if g is None:
        return {"available": False, "why": f"no stored oracle results for {gname}"}
    rows = []
    for k, r in enumerate(g["results"]):
        p = k if ids == "same" else int(g["rves"][k])
        ref = np.array(r["sigma"]).reshape(3, 3)
        err = float(np.linalg.norm(sigma[p] - ref) / np.linalg.norm(ref))
        diam = float(r.get("diameter", r.get("envelope", 0.0)))
        rows.append((p, err, diam, status[p] == 0 and r["status"] == "OK"))
    errs = np.array([x[1] for x in rows])
    bound = np.array([max(1e-5, x[2]) for x in rows])
    return {"available": True, "vs": f"FP64 oracle, tests/golden/oracle_stress_{gname}.json "
                                     f"({g['what']})",
            "n": len(rows), "max": float(errs.max()), "median": float(np.median(errs)),
            "over_1e-5": int((errs > 1e-5).sum()),
            "over_bound": int((errs > bound).sum()),
            "bound": "max(1e-5, diameter of the oracle's own rounding family)",
            "well_conditioned": {"n": int(sum(x[2] <= 1e-6 for x in rows)),
                                 "max": float(max([x[1] for x in rows if x[2] <= 1e-6], default=0.0))},
            "both_converged": int(sum(x[3] for x in rows)),
            "per_rve": [[x[0], round(x[1], 12), round(x[2], 12)] for x in rows]}


def fp64_alu_seconds(nets, iters, rates):
    """Lower bound on the FP64 kernel's time from its operation counts and the
    measured FP64 rates: per element with a free end 13 add/multiply, 2
    divisions and 1 square root; per free node 34 + 3 x degree add/multiply
    and 3 divisions (the update, the element-table sum, damping, residual,
    acceleration and velocity), every operation on the FP64 pipe."""
    fma, div, sqrt = rates
    t = 0.0
    for n, it in zip(nets, iters):
        deg = np.bincount(n.elems.ravel(), minlength=n.n_nodes)
        free = (n.fixed == 0) & (deg > 0)
        ef = int((free[n.elems[:, 0]] | free[n.elems[:, 1]]).sum())
        nf = int(free.sum())
        addmul = 13 * ef + 34 * nf + 3 * int(deg[free].sum())
        t += int(it) * (addmul / fma + (2 * ef + 3 * nf) / div + ef / sqrt)
    return t


def _plan_summary(fe2, nets):
    """Per launch class of the mixed solver: RVEs, cluster size, and per kernel
    (lead, FP32) whether the element table is staged and the CTA size."""
    P = fe2.plan(nets)
    return [{"rves": int(P["rves"][c]), "parts": int(P["parts"][c]),
             "staged": [int(x) for x in P["staged"][c]], "block": [int(x) for x in P["block"][c]]}
            for c in range(P["n_classes"])]


def run_ours(args, rank, world):
    import torch
    import paper_2305_07030_gb300 as fe2

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    w = WORKLOADS[args.workload][0]()
    if args.rves:
        w = w.subset([int(x) for x in args.rves.split(",")])
    nets = w.nets
    P = len(nets)
    mixed = args.precision == "mixed"
    if args.autotune and mixed:
        # tune the cluster and CTA sizes per size bucket on up to 16 RVEs
        # spread over the sizes, before the batch is created
        pick = ri.stratified_idx([n.n_nodes for n in nets], min(16, P))
        sub = w.subset(pick)
        fe2.autotune(sub.nets, sub.F, sub.damping, trial_iters=args.autotune_iters)
    batch = fe2.Batch(nets, damping=w.damping)
    opts = dict(precision=args.precision, init="affine", tol=1e-8, max_iter=args.max_iter,
                lead_iters=args.lead_iters, lead_tol=args.lead_tol, block_threads=args.block,
                launch=args.launch)
    F_host = np.ascontiguousarray(w.F.reshape(P, 9))
    F_dev = torch.tensor(F_host.reshape(-1), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    sig_dev = torch.zeros(9 * P, dtype=torch.float64, device="cuda")
    it_dev = torch.zeros(P, dtype=torch.int64, device="cuda")
    st_dev = torch.zeros(P, dtype=torch.int32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > L2 (129 MB)
    dist = world > 1
    if dist:
        import torch.distributed as tdist

    def barrier():
        if dist:
            tdist.barrier()
        torch.cuda.synchronize()

    def step_device():
        batch.solve_dev(F_dev, stream=stream, **opts)
        batch.results_dev(sigma_dev=sig_dev, iters_dev=it_dev, status_dev=st_dev, stream=stream)

    for _ in range(args.warmup):
        step_device()
    barrier()
    times, kernel_ms, iters_all = [], [], []
    with ClockSampler(dev) as clk:
        for _ in range(args.steps):
            flush.fill_(1)
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step_device()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
            kernel_ms.append(batch.kernel_times_ms())
            iters_all.append(it_dev.cpu().numpy().copy())
        # end-to-end through the public API with host buffers: H2D of F from
        # pinned memory and D2H of the stresses inside the timed region
        e2e_times = []
        for _ in range(max(1, min(args.steps, 3))):
            flush.fill_(1)
            barrier()
            t0 = time.perf_counter()
            batch.solve(F_host, **opts)
            res = batch.stress()
            e2e_times.append(time.perf_counter() - t0)
    clocks = clk.summary()
    launches = batch.info()["launches"]
    if dist:
        tt = torch.tensor([max(times), max(e2e_times)], dtype=torch.float64, device="cuda")
        tdist.all_reduce(tt, op=tdist.ReduceOp.MAX)
        t_e2e = float(tt[1])
    else:
        t_e2e = max(e2e_times)
    mean_step = statistics.mean(times)
    iters = iters_all[-1]
    nn = np.array([n.n_nodes for n in nets])
    if rank != 0:
        batch.close()
        return None
    sigma = res["sigma"]
    status = np.array([{"OK": 0, "MAXITER": 1, "NAN": 2}.get(x, 3) for x in res["status"]])
    leads = batch.diagnostics()["lead_iters"] if mixed else np.zeros(P, int)
    smem_gbs, _ = fe2.probe_smem_bandwidth()
    per_launch = 3 if mixed else 1
    n_cls = len(kernel_ms[-1]) // per_launch
    if mixed:
        # the dominant kernel: the FP32 phase; roofline per launch on the
        # node-iterations it ran (all nodes of its RVEs, FP32 iterations only)
        cls = fe2.plan(nets)["rve_class"]
        best = None
        for c in range(n_cls):
            members = np.nonzero(cls == c)[0]
            alg = BYTES_PER_NODE_ITER["mixed"] * float(sum(nn[p] * (int(iters[p]) - int(leads[p]))
                                                           for p in members))
            kms = statistics.mean(k[per_launch * c + 1] for k in kernel_ms)
            if best is None or kms > best[1]:
                best = (alg, kms, len(members))
        alg, kms, n_in = best
        achieved = alg / (kms * 1e-3) / 1e9
        roof = {"bound": "smem", "achieved": achieved, "peak": smem_gbs, "unit": "GB/s",
                "frac": achieved / smem_gbs, "traffic": fp32_dram_traffic(n_in),
                "kernel": "dr_mixed_fp32_kernel", "kernel_ms": kms,
                "lead_kernel_ms": statistics.mean(sum(k[per_launch * c] for c in range(n_cls))
                                                  for k in kernel_ms),
                "resume_kernel_ms": statistics.mean(sum(k[per_launch * c + 2] for c in range(n_cls))
                                                    for k in kernel_ms),
                "lead_iters_mean": float(np.mean(leads)),
                "bytes_per_node_iter": BYTES_PER_NODE_ITER["mixed"],
                "units": "node-iterations of the FP32 phase (all nodes of the launch's RVEs)",
                "step_frac": BYTES_PER_NODE_ITER["mixed"] * float((nn * iters).sum()) / mean_step / 1e9
                / smem_gbs,
                "peak_source": "measured live: fe2_probe_smem_bandwidth (float4 shared-memory "
                               "reads on every SM)"}
    else:
        rates = fe2.probe_fp64_rates()
        kms = statistics.mean(sum(k) for k in kernel_ms) / max(1, n_cls)
        kmax = statistics.mean(max(k) for k in kernel_ms)
        t_alu = fp64_alu_seconds(nets, iters, rates)
        node_iters = float((nn * iters).sum())
        roof = {"bound": "alu", "achieved": node_iters / (kmax * 1e-3) / 1e9,
                "peak": node_iters / t_alu / 1e9, "unit": "G node-iterations/s",
                "frac": t_alu / (kmax * 1e-3), "traffic": None, "kernel": "dr_fp64_kernel / dr_fp64_cluster_kernel",
                "kernel_ms": kmax, "kernel_ms_mean_per_class": kms,
                "fp64_rates_per_s": {"fma": rates[0], "div": rates[1], "sqrt": rates[2]},
                "peak_source": "derived: the kernel's FP64 operation counts per element and free "
                               "node at the rates measured live by fe2_probe_fp64_rates",
                "smem_view": {"bytes_per_node_iter": BYTES_PER_NODE_ITER["fp64"],
                              "GBps": BYTES_PER_NODE_ITER["fp64"] * node_iters / (kmax * 1e-3) / 1e9,
                              "frac_of_smem": BYTES_PER_NODE_ITER["fp64"] * node_iters /
                              (kmax * 1e-3) / 1e9 / smem_gbs}}
    value = world * P / mean_step
    dof_iters = float((3 * nn * iters).sum())
    out = {
        "metric": "converged RVE solves/s",
        "value": value,
        "unit": "solves/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": mean_step * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64" if mixed else "f64",
        "data": "synthetic",
        # the workload alone, identical in the reference arm's line
        "config": {"workload": WORKLOADS[args.workload][1]},
        "run": {"precision": args.precision, "rves": P, "nodes": int(nn.sum()),
                "launch": args.launch, "lead_tol": args.lead_tol,
                "l2": "flushed between steps (256 MB write)",
                "tuning": {str(k): list(v) for k, v in fe2.tuning_get().items()},
                "classes": _plan_summary(fe2, nets) if mixed else None,
                "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "dof_iters_per_s": world * dof_iters / mean_step,
        "iters": {"mean": float(iters.mean()), "min": int(iters.min()), "max": int(iters.max())},
        "converged": int((status == 0).sum()),
        "e2e": {"value": world * P / t_e2e, "unit": "solves/s", "samples": len(e2e_times),
                "h2d_bytes_per_step": 9 * 8 * P, "d2h_bytes_per_step": (9 * 8 + 8 + 8 + 4) * P},
        "gpu_launches": launches,
        "roofline": roof,
        "stress_err": stress_errors(args, sigma, status),
        "clocks": clocks,
    }
    if args.dump:
        np.savez(args.dump, sigma=sigma, iters=iters, status=status, n_nodes=nn,
                 lead=np.asarray(leads), kernel_ms=np.asarray(kernel_ms[-1]),
                 rve_class=(fe2.plan(nets)["rve_class"] if mixed else np.zeros(P, np.int32)))
    if mixed and args.workload == "rve5000x64" and not args.no_naive:
        nv = naive_comparator(w, iters)
        nv["speedup_of_batched"] = value / nv["solves_per_s"]
        out["naive_fp64"] = nv
    if not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(w, iters, args.cpu_seconds)
    batch.close()
    return out


def naive_comparator(w, iters):
    """The paper's naive per-RVE FP64 launch loop on the same GPU, timed on a
    bounded sample (RVE 0 in a batch of its own, capped iteration count) and
    scaled to whole solves with the batched path's mean iteration count."""
    import paper_2305_07030_gb300 as fe2
    cap = 3000
    b1 = fe2.Batch(w.nets[:1], damping=w.damping[:1])
    b1.solve_naive(w.F[:1], init="affine", tol=1e-8, max_iter=200)  # warm-up
    t0 = time.perf_counter()
    b1.solve_naive(w.F[:1], init="affine", tol=1e-8, max_iter=cap)
    dt = time.perf_counter() - t0
    r = b1.stress()
    b1.close()
    done = int(r["iters"][0])
    per_iter = dt / done
    return {"solves_per_s": 1.0 / (per_iter * float(np.mean(iters))),
            "s_per_iteration": per_iter,
            "sample": f"RVE 0 ({w.nets[0].n_nodes} nodes) for {done} iterations; solves/s = "
                      f"1/(s_per_iteration x mean batched iterations)"}


def cpu_baseline(w, iters, seconds):
    """The FP64 oracle on the host cores, bounded sample: one RVE per core
    (spread over the batch), each capped at a fixed iteration count, scaled to
    solves with the batched path's mean DOF-iterations per solve."""
    import oracle
    cores = os.cpu_count() or 1
    k = min(cores, w.n_rve)
    sub = w.subset(np.rint(np.linspace(0, w.n_rve - 1, k)).astype(int).tolist())
    # calibrate the cap so that the sample takes about `seconds`
    t0 = time.perf_counter()
    oracle.solve(sub.nets[0], sub.F[0], sub.damping[0], init=1, max_iter=200)
    per_iter = (time.perf_counter() - t0) / 200 * max(n.n_nodes for n in sub.nets) / sub.nets[0].n_nodes
    cap = max(200, int(seconds / per_iter))
    t0 = time.perf_counter()
    res = oracle.solve_batch(sub, init=1, max_iter=cap, threads=k)
    dt = time.perf_counter() - t0
    it_done = sum(r["iters"] for r in res)
    dof_iters = sum(3 * sub.nets[p].n_nodes * res[p]["iters"] for p in range(k))
    nn = np.array([n.n_nodes for n in w.nets])
    per_solve = float(np.mean(3.0 * nn * np.asarray(iters)))
    solves = dof_iters / dt / per_solve
    return {"value": solves, "unit": "solves/s", "cores": k, "kind": "oracle",
            "dof_iters_per_s": dof_iters / dt,
            "sample": f"{k} RVEs in parallel, at most {cap} iterations each ({it_done} total, "
                      f"{dt:.1f} s); solves/s = DOF-iters/s / mean DOF-iterations of a batched "
                      f"solve ({per_solve:.4g})"}


def oracle_dofs_per_solve(workload):
    """Mean DOF-iterations (3 x nodes x iterations) of one converged oracle
    solve of this workload, from the stored oracle results (the workload's
    RVEs, or its size-stratified 64-RVE subset for the uneven batches)."""
    g = golden(WORKLOADS[workload][2])
    if g is not None:
        d = [3.0 * r["n_nodes"] * r["iters"] for r in g["results"]]
        return float(np.mean(d)), f"oracle's own iteration counts ({g['what']})"
    return float("nan"), "stored oracle results missing"


def run_reference(args):
    """The FP64 CPU oracle as the reference arm (bounded sample per step)."""
    import oracle
    name = args.workload
    if name in ("uneven1k33k", "uneven500_20k"):
        name += "_s64"  # the sample comes from the size-stratified subset
    w = WORKLOADS[name][0]()
    cores = os.cpu_count() or 1
    k = min(cores, w.n_rve)
    sub = w.subset(np.rint(np.linspace(0, w.n_rve - 1, k)).astype(int).tolist())
    per_step = max(1.0, 60.0 / max(1, args.steps + args.warmup))
    t0 = time.perf_counter()
    oracle.solve(sub.nets[0], sub.F[0], sub.damping[0], init=1, max_iter=200)
    per_iter = (time.perf_counter() - t0) / 200 * max(n.n_nodes for n in sub.nets) / sub.nets[0].n_nodes
    cap = max(200, int(per_step / per_iter))
    for _ in range(args.warmup):
        oracle.solve_batch(sub, init=1, max_iter=max(200, cap // 10), threads=k)
    times, dofs = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        res = oracle.solve_batch(sub, init=1, max_iter=cap, threads=k)
        times.append(time.perf_counter() - t0)
        dofs.append(sum(3 * sub.nets[p].n_nodes * res[p]["iters"] for p in range(k)))
    dof_rate = sum(dofs) / sum(times)
    per_solve, src = oracle_dofs_per_solve(args.workload)
    value = dof_rate / per_solve
    return {"metric": "converged RVE solves/s", "value": value, "unit": "solves/s",
            "impl": "reference", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload][1]},
            "run": {"precision": "fp64 (oracle)", "parallelism": f"{k} host threads"},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": k, "kind": "oracle",
                             "sample": f"{k} RVEs on {k} threads, at most {cap} iterations each "
                                       f"per step; solves/s = DOF-iters/s / {per_solve:.4g} "
                                       f"DOF-iterations per solve, the {src}"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def run_serving(args):
    """Serving scenario: Gauss points of a synthetic macroscale mesh emit one
    RVE request per macro step; arrivals are Poisson; F grows by 0.5 % stretch
    per step; each RVE restarts warm from its previous step, on the device.
    Reports throughput and p50/p99 request latency (arrival to completion)."""
    import torch
    import paper_2305_07030_gb300 as fe2
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    n_pts, n_steps = args.serve_points, args.serve_steps
    sizes, S, arrivals = ri.serving_requests(n_pts, n_steps, args.serve_lo, args.serve_hi,
                                             rate=args.serve_rate)
    nets = []
    for g in range(n_pts):
        rng = np.random.Generator(np.random.PCG64((ri.SEED_BASE + 5) * 1000 + g))
        nets.append(ri.random_network(int(sizes[g]), rng))
    damping = np.array([ri.default_damping(int(n)) for n in sizes])
    rve, t_arr, F = [], [], []
    for k in range(n_steps):
        for g in range(n_pts):
            rve.append(g)
            t_arr.append(arrivals[k, g])
            F.append(ri.serving_F(S[g], k))
    order = np.argsort(np.array(t_arr), kind="stable")
    rve = np.array(rve, np.int32)[order]
    t_arr = np.array(t_arr)[order]
    t_arr -= t_arr[0]
    F = np.array(F)[order]
    with fe2.Batch(nets, damping=damping) as b:
        t0 = time.perf_counter()
        out = b.serve(rve, t_arr, F, max_batch=args.serve_batch,
                      max_inflight_bytes=args.serve_inflight_gb * 1e9,
                      first=dict(max_iter=args.max_iter),
                      next=dict(max_iter=args.max_iter, init="warm"))
        wall = time.perf_counter() - t0
    lat = out["t_done"] - t_arr
    return {"metric": "serving p99 latency", "value": float(np.percentile(lat, 99)), "unit": "s",
            "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
            "dtype": "f32+f64",
            "config": {"workload": f"{n_pts} Gauss points x {n_steps} macro steps, RVE nodes "
                                   f"log-U({args.serve_lo},{args.serve_hi}), Poisson arrivals "
                                   f"{args.serve_rate}/s, F=diag(1+0.005k,1,1)(I+0.02 S), warm "
                                   f"restarts, micro-batches <= {args.serve_batch}, in-flight "
                                   f"budget {args.serve_inflight_gb or 'none'} GB, max_iter "
                                   f"{args.max_iter}"},
            "latency_p50_s": float(np.percentile(lat, 50)),
            "latency_p99_s": float(np.percentile(lat, 99)),
            "latency_max_s": float(lat.max()),
            "requests": int(len(rve)), "wall_s": wall,
            "throughput_req_per_s": len(rve) / wall,
            "iters_first_step_mean": float(out["iters"][:n_pts].mean()),
            "iters_mean": float(out["iters"].mean()),
            "status_ok": int((out["status"] == 0).sum()),
            # [request, RVE, RVE nodes, status, iterations] of every request that did not converge
            "not_ok": [[int(i), int(rve[i]), int(sizes[rve[i]]), int(out["status"][i]),
                        int(out["iters"][i])] for i in np.nonzero(out["status"] != 0)[0]]}


def run_experiments(args):
    """The paper's experiment shapes (Results, Figs. 2-4) on synthetic RVEs:
    self-speedup of the batched persistent solver against the number of
    concurrent RVEs for three sizes, a sweep of the CTA (team) size including
    the paper's 512 threads, and two comparators at each concurrency: a
    multi-stream baseline that solves every RVE as a batch of its own on its
    own stream (the stand-in for the paper's 32 MPS ranks sharing one GPU) and
    the naive per-RVE launch loop. Every RVE runs exactly K iterations
    (tol = 0, max_iter = K), so times compare equal work; self-speedup(N) =
    N T(1) / T(N)."""
    import torch
    import paper_2305_07030_gb300 as fe2
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    K = args.exp_iters
    sizes = [int(x) for x in args.exp_sizes.split(",")]
    counts = [int(x) for x in args.exp_counts.split(",")]
    blocks = [int(x) for x in args.exp_blocks.split(",")]
    stream = torch.cuda.current_stream()

    def timed(fn, reps=2):
        fn()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            best = min(best, time.perf_counter() - t0)
        return best

    out = {"metric": "experiment shapes", "iterations_per_rve": K, "sizes": {}}
    for n in sizes:
        rng = np.random.Generator(np.random.PCG64((ri.SEED_BASE + 6) * 1000 + n))
        net = ri.random_network(n, rng)
        F = ri.symmetric_perturbation(rng)
        c = ri.default_damping(n)
        rows = {}
        for prec in ("mixed", "fp64"):
            opts = dict(precision=prec, tol=0.0, max_iter=K, lead_iters=K // 10)
            for blk in blocks:
                tl = []
                for N in counts:
                    with fe2.Batch([net] * N, damping=[c] * N) as b:
                        Fd = torch.tensor(np.tile(F.reshape(-1), N), dtype=torch.float64,
                                          device="cuda")
                        t = timed(lambda: b.solve_dev(Fd, stream=stream, block_threads=blk, **opts))
                    tl.append(t)
                rows[f"{prec}_block{blk}"] = {
                    "seconds": tl, "self_speedup": [N * tl[0] / t for N, t in zip(counts, tl)]}
            # multi-stream comparator: one single-RVE batch per stream, all at once
            ms = []
            for N in counts:
                if N > args.exp_mps_max:
                    ms.append(None)
                    continue
                bs = [fe2.Batch([net], damping=[c]) for _ in range(N)]
                streams = [torch.cuda.Stream() for _ in range(N)]
                Fd = torch.tensor(F.reshape(-1), dtype=torch.float64, device="cuda")

                def all_streams():
                    for b, st in zip(bs, streams):
                        b.solve_dev(Fd, stream=st, **opts)
                ms.append(timed(all_streams))
                for b in bs:
                    b.close()
            rows[f"{prec}_multistream"] = {"seconds": ms}
        # the naive per-RVE loop (RVEs one after another): one RVE, scaled by N
        with fe2.Batch([net], damping=[c]) as b:
            kn = min(K, args.exp_naive_iters)
            t1 = timed(lambda: b.solve_naive(F[None], tol=0.0, max_iter=kn), reps=1) * K / kn
        rows["naive_fp64"] = {"seconds": [N * t1 for N in counts],
                              "note": f"one RVE for {kn} iterations, scaled to K and to N RVEs"}
        out["sizes"][str(n)] = {"nodes": n, "elements": int(net.n_elems), "counts": counts,
                                "rows": rows}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rve5000x64", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-naive", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--rves", default="", help="comma-separated RVE subset (profiling runs)")
    ap.add_argument("--max-iter", type=int, default=10_000_000)
    ap.add_argument("--lead-iters", type=int, default=-1)
    ap.add_argument("--lead-tol", type=float, default=1e-2,
                    help="mixed: relative residual that ends the double-float lead")
    ap.add_argument("--block", type=int, default=0, help="threads per CTA (0 = library default)")
    ap.add_argument("--launch", default="graph", choices=["graph", "stream"],
                    help="replay the solve as a CUDA graph (default) or launch on streams")
    ap.add_argument("--tuning", default="", help="JSON file written by fe2_autotune to load first")
    ap.add_argument("--dump", default="", help="write the per-RVE results (npz) to this path")
    ap.add_argument("--autotune", action="store_true",
                    help="mixed: run fe2_autotune on a size-stratified sample first")
    ap.add_argument("--autotune-iters", type=int, default=2000)
    ap.add_argument("--tune", default="",
                    help="explicit tuning: bucket:parts:block_fp32[:block_lead],... (2^bucket <= nodes)")
    ap.add_argument("--serve", action="store_true", help="run the serving scenario instead")
    ap.add_argument("--experiments", action="store_true",
                    help="run the paper's experiment shapes (self-speedup, team size, comparators)")
    ap.add_argument("--exp-iters", type=int, default=2000)
    ap.add_argument("--exp-sizes", default="1000,5000,20000")
    ap.add_argument("--exp-counts", default="1,2,4,8,16,32,64,128,256")
    ap.add_argument("--exp-blocks", default="256,512")
    ap.add_argument("--exp-mps-max", type=int, default=32)
    ap.add_argument("--exp-naive-iters", type=int, default=200)
    ap.add_argument("--serve-points", type=int, default=128)
    ap.add_argument("--serve-steps", type=int, default=3)
    ap.add_argument("--serve-lo", type=int, default=1000)
    ap.add_argument("--serve-hi", type=int, default=8000)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-batch", type=int, default=32)
    ap.add_argument("--serve-inflight-gb", type=float, default=0.0,
                    help="budget of the in-flight working set (GB); 0 = none")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.serve:
        if rank == 0:
            print(json.dumps(run_serving(args)))
        return
    if args.experiments:
        if rank == 0:
            print(json.dumps(run_experiments(args)))
        return
    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(run_reference(args)))
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        tdist.init_process_group("nccl")
        args.no_cpu = args.no_cpu or rank != 0
        args.no_naive = args.no_naive or rank != 0
    if args.tuning or args.tune:
        import paper_2305_07030_gb300 as fe2
        if args.tuning:
            fe2.tuning_load(args.tuning)
        if args.tune:
            ent = fe2.tuning_get()
            for item in args.tune.split(","):
                v = [int(x) for x in item.split(":")]
                ent[v[0]] = tuple(v[1:]) + (0,) * (4 - len(v))
            fe2.tuning_set(ent)
    out = run_ours(args, rank, world)
    if out is not None:
        print(json.dumps(out))
    if world > 1:
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
