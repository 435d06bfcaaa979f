"""Benchmark: converged RVE solves/s of the batched dynamic-relaxation path.

One step = one batched solve of every RVE of the workload to convergence
(relative residual 1e-8) through the C ABI, mixed precision (FP32 force and
update arithmetic, FP64 residual test and stress). Default workload: 64 RVEs
of 5,000 nodes (kNN k = 4, lognormal EA, F = I + 0.02 sym(G)), the
equal-size batch on which the naive per-RVE FP64 launch loop is compared.

Prints ONE JSON line (rank 0). ``--impl reference`` times the FP64 CPU oracle
instead (bounded sample on the host cores). Multi-GPU (torchrun): every rank
solves its own copy of the batch (independent replicas, weak scaling).
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

WORKLOADS = {
    "rve5000x64": lambda: ri.equal_rves(64, 5000),
    "rve512x1": ri.single_rve_512,
}
WORKLOAD_TEXT = {
    "rve5000x64": "64 RVEs x 5000 nodes, kNN k=4, EA lognormal(0,0.3), F=I+0.02 sym(N(0,1)), "
                  "tol 1e-8, affine start, c=0.002(512/n)^(1/3)",
    "rve512x1": "1 RVE x 512 nodes, kNN k=4, EA=1, F=diag(1.05,1,1), tol 1e-8, affine start",
}


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


def run_ours(args, rank, world):
    import torch
    import paper_2305_07030_gb300 as fe2

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    w = WORKLOADS[args.workload]()
    if args.rves:
        w = w.subset([int(x) for x in args.rves.split(",")])
    nets = w.nets
    P = len(nets)
    batch = fe2.Batch(nets, damping=w.damping)
    opts = dict(precision=args.precision, init="affine", tol=1e-8, max_iter=args.max_iter,
                lead_iters=args.lead_iters, block_threads=args.block)
    F_host = np.ascontiguousarray(w.F.reshape(P, 9))
    F_dev = torch.tensor(F_host.reshape(-1), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    sig_dev = torch.zeros(9 * P, dtype=torch.float64, device="cuda")
    it_dev = torch.zeros(P, dtype=torch.int64, device="cuda")
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
        batch.results_dev(sigma_dev=sig_dev, iters_dev=it_dev, stream=stream)

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
        for _ in range(max(1, min(args.steps, 2))):
            flush.fill_(1)
            barrier()
            t0 = time.perf_counter()
            batch.solve(F_host, **opts)
            res = batch.stress()
            e2e_times.append(time.perf_counter() - t0)
    clocks = clk.summary()
    launches = batch.info()["launches"]
    t_step = max(times) if not dist else None
    if dist:
        tt = torch.tensor([max(times), max(e2e_times)], dtype=torch.float64, device="cuda")
        tdist.all_reduce(tt, op=tdist.ReduceOp.MAX)
        t_step, t_e2e = float(tt[0]), float(tt[1])
    else:
        t_e2e = max(e2e_times)
    mean_step = statistics.mean(times)
    iters = iters_all[-1]
    nn = np.array([n.n_nodes for n in nets])
    if rank != 0:
        return None
    # per-RVE free nodes and directed edges touching free nodes (from the inputs)
    stats = []
    for n in nets:
        fx = n.fixed.astype(bool)
        deg = np.bincount(n.elems.ravel(), minlength=n.n_nodes)
        stats.append((int((~fx).sum()), int(deg[~fx].sum())))
    # Algorithmic shared-memory bytes of the dominant kernel per launch: the FP32
    # kernel reads every neighbour's staged position and increment (32 B per
    # directed edge) and reads/writes each free node's own (48 B); the FP64
    # kernel reads 24 B per edge and writes 24 B per free node.
    leads = batch.diagnostics()["lead_iters"] if args.precision == "mixed" else np.zeros(P, int)
    if args.precision == "fp64":
        alg = sum(int(it) * (24.0 * nnz + 24.0 * nf) for (nf, nnz), it in zip(stats, iters))
        kms = statistics.mean(k[0] for k in kernel_ms)
        kname = "dr_fp64_kernel"
    else:
        alg = sum((int(it) - int(ld)) * (32.0 * nnz + 48.0 * nf)
                  for (nf, nnz), it, ld in zip(stats, iters, leads))
        kms = statistics.mean(k[1] for k in kernel_ms)  # [lead, fp32] per step
        kname = "dr_mixed_fp32_kernel"
    lead_ms = statistics.mean(k[0] for k in kernel_ms) if args.precision == "mixed" else 0.0
    smem_gbs, _ = fe2.probe_smem_bandwidth()
    achieved = alg / (kms * 1e-3) / 1e9
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
        "dtype": "f32+f64" if args.precision == "mixed" else "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT[args.workload], "precision": args.precision,
                   "l2": "flushed between steps (256 MB write)",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "dof_iters_per_s": world * dof_iters / mean_step,
        "iters": {"mean": float(iters.mean()), "min": int(iters.min()), "max": int(iters.max())},
        "e2e": {"value": world * P / t_e2e, "unit": "solves/s",
                "h2d_bytes_per_step": 9 * 8 * P, "d2h_bytes_per_step": (9 * 8 + 8 + 8 + 4) * P},
        "gpu_launches": launches,
        "roofline": {"bound": "smem", "achieved": achieved, "peak": smem_gbs, "unit": "GB/s",
                     "frac": achieved / smem_gbs,
                     "traffic": fp32_dram_traffic(P) if args.precision == "mixed" else None,
                     "kernel": kname, "kernel_ms": kms, "lead_kernel_ms": lead_ms,
                     "lead_iters_mean": float(np.mean(leads)),
                     "peak_source": "measured live: fe2_probe_smem_bandwidth (float4 shared-memory "
                                    "reads on every SM)"},
        "clocks": clocks,
    }
    if not args.no_naive:
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
    """The FP64 oracle on the host cores, bounded sample: one RVE per core,
    each capped at a fixed iteration count, scaled to solves with the batched
    path's mean iteration count."""
    import oracle
    cores = os.cpu_count() or 1
    k = min(cores, w.n_rve)
    sub = w.subset(range(k))
    # calibrate the cap so that the sample takes about `seconds`
    t0 = time.perf_counter()
    oracle.solve(sub.nets[0], sub.F[0], sub.damping[0], init=1, max_iter=200)
    per_iter = (time.perf_counter() - t0) / 200
    cap = max(200, int(seconds / per_iter))
    t0 = time.perf_counter()
    res = oracle.solve_batch(sub, init=1, max_iter=cap, threads=k)
    dt = time.perf_counter() - t0
    it_done = sum(r["iters"] for r in res)
    dof_iters = sum(3 * sub.nets[p].n_nodes * res[p]["iters"] for p in range(k))
    mean_n = float(np.mean([n.n_nodes for n in w.nets]))
    solves = dof_iters / dt / (3 * mean_n * float(np.mean(iters)))
    return {"value": solves, "unit": "solves/s", "cores": k, "kind": "oracle",
            "dof_iters_per_s": dof_iters / dt,
            "sample": f"{k} RVEs in parallel, {cap} iterations each ({it_done} total, {dt:.1f} s); "
                      f"solves/s = DOF-iters/s / (3 x mean nodes x mean batched iterations)"}


def oracle_iterations(workload):
    """Mean iterations to convergence of the oracle on this workload."""
    path = os.path.join(ROOT, "tests", "golden", "oracle_iterations.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(np.mean(d[workload]["iters"])), "oracle's own mean iteration count"
    except (OSError, KeyError):
        return float("nan"), "oracle iteration counts missing"


def run_reference(args):
    """The FP64 CPU oracle as the reference arm (bounded sample per step)."""
    import oracle
    w = WORKLOADS[args.workload]()
    cores = os.cpu_count() or 1
    k = min(cores, w.n_rve)
    sub = w.subset(range(k))
    per_step = max(1.0, 60.0 / max(1, args.steps + args.warmup))
    t0 = time.perf_counter()
    oracle.solve(sub.nets[0], sub.F[0], sub.damping[0], init=1, max_iter=200)
    per_iter = (time.perf_counter() - t0) / 200
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
    # iterations per solve: the oracle's own counts to convergence for this
    # workload (tests/golden/oracle_iterations.json, written by a script that
    # runs only the oracle)
    iters_per_solve, src = oracle_iterations(args.workload)
    mean_n = float(np.mean([n.n_nodes for n in w.nets]))
    value = dof_rate / (3 * mean_n * iters_per_solve)
    return {"metric": "converged RVE solves/s", "value": value, "unit": "solves/s",
            "impl": "reference", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT[args.workload], "precision": "fp64 (oracle)"},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": k, "kind": "oracle",
                             "sample": f"{k} RVEs on {k} threads, {cap} iterations each per step; "
                                       f"solves/s = DOF-iters/s / (3 x {mean_n:.0f} x "
                                       f"{iters_per_solve:.0f} iterations per solve, {src})"},
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
        out = b.serve(rve, t_arr, F, max_batch=args.serve_batch)
        wall = time.perf_counter() - t0
    lat = out["t_done"] - t_arr
    return {"metric": "serving p99 latency", "value": float(np.percentile(lat, 99)), "unit": "s",
            "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
            "dtype": "f32+f64",
            "config": {"workload": f"{n_pts} Gauss points x {n_steps} macro steps, RVE nodes "
                                   f"log-U({args.serve_lo},{args.serve_hi}), Poisson arrivals "
                                   f"{args.serve_rate}/s, F=diag(1+0.005k,1,1)(I+0.02 S), warm "
                                   f"restarts, micro-batches <= {args.serve_batch}"},
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
    ap.add_argument("--block", type=int, default=0, help="threads per CTA (0 = library default)")
    ap.add_argument("--serve", action="store_true", help="run the serving scenario instead")
    ap.add_argument("--serve-points", type=int, default=128)
    ap.add_argument("--serve-steps", type=int, default=3)
    ap.add_argument("--serve-lo", type=int, default=1000)
    ap.add_argument("--serve-hi", type=int, default=8000)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-batch", type=int, default=32)
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.serve:
        if rank == 0:
            print(json.dumps(run_serving(args)))
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
    out = run_ours(args, rank, world)
    if out is not None:
        print(json.dumps(out))
    if world > 1:
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
