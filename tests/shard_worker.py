"""Worker of the world_size-2 sharding test (runs in spawned processes).

Each rank joins a gloo group on 127.0.0.1, solves its share of the batch
with the FP64 oracle standing in for the GPU (the test exercises the
partition and the gather, which are host logic), and rank 0 saves the
gathered results.
"""
import os
import sys

import numpy as np


def _oracle_solve(nets, F, damping, **opts):
    import oracle
    sig, it, st = [], [], []
    code = {"OK": 0, "MAXITER": 1, "NAN": 2}
    for net, f, c in zip(nets, F, damping):
        r = oracle.solve(net, f, c, init=1, **opts)
        sig.append(r["sigma"])
        it.append(r["iters"])
        st.append(code[r["status"]])
    return np.array(sig).reshape(-1, 3, 3), np.array(it, np.int64), np.array(st, np.int32)


def run(rank, world, port, out_path, sizes, seed):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch.distributed as dist

    import rve_inputs as ri
    from paper_2305_07030_gb300.distributed import solve_sharded

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        rng = np.random.default_rng(seed)
        nets = [ri.random_network(int(n), rng) for n in sizes]
        F = np.array([ri.symmetric_perturbation(rng) for _ in nets])
        c = np.array([ri.default_damping(n.n_nodes) for n in nets])
        sig, it, st, rank_of = solve_sharded(nets, F, c, solve_fn=_oracle_solve, device="cpu",
                                             max_iter=3000)
        if rank == 0:
            np.savez(out_path, sigma=sig, iters=it, status=st, rank_of=rank_of)
    finally:
        dist.destroy_process_group()
