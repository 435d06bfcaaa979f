"""Batches sharded over several GPUs, one process per GPU (torch.distributed).

The microscale problems of the FE2 scheme are independent (Section I), so a
batch shards with no exchange while the relaxation runs: every rank computes
the same longest-processing-time partition (fe2_shard_plan), solves its own
RVEs through the C ABI on its GPU, and the per-RVE results (9 stress
components, iteration count, status) are all-gathered so that every rank
holds the whole batch's results in the caller's RVE order. Each RVE's result
is taken from the one rank that solved it, so the gathered values are
bit-identical to a solve of the same RVEs on one GPU with the same
configuration. torch.distributed is only the transport here.
"""
from __future__ import annotations

import numpy as np

from . import Batch, shard_plan

_FIELDS = 11  # sigma (9), iterations, status


def _gpu_solve(nets, F, damping, **opts):
    if not nets:
        return np.zeros((0, 3, 3)), np.zeros(0, np.int64), np.zeros(0, np.int32)
    with Batch(nets, damping=damping) as b:
        b.solve(F, **opts)
        out = b.stress()
    status = {"OK": 0, "MAXITER": 1, "NAN": 2, "PENDING": 3}
    return out["sigma"], out["iters"], np.array([status[s] for s in out["status"]], np.int32)


def solve_sharded(nets, F, damping, group=None, solve_fn=None, iters_hint=None, device=None,
                  **opts):
    """Solve a batch over the ranks of ``group``.

    ``solve_fn(nets, F, damping, **opts) -> (sigma (k,3,3), iters (k,), status (k,))``
    solves one rank's share; by default a Batch on the current CUDA device.
    ``device`` holds the all-gather buffers ("cuda" for NCCL, "cpu" for gloo;
    default: cuda when the backend is NCCL). Returns (sigma (P,3,3), iters (P,),
    status (P,), rank_of (P,)) on every rank.
    """
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    P = len(nets)
    F = np.asarray(F, np.float64).reshape(P, 3, 3)
    damping = np.asarray(damping, np.float64)
    rank_of, _ = shard_plan([n.X.shape[0] for n in nets], world, iters_hint)
    mine = np.nonzero(rank_of == rank)[0]
    sig, it, st = (solve_fn or _gpu_solve)([nets[i] for i in mine], F[mine], damping[mine], **opts)
    if device is None:
        device = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    buf = np.zeros((P, _FIELDS))
    buf[mine, :9] = np.asarray(sig).reshape(len(mine), 9)
    buf[mine, 9] = np.asarray(it, np.float64)   # exact below 2^53
    buf[mine, 10] = np.asarray(st, np.float64)
    local = torch.from_numpy(buf).to(device)
    parts = [torch.empty_like(local) for _ in range(world)]
    dist.all_gather(parts, local, group=group)
    got = np.stack([p.cpu().numpy() for p in parts])  # (world, P, fields)
    rows = got[rank_of, np.arange(P)]
    return (rows[:, :9].reshape(P, 3, 3), rows[:, 9].astype(np.int64), rows[:, 10].astype(np.int32),
            rank_of)
