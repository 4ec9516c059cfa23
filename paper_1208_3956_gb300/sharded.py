"""Sources sharded over ranks, one process per GPU, each holding its own factors.

The solves of different sources are independent, so the data path needs no
collective.  The least-squares misfit and its gradient with respect to
m = 1/c^2 are sums over sources: each rank computes its share with the library
(forward and adjoint solves on its own factors) and one all-reduce of
1 + n_x n_y (n_z) FP64 values sums them over the ranks.

    lo, hi = shard(nsrc, rank, world)
    J, grad = gradient_over_ranks(solver, src_idx, rec_idx, d, tol)
"""
from __future__ import annotations

import numpy as np


def shard(n: int, rank: int, world: int) -> tuple:
    """Contiguous, balanced share [lo, hi) of n items for this rank (the first n % world
    ranks take one more)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    base, rem = divmod(int(n), world)
    lo = rank * base + min(rank, rem)
    return lo, lo + base + (1 if rank < rem else 0)


def gradient_over_ranks(solver, src_idx, rec_idx, d, tol=1e-6, group=None):
    """(misfit, dJ/dm on the interior grid) summed over the sources of all ranks.

    solver: this rank's factored HelmDD (or anything with .n and .gradient(src, rec, d, tol)).
    src_idx / d: every source and its receiver data ([nsrc][nrec]); this rank takes its
    shard.  Without an initialised process group the call is the single-process gradient.
    """
    import torch
    import torch.distributed as dist

    src_idx = np.asarray(src_idx, dtype=np.int64)
    d = np.asarray(d, dtype=np.complex128)
    if d.shape != (src_idx.size, np.asarray(rec_idx).size):
        raise ValueError("d must have shape (nsrc, nrec)")
    dist_on = dist.is_available() and dist.is_initialized()
    world = dist.get_world_size(group) if dist_on else 1
    rank = dist.get_rank(group) if dist_on else 0
    lo, hi = shard(src_idx.size, rank, world)
    shape = tuple(reversed(tuple(solver.n)))
    if hi > lo:
        J, g = solver.gradient(src_idx[lo:hi], rec_idx, d[lo:hi], tol)
        g = np.asarray(g, dtype=np.float64).reshape(shape)
    else:
        J, g = 0.0, np.zeros(shape)
    if world == 1:
        return float(J), g
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    buf = torch.as_tensor(np.concatenate([[J], g.ravel()]), dtype=torch.float64, device=dev)
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    out = buf.cpu().numpy()
    return float(out[0]), out[1:].reshape(shape)
