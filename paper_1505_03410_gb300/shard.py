"""Batches of independent Lasso problems over several GPUs, one process per GPU.

Every rank solves a contiguous share of the problems with ``lasso_batch`` on
its own device; afterwards the host gathers the outputs on one rank.  The
problems share nothing while they are solved (each one is its own path over
the common design), so the data path has no collective: the only exchange is
the gather of finished results.  Launch one process per GPU (torchrun), make
each rank's GPU its current device (``torch.cuda.set_device``; NCCL's object
gather needs it) and initialise ``torch.distributed`` (NCCL or gloo) before
calling.
"""
from __future__ import annotations

import numpy as np

from .lassogs import STATS_DTYPE, solve_batch


def problem_range(B: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous share [start, stop) of B problems for one of `world` ranks;
    the shares cover every problem once and differ in size by at most one."""
    if world < 1 or not 0 <= rank < world or B < 0:
        raise ValueError(f"need B >= 0 and 0 <= rank < world (B={B}, world={world}, rank={rank})")
    return (B * rank) // world, (B * (rank + 1)) // world


def _world(group):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist.get_world_size(group), dist.get_rank(group)
    return 1, 0


def _sparse_block(beta):
    """The nonzeros of a (B_r, T, p) coefficient block: flat indices (int64)
    into the block and their values; a Lasso solution has at most n nonzeros
    per lambda, so this is far smaller than the dense block."""
    flat = beta.reshape(-1)
    idx = np.flatnonzero(flat)
    return idx.astype(np.int64), flat[idx]


def solve_batch_sharded(XT, Y, ratios, n=None, row_mask=None, beta0=None, opts=None, group=None, dst=0,
                        solver=None, beta_format="sparse"):
    """Solve the B problems of (Y, row_mask, beta0) -- the layouts of
    ``solve_batch`` -- split over the ranks of `group`, each rank on its own
    GPU.  Returns, on rank `dst`, host arrays for the whole batch: beta, mask
    (B, T, words) uint32 and stats, a structured array (B, T) of
    ``STATS_DTYPE``; on the other ranks, None.

    beta_format: "sparse" (default) gathers only the nonzero coefficients and
    returns beta as a scipy.sparse CSR matrix of shape (B * T, p), row
    b * T + t holding problem b's solution at lambda_t; "dense" gathers the
    full (B, T, p) float64 array (B * T * p * 8 bytes through host memory:
    about 25 GB for 1024 problems, 30 lambdas and 100000 features).
    `solver` replaces ``solve_batch`` (same signature and outputs), e.g. to
    add options."""
    if beta_format not in ("sparse", "dense"):
        raise ValueError(f"beta_format must be 'sparse' or 'dense', not {beta_format!r}")
    import torch.distributed as dist
    solver = solver or solve_batch
    world, rank = _world(group)
    B = int(Y.shape[0])
    T = int(ratios.shape[0])
    p = int(XT.shape[0])
    words = (p + 31) // 32
    a, b = problem_range(B, world, rank)
    if b > a:
        out = solver(XT, Y[a:b].contiguous(), ratios, n=n,
                     row_mask=row_mask[a:b].contiguous() if row_mask is not None else None,
                     beta0=beta0[a:b].contiguous() if beta0 is not None else None, opts=opts)
        beta_np = out["beta"].cpu().numpy()
        local = (a, _sparse_block(beta_np) if beta_format == "sparse" else beta_np,
                 out["mask"].cpu().numpy().view(np.uint32) if out.get("mask") is not None else None,
                 out["stats"].cpu().numpy().view(STATS_DTYPE).reshape(b - a, T))
    else:
        empty = np.empty((0, T, p))
        local = (a, _sparse_block(empty) if beta_format == "sparse" else empty,
                 np.empty((0, T, words), dtype=np.uint32), np.empty((0, T), dtype=STATS_DTYPE))
    if world == 1:
        parts = [local]
    else:
        parts = [None] * world if rank == dst else None
        dist.gather_object(local, parts, dst=dst, group=group)
        if rank != dst:
            return None
    parts.sort(key=lambda t: t[0])
    stats = np.concatenate([t[3] for t in parts], axis=0)
    mask = None
    if all(t[2] is not None for t in parts):
        mask = np.concatenate([t[2] for t in parts], axis=0)
    assert stats.shape[0] == B
    if beta_format == "dense":
        beta = np.concatenate([t[1] for t in parts], axis=0)
        assert beta.shape[0] == B
    else:
        import scipy.sparse as sp
        # a rank's flat index (b_local * T + t) * p + j, shifted by its first problem
        idx = np.concatenate([t[1][0] + t[0] * T * p for t in parts])
        val = np.concatenate([t[1][1] for t in parts])
        beta = sp.csr_matrix((val, (idx // p, idx % p)), shape=(B * T, p))
    return dict(beta=beta, mask=mask, stats=stats)
