"""Batches of independent problems over several ranks (one GPU each): the
problem split and the host-side gather, on the CPU with two gloo ranks and a
stand-in for the GPU solver (the solver itself is covered by the GPU tests)."""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1505_03410_gb300.lassogs import STATS_DTYPE  # noqa: E402
from paper_1505_03410_gb300.shard import problem_range, solve_batch_sharded  # noqa: E402


@pytest.mark.parametrize("B", [0, 1, 7, 8, 256, 1023])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_problem_range_covers_every_problem_once(B, world):
    ranges = [problem_range(B, world, r) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == B
    for (a0, b0), (a1, b1) in zip(ranges, ranges[1:]):
        assert b0 == a1
    sizes = [b - a for a, b in ranges]
    assert max(sizes) - min(sizes) <= 1


def test_problem_range_rejects_bad_ranks():
    with pytest.raises(ValueError):
        problem_range(10, 2, 2)
    with pytest.raises(ValueError):
        problem_range(10, 0, 0)


def fake_solver(XT, Y, ratios, n=None, row_mask=None, beta0=None, opts=None):
    """Stand-in for solve_batch with the same output layout: problem b's
    coefficients are Y[b, 0] + t + j / 1000, its records carry lambda = Y[b, 0]
    and status = the count of rows in its mask."""
    B, T, p = Y.shape[0], ratios.shape[0], XT.shape[0]
    y0 = Y[:, 0].double().numpy()
    beta = y0[:, None, None] + np.arange(T)[None, :, None] + np.arange(p)[None, None, :] / 1000.0
    st = np.zeros((B, T), dtype=STATS_DTYPE)
    st["lambda"] = y0[:, None]
    st["status"] = (row_mask.numpy().sum(axis=1) if row_mask is not None else np.zeros(B))[:, None]
    mask = np.full((B, T, (p + 31) // 32), 7, dtype=np.uint32)
    return dict(beta=torch.from_numpy(beta), mask=torch.from_numpy(mask.view(np.int32)),
                stats=torch.from_numpy(st.view(np.uint8).reshape(-1).copy()))


def _inputs(B=7, n=5, p=40, T=3):
    XT = torch.zeros((p, 8), dtype=torch.float32)
    Y = torch.arange(B * n, dtype=torch.float64).reshape(B, n)
    rm = torch.from_numpy((np.arange(B)[:, None] > np.arange(n)[None, :]).astype(np.uint8))
    ratios = torch.ones(T, dtype=torch.float64)
    return XT, Y, rm, ratios


def _check_full(out, B=7, n=5, p=40, T=3):
    XT, Y, rm, ratios = _inputs(B, n, p, T)
    ref = fake_solver(XT, Y, ratios, row_mask=rm)
    beta = out["beta"]
    if not isinstance(beta, np.ndarray):  # the sparse gather: rows b * T + t
        assert beta.shape == (B * T, p)
        beta = beta.toarray().reshape(B, T, p)
    np.testing.assert_array_equal(beta, ref["beta"].numpy())
    np.testing.assert_array_equal(out["stats"]["lambda"], Y[:, 0].numpy()[:, None].repeat(T, 1))
    np.testing.assert_array_equal(out["stats"]["status"], rm.numpy().sum(axis=1)[:, None].repeat(T, 1))
    assert out["mask"].shape == (B, T, 2) and np.all(out["mask"] == 7)


@pytest.mark.parametrize("fmt", ["sparse", "dense"])
def test_single_process_is_the_whole_batch(fmt):
    XT, Y, rm, ratios = _inputs()
    out = solve_batch_sharded(XT, Y, ratios, row_mask=rm, solver=fake_solver, beta_format=fmt)
    assert isinstance(out["beta"], np.ndarray) == (fmt == "dense")
    _check_full(out)


def test_sparse_gather_keeps_zeros_out():
    """The sparse form holds exactly the nonzero coefficients."""
    XT, Y, rm, ratios = _inputs(B=3, p=40, T=2)

    def solver(*args, **kw):
        out = fake_solver(*args, **kw)
        beta = out["beta"].numpy().copy()
        beta[:, :, ::3] = 0.0
        return dict(out, beta=torch.from_numpy(beta))
    out = solve_batch_sharded(XT, Y, ratios, row_mask=rm, solver=solver)
    dense = solver(XT, Y, ratios, row_mask=rm)["beta"].numpy()
    assert out["beta"].nnz == int(np.count_nonzero(dense))
    np.testing.assert_array_equal(out["beta"].toarray().reshape(dense.shape), dense)


def test_bad_beta_format_is_rejected():
    XT, Y, rm, ratios = _inputs()
    with pytest.raises(ValueError):
        solve_batch_sharded(XT, Y, ratios, solver=fake_solver, beta_format="csr")


def _worker(rank, world, port, q, B, fmt="sparse"):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1505_03410_gb300.shard import solve_batch_sharded as sbs
        XT, Y, rm, ratios = _inputs(B=B)
        out = sbs(XT, Y, ratios, row_mask=rm, solver=fake_solver, beta_format=fmt)
        q.put((rank, None if out is None else (out["beta"], out["stats"], out["mask"])))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("B,fmt", [(7, "sparse"), (1, "sparse"), (7, "dense")])
def test_two_gloo_ranks_gather_the_whole_batch(B, fmt):
    """Rank 0 ends with every problem's outputs in order; rank 1 with None.
    With B = 1 the second rank has no problem and still takes part."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29631 + B + (8 if fmt == "dense" else 0)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q, B, fmt)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for pr in procs:
        pr.join(60)
        assert pr.exitcode == 0
    assert res[1] is None
    beta, stats, mask = res[0]
    _check_full(dict(beta=beta, stats=stats, mask=mask), B=B)
