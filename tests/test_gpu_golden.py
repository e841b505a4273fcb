"""The benchmark workloads at full size, every lambda, against the FP64
oracle's stored results (tests/golden/oracle_paths.py wrote them by running
the oracle, Algorithm 1 of Sec. 4.1, on the same seeded inputs).

Per (problem, lambda) the GPU must reproduce the oracle's pass and check
counts, |A| and the number of nonzeros exactly, the support with its signs
and the safe-active mask bit for bit (compared through digests), the primal
objective to 1e-9 relative and the coefficients to 1e-5.  The inputs are
regenerated here from their seeds and must hash to the stored fingerprints
(the generators use no BLAS, so every machine gets the same bytes)."""
import os

import numpy as np
import pytest

import gen
from tests.golden.oracle_paths import digest64, fingerprint, support_digest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1505_03410_gb300.build import build
    build()
    import paper_1505_03410_gb300 as p
    return p


def _load(name):
    path = os.path.join(GOLDEN, name + ".npz")
    if not os.path.exists(path):
        pytest.fail(f"{path} is missing: run tests/golden/oracle_paths.py {name}")
    return dict(np.load(path))


def _compare(tag, beta, mask, st, gold, b=None, values=True):
    """beta (T, p), mask (T, words), st (T,) records vs the stored arrays of
    problem b (None: a single path)."""
    pick = (lambda k: gold[k]) if b is None else (lambda k: gold[k][b])
    T = beta.shape[0]
    bad = []
    conv = pick("converged").astype(bool)
    if not np.array_equal(st["status"] == 0, conv):
        bad.append(("status", np.nonzero((st["status"] == 0) != conv)[0][:5]))
    for key in ("epochs", "checks", "n_active", "n_nonzero"):
        d = np.nonzero(st[key] != pick(key))[0]
        if d.size:
            bad.append((key, d[:5], st[key][d[:5]], pick(key)[d[:5]]))
    rel = np.abs(st["primal"] - pick("primal")) / np.abs(pick("primal"))
    if np.any(rel > 1e-9):
        bad.append(("primal", np.nonzero(rel > 1e-9)[0][:5], rel.max()))
    sd = np.array([support_digest(beta[t]) for t in range(T)], dtype=np.uint64)
    d = np.nonzero(sd != pick("support_digest"))[0]
    if d.size:
        bad.append(("support", d[:5]))
    md = np.array([digest64(mask[t]) for t in range(T)], dtype=np.uint64)
    d = np.nonzero(md != pick("mask_digest"))[0]
    if d.size:
        bad.append(("mask", d[:5]))
    if values:
        sfx = "" if b is None else f"_{b}"
        ptr, idx, val = gold["sup_ptr" + sfx], gold["sup_idx" + sfx], gold["sup_val" + sfx]
        for t in range(T):
            ii = idx[ptr[t]:ptr[t + 1]]
            err = np.abs(beta[t, ii] - val[ptr[t]:ptr[t + 1]].astype(np.float64))
            if err.size and err.max() > 1e-5:
                bad.append(("beta", t, err.max()))
                break
    assert not bad, (tag, b, bad)


def _workload2(pkg, screen_rule):
    gold = _load("workload2_" + ("dome" if screen_rule else "sphere"))
    w = gen.workload2()
    assert fingerprint(w["XT"]) == str(gold["x_sha256"]), "the regenerated design differs from the stored one"
    assert fingerprint(w["y"]) == str(gold["y_sha256"]), "the regenerated responses differ from the stored ones"
    n, p = w["n"], w["p"]
    dev = torch.device("cuda:0")
    ratios = gold["ratios"]
    out = pkg.solve_path(torch.from_numpy(w["XT"]).to(dev), torch.from_numpy(w["y"]).to(dev),
                         torch.from_numpy(ratios).to(dev), n=n,
                         opts=pkg.lasso_default_opts(screen_period=w["f"], gap_tol_rel=w["tol"],
                                                     screen_rule=screen_rule))
    torch.cuda.synchronize()
    st = pkg.stats_to_numpy(out["stats"])
    _compare(f"workload2 screen_rule={screen_rule}", out["beta"].cpu().numpy(),
             out["mask"].cpu().numpy().view(np.uint32), st, gold)


def test_workload2_every_lambda(pkg):
    """Toeplitz 500 x 50000 FP32, the 100-point grid to lambda_max/1000: the
    benchmark's path, in its launch configuration."""
    _workload2(pkg, 0)


def test_workload2_dome_every_lambda(pkg):
    """The same path with the GAP SAFE dome beside the sphere (Eq. (11))."""
    _workload2(pkg, 1)


@pytest.mark.parametrize("gemm,group,per_pass", [(2, 0, 0), (1, 0, 0), (1, 32, 0), (2, 0, 1)])
def test_workload3_every_problem_every_lambda(pkg, gemm, group, per_pass):
    """The 256 row-subset problems of the stability-selection workload
    (Gaussian 1000 x 20000, 50 lambdas to lambda_max/100), batched: lockstep
    with the split-BF16 tensor-core first check (gemm 2) and per-CTA FP32
    checks (gemm 1).  Counts, objectives, supports and masks of every
    (problem, lambda); coefficients of 16 problems spread over the batch.
    With groups of 32 CTAs per problem the chain runs in Gram form; with
    per_pass = 1 the lockstep takes a product before every coordinate pass."""
    gold = _load("workload3_batch")
    w = gen.workload3()
    assert fingerprint(w["XT"]) == str(gold["x_sha256"]), "the regenerated design differs from the stored one"
    assert fingerprint(w["row_mask"]) == str(gold["row_mask_sha256"])
    assert fingerprint(w["Y"]) == str(gold["y_sha256"]), "the regenerated responses differ from the stored ones"
    n, p = w["n"], w["p"]
    Y = w["Y"]
    B, T = Y.shape[0], len(gold["ratios"])
    dev = torch.device("cuda:0")
    out = pkg.solve_batch(torch.from_numpy(w["XT"]).to(dev), torch.from_numpy(Y).to(dev),
                          torch.from_numpy(gold["ratios"]).to(dev), n=n,
                          row_mask=torch.from_numpy(w["row_mask"]).to(dev),
                          opts=pkg.lasso_default_opts(screen_period=w["f"], gap_tol_rel=w["tol"], gemm_dtype=gemm,
                                                      batch_group=group, lockstep_pass=per_pass))
    torch.cuda.synchronize()
    st = pkg.stats_to_numpy(out["stats"]).reshape(B, T)
    beta = out["beta"].cpu().numpy()
    mask = out["mask"].cpu().numpy().view(np.uint32)
    values = set(int(v) for v in gold["values_for"])
    for b in range(B):
        _compare(f"workload3 gemm={gemm} group={group} per_pass={per_pass}", beta[b], mask[b], st[b], gold, b=b, values=b in values)
