"""Full-size runs in the benchmark's launch configuration, checked through
properties that hold at any size and are recomputed here in FP64 from the
returned coefficients alone (the oracle's path at these sizes takes minutes):

* the duality gap certifies every lambda: with rho = y - X beta and the dual
  point theta = rho / max(lambda, ||X^T rho||_inf) (Sec. 2, the rescaling the
  solver uses), P(beta) - D(theta) <= eps = 1e-6 ||y||^2 (Eq. (1), (2));
* the soft KKT conditions of Eq. (4) follow from the gap: for every j,
  |x_j^T rho| <= lambda + sqrt(2 gap) ||x_j|| (|x_j^T rho_hat| <= lambda at the
  optimum, and ||rho - rho_hat||^2 <= 2 (P(beta) - P*) <= 2 gap);
* lambda_t = lambda_max * ratio_t with lambda_max = ||X^T y||_inf (Sec. 1.2).
The comparison element by element is in test_gpu_path / test_gpu_batch on the
first lambdas of the same workloads."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1505_03410_gb300.build import build
    build()
    import paper_1505_03410_gb300 as p
    return p


def _certify(X, y, lam, beta, tol_rel, nrm):
    """FP64 recomputation of the certificate of one (problem, lambda); nrm are
    the column norms of X."""
    rho = y - X @ beta
    c = X.T @ rho
    s = max(lam, np.abs(c).max())
    theta = rho / s
    P = 0.5 * rho @ rho + lam * np.abs(beta).sum()
    D = 0.5 * y @ y - 0.5 * lam * lam * np.sum((theta - y / lam) ** 2)
    gap = P - D
    eps = tol_rel * (y @ y)
    # the solver stops at gap <= eps computed in FP64 from its own double-float
    # state; allow the rounding of two evaluations of O(||y||^2) terms
    assert gap <= eps + 1e-12 * (y @ y), (gap, eps)
    assert np.all(np.abs(c) <= lam + np.sqrt(2 * max(gap, 0.0) + 1e-12 * (y @ y)) * nrm + 1e-9 * lam)
    return gap


def test_workload2_full_path_certified(pkg):
    """Toeplitz 500 x 50000 FP32, all 100 lambdas to lambda_max/1000, as
    bench.py launches it."""
    w = gen.workload2()
    n, p, T = w["n"], w["p"], w["T"]
    ratios = pkg.lasso_lambda_grid(T, w["delta"])
    dev = torch.device("cuda:0")
    out = pkg.solve_path(torch.from_numpy(w["XT"]).to(dev), torch.from_numpy(w["y"]).to(dev),
                         torch.from_numpy(ratios).to(dev), n=n,
                         opts=pkg.lasso_default_opts(screen_period=w["f"], gap_tol_rel=w["tol"]))
    torch.cuda.synchronize()
    st = pkg.stats_to_numpy(out["stats"])
    beta = out["beta"].cpu().numpy()
    assert np.all(st["status"] == 0)
    X = w["XT"][:, :n].astype(np.float64).T
    y = w["y"]
    lmax = np.abs(X.T @ y).max()
    np.testing.assert_allclose(st["lambda"], lmax * ratios, rtol=1e-12)
    nrm = np.linalg.norm(X, axis=0)
    for t in range(T):
        gap = _certify(X, y, st["lambda"][t], beta[t], w["tol"], nrm)
        np.testing.assert_allclose(gap, st["gap"][t], rtol=1e-6, atol=1e-9 * (y @ y))
    # the same pass and check counts as the oracle on its first lambdas (it
    # runs the whole path in minutes; the first 40 are compared in full elsewhere)
    o = oracle.lasso_path(w["XT"], y, ratios[:10], n=n, screen_period=w["f"], gap_tol_rel=w["tol"])
    np.testing.assert_array_equal(st["epochs"][:10], o["stats"]["epochs"].astype(np.int64))


def test_workload3_full_batch_certified(pkg):
    """Stability selection at full size: 256 row-subset problems on the
    Gaussian 1000 x 20000 design, all 50 lambdas, in the default mode
    (lockstep tensor-core first checks, X^T rho over all p so that the dual
    point is feasible for the full problem); 16 problems spread over the
    batch are certified."""
    w = gen.workload3()
    n, p, T = w["n"], w["p"], w["T"]
    ratios = pkg.lasso_lambda_grid(T, w["delta"])
    dev = torch.device("cuda:0")
    out = pkg.solve_batch(torch.from_numpy(w["XT"]).to(dev), torch.from_numpy(w["Y"]).to(dev),
                          torch.from_numpy(ratios).to(dev), n=n,
                          row_mask=torch.from_numpy(w["row_mask"]).to(dev),
                          opts=pkg.lasso_default_opts(screen_period=w["f"], gap_tol_rel=w["tol"]))
    torch.cuda.synchronize()
    B = w["Y"].shape[0]
    st = pkg.stats_to_numpy(out["stats"]).reshape(B, T)
    assert np.all(st["status"] == 0)
    beta = out["beta"].cpu().numpy()
    X = w["XT"][:, :n].astype(np.float64).T
    for b in np.linspace(0, B - 1, 16).astype(int):
        rows = np.nonzero(w["row_mask"][b])[0]
        Xb, yb = X[rows], w["Y"][b, rows]
        lmax = np.abs(Xb.T @ yb).max()
        np.testing.assert_allclose(st["lambda"][b], lmax * ratios, rtol=1e-12)
        nrm = np.linalg.norm(Xb, axis=0)
        for t in range(T):
            _certify(Xb, yb, st["lambda"][b, t], beta[b, t], w["tol"], nrm)
