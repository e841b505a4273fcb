"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these compares the oracle with itself: each checks a closed form, a
theorem, an identity or an independent exact solver (brute-force
enumeration).  Mistakes planted in a copy of the oracle must make at least
one of them fail (test_oracle_mutations.py).
"""
import numpy as np
import pytest

import gen
from oracle.bruteforce import lasso_bruteforce, primal


def _dense(prob):
    return prob["XT"][:, :prob["n"]].T.astype(np.float64)


def _problem(seed, n, p, k=3, noise=0.1, correlated=False):
    return gen.small_problem(seed, n, p, dtype=np.float64, k=k, noise=noise, correlated=correlated)


# ---------------------------------------------------------------- grid, lambda_max
def test_grid_is_geometric(orc):
    """Sec. 3.3: lambda_t = lambda_max 10^(-delta t/(T-1))."""
    r = orc.lambda_ratios(100, 3.0)
    assert r[0] == 1.0
    assert abs(r[-1] - 1e-3) <= 1e-18
    q = r[1:] / r[:-1]
    np.testing.assert_allclose(q, 10 ** (-3.0 / 99), rtol=1e-13)
    assert np.all(np.diff(r) < 0)
    assert orc.lambda_ratios(1, 3.0).tolist() == [1.0]


def test_lambda_max_and_zero_solution(orc):
    """Sec. 1.2: lambda_max = ||X^T y||_inf and beta = 0 is optimal for
    lambda >= lambda_max; at lambda_max the gap of (0, y/lambda_max) is 0."""
    prob = _problem(1, 30, 50)
    X, y = _dense(prob), prob["y"]
    pre = orc.precompute(X, y)
    assert pre["lambda_max"] == pytest.approx(np.abs(X.T @ y).max(), rel=1e-14)
    out = orc.lasso_path(X, y, [1.0], gap_tol_rel=1e-12)
    assert np.all(out["beta"][0] == 0.0)
    assert out["stats"]["epochs"][0] == 0
    assert abs(out["stats"]["gap"][0]) <= 1e-14 * pre["ynorm2"]
    # only the argmax feature survives the test at lambda_max (r ~ 0)
    kept = orc.unpack_mask(out["mask"][0], 50)
    assert kept.sum() == 1 and kept[pre["argmax"]]
    # above lambda_max, beta = 0 is optimal and theta_hat = y/lambda is
    # feasible, so the gap of (0, theta) is 0 and nothing is kept
    for mult in (1.5, 3.0):
        res = orc.check(X, y, np.zeros(50), y, mult * pre["lambda_max"])
        assert abs(res["gap"]) <= 1e-14 * pre["ynorm2"]
        assert res["alpha"] == pytest.approx(1.0 / (mult * pre["lambda_max"]), rel=1e-15)
        assert res["n_kept"] == 0


def test_first_feature_enters_linearly(orc):
    """Just below lambda_max only j* = argmax |x_j^T y| is active and
    beta_j* = sign(x_j*^T y) (lambda_max - lambda) / ||x_j*||^2 (KKT, Eq. (4))."""
    prob = _problem(2, 40, 60)
    X, y = _dense(prob), prob["y"]
    c0 = X.T @ y
    js = int(np.argmax(np.abs(c0)))
    lmax = abs(c0[js])
    ratio = 1.0 - 1e-4
    out = orc.lasso_path(X, y, [1.0, ratio], gap_tol_rel=1e-15)
    b = out["beta"][1]
    expect = np.zeros(60)
    expect[js] = np.sign(c0[js]) * (lmax - lmax * ratio) / (X[:, js] @ X[:, js])
    np.testing.assert_allclose(b, expect, atol=1e-12 * lmax)


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("seed", [3, 4])
def test_orthonormal_soft_threshold(orc, seed):
    """Orthonormal design: the Lasso solution is ST(lambda, X^T y) coordinate-
    wise (Eq. (4) decouples), and cyclic CD reaches it in one pass."""
    rng = np.random.default_rng(seed)
    n, p = 40, 16
    Q, _ = np.linalg.qr(rng.standard_normal((n, p)))
    y = rng.standard_normal(n) * 3
    c = Q.T @ y
    lmax = np.abs(c).max()
    ratios = orc.lambda_ratios(12, 2.0)
    out = orc.lasso_path(Q, y, ratios, gap_tol_rel=1e-14)
    for t, r in enumerate(ratios):
        lam = lmax * r
        expect = np.sign(c) * np.maximum(np.abs(c) - lam, 0.0)
        np.testing.assert_allclose(out["beta"][t], expect, atol=1e-12 * lmax)
        assert out["stats"]["converged"][t] == 1


def test_hand_example_identity_design(orc):
    """X = I_2, y = (3, -1), lambda = 2: beta = ST(2, y) = (1, 0),
    P = 1/2 ||(1,0)-(3,-1)||^2 + 2*1 = 4.5, theta = (y - X beta)/lambda =
    (1, -1/2), D = 1/2*10 - 1/2 ||2 theta - y||^2 = 4.5 (Eq. (1)-(3))."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")
    cases = json.load(open(path))["cases"]
    for case in cases:
        X = np.array(case["X"], dtype=np.float64)
        y = np.array(case["y"], dtype=np.float64)
        lmax = np.abs(X.T @ y).max()
        ratio = case["lambda"] / lmax
        out = orc.lasso_path(X, y, [1.0, ratio], gap_tol_rel=1e-15)
        np.testing.assert_allclose(out["beta"][1], case["beta"], atol=1e-12)
        assert out["stats"]["primal"][1] == pytest.approx(case["primal"], rel=1e-12)
        assert out["stats"]["dual"][1] == pytest.approx(case["dual"], rel=1e-12)


# ---------------------------------------------------------------- exact solver
@pytest.mark.parametrize("seed,n,p", [(5, 20, 8), (6, 12, 10), (7, 6, 9)])
def test_bruteforce_agreement(orc, seed, n, p):
    """Support-and-sign enumeration gives the exact optimum; the oracle's
    tight solution must match its objective, support and coefficients."""
    prob = _problem(seed, n, p, k=3, noise=0.3)
    X, y = _dense(prob), prob["y"]
    ratios = orc.lambda_ratios(8, 1.5)
    out = orc.lasso_path(X, y, ratios, gap_tol_rel=1e-15, max_epochs=200000)
    lmax = out["lambda_max"]
    for t in range(1, len(ratios)):
        lam = lmax * ratios[t]
        bb, Pb = lasso_bruteforce(X, y, lam)
        b = out["beta"][t]
        assert primal(X, y, b, lam) == pytest.approx(Pb, rel=1e-9)
        assert out["stats"]["primal"][t] == pytest.approx(Pb, rel=1e-9)
        np.testing.assert_array_equal(b != 0, bb != 0)
        np.testing.assert_allclose(b, bb, atol=1e-6)


# ---------------------------------------------------------------- KKT, safety
def test_kkt_at_tight_solution(orc):
    """Eq. (3)-(4): theta = (y - X beta)/lambda has |x_j^T theta| <= 1 and
    x_j^T theta = sign(beta_j) on the support."""
    prob = _problem(8, 50, 200, k=5)
    X, y = _dense(prob), prob["y"]
    ratios = orc.lambda_ratios(10, 2.0)
    out = orc.lasso_path(X, y, ratios, gap_tol_rel=1e-14)
    for t in range(1, 10):
        lam = out["stats"]["lambda"][t]
        b = out["beta"][t]
        theta = (y - X @ b) / lam
        corr = X.T @ theta
        g = np.sqrt(2 * max(out["stats"]["gap"][t], 0) + 1e-30) / lam
        assert np.all(np.abs(corr) <= 1 + 10 * g + 1e-9)
        sup = b != 0
        np.testing.assert_allclose(corr[sup], np.sign(b[sup]), atol=10 * g + 1e-9)


def test_every_sphere_contains_dual_optimum(orc):
    """Thm. 2 + Prop. 1: at every check, theta_hat lies in B(theta_k, r_k)
    with r_k = sqrt(2 G)/lambda; theta_hat from the exact brute-force beta."""
    prob = _problem(9, 15, 10, k=3, noise=0.2)
    X, y = _dense(prob), prob["y"]
    ratios = orc.lambda_ratios(6, 1.5)
    out = orc.lasso_path(X, y, ratios, gap_tol_rel=1e-13, log_checks=5000, screen_period=2)
    lmax = out["lambda_max"]
    thetas = {}
    for t in range(len(ratios)):
        lam = lmax * ratios[t]
        bb, _ = lasso_bruteforce(X, y, lam)
        thetas[t] = (y - X @ bb) / lam
    log = out["log"]
    assert len(log["t"]) > 10
    for k in range(len(log["t"])):
        t = int(log["t"][k])
        center = log["alpha"][k] * log["rho"][k]
        d = np.linalg.norm(center - thetas[t])
        assert d <= log["radius"][k] * (1 + 1e-9) + 1e-12, (k, t, d, log["radius"][k])


def test_refined_radius_of_thm2(orc):
    """Thm. 2 + Prop. 1 (refined_radius = 1): theta_hat lies in
    B(theta, (R^2 - r(beta)^2)^(1/2)) with R = ||theta - y/lambda|| and
    r(beta) = (||y||^2 - ||X beta - y||^2 - 2 lambda ||beta||_1)_+^(1/2) / lambda,
    and that radius is at most sqrt(2 G)/lambda.  Runs from a poor start
    (P(beta0) > P(0) at every lambda, warm starts off) so that the clipped
    r(beta) = 0 case occurs and the radius is strictly smaller there; the
    path still reaches the exact brute-force solution."""
    prob = _problem(21, 15, 10, k=3, noise=0.2)
    X, y = _dense(prob), prob["y"]
    rng = np.random.default_rng(21)
    beta0 = 3.0 * rng.standard_normal(10)
    ratios = orc.lambda_ratios(5, 1.5)[1:]
    out = orc.lasso_path(X, y, ratios, beta0=beta0, warm_start=False, gap_tol_rel=1e-13,
                         log_checks=5000, screen_period=1, refined_radius=1)
    lmax = out["lambda_max"]
    sols = {t: lasso_bruteforce(X, y, lmax * ratios[t])[0] for t in range(len(ratios))}
    log = out["log"]
    strict = 0
    for k in range(len(log["t"])):
        t = int(log["t"][k])
        lam = lmax * ratios[t]
        theta = log["alpha"][k] * log["rho"][k]
        R2 = np.sum((theta - y / lam) ** 2)
        D = 0.5 * y @ y - 0.5 * lam ** 2 * R2             # Eq. (2)
        P = log["gap"][k] + D
        r2 = max(0.0, y @ y - 2 * P) / lam ** 2           # r(beta)^2, clipped
        thm2 = np.sqrt(max(R2 - r2, 0.0))
        gap_r = np.sqrt(2 * max(log["gap"][k], 0.0)) / lam
        # equal up to the rounding inflation of the gap (far below 1e-12 ||y||^2)
        assert abs(log["radius"][k] ** 2 - thm2 ** 2) <= 1e-7 * thm2 ** 2 + 1e-12 * (y @ y) / lam ** 2, \
            (k, log["radius"][k], thm2)
        assert log["radius"][k] ** 2 <= gap_r ** 2 * (1 + 1e-9) + 1e-12 * (y @ y) / lam ** 2
        theta_hat = (y - X @ sols[t]) / lam
        assert np.linalg.norm(theta - theta_hat) <= log["radius"][k] * (1 + 1e-9) + 1e-12
        strict += log["radius"][k] < 0.99 * gap_r
    assert strict > 0
    for t in range(len(ratios)):
        np.testing.assert_allclose(out["beta"][t], sols[t], atol=1e-6)


def test_screened_features_are_zero(orc):
    """Eq. (5): a feature the test screens has beta_hat_j = 0 -- checked
    against the exact brute-force solution and the tight CD output."""
    prob = _problem(10, 16, 11, k=3, noise=0.2)
    X, y = _dense(prob), prob["y"]
    ratios = orc.lambda_ratios(7, 1.5)
    out = orc.lasso_path(X, y, ratios, gap_tol_rel=1e-14)
    lmax = out["lambda_max"]
    n_screened = 0
    for t in range(len(ratios)):
        kept = orc.unpack_mask(out["mask"][t], 11)
        bb, _ = lasso_bruteforce(X, y, lmax * ratios[t])
        assert np.all(bb[~kept] == 0)
        assert np.all(out["beta"][t][~kept] == 0)
        n_screened += (~kept).sum()
    assert n_screened > 0


def test_finite_identification(orc):
    """Thm. 1: on a tight solve the final safe-active set equals the
    equicorrelation set {j : |x_j^T theta_hat| = 1}."""
    prob = _problem(11, 60, 300, k=6, noise=0.05)
    X, y = _dense(prob), prob["y"]
    ratios = orc.lambda_ratios(8, 1.0)
    out = orc.lasso_path(X, y, ratios, gap_tol_rel=1e-15)
    for t in range(1, 8):
        lam = out["stats"]["lambda"][t]
        theta = (y - X @ out["beta"][t]) / lam
        eq = np.abs(X.T @ theta) >= 1 - 1e-7
        kept = orc.unpack_mask(out["mask"][t], 300)
        np.testing.assert_array_equal(kept, eq)


def test_prop3_sequential_identity(orc):
    """Prop. 3: for any (beta, theta) with theta feasible,
    2G_t/l_t^2 = (1 - l_t/l_{t-1}) ||(X beta - y)/l_t||^2
                 - (l_{t-1}/l_t - 1) ||theta||^2 + 2 G_{t-1} / (l_{t-1} l_t)."""
    rng = np.random.default_rng(12)
    prob = _problem(12, 25, 40)
    X, y = _dense(prob), prob["y"]
    beta = np.zeros(40)
    beta[rng.choice(40, 4, replace=False)] = 0.1 * rng.standard_normal(4)
    rho = y - X @ beta
    m = np.abs(X.T @ rho).max()
    l1, l0 = 0.3 * m, 0.5 * m  # both below m: theta = rho/m at both
    c0 = orc.check(X, y, beta, rho, l0)
    c1 = orc.check(X, y, beta, rho, l1)
    assert c0["alpha"] == c1["alpha"] == pytest.approx(1 / m, rel=1e-15)
    theta = c1["alpha"] * rho
    lhs = 2 * c1["gap"] / l1 ** 2
    rhs = ((1 - l1 / l0) * np.sum((rho / l1) ** 2) - (l0 / l1 - 1) * np.sum(theta ** 2)
           + 2 * c0["gap"] / (l0 * l1))
    assert lhs == pytest.approx(rhs, rel=1e-10)
    # the objectives themselves, written from Eq. (1) and Eq. (2)
    assert c1["primal"] == pytest.approx(0.5 * rho @ rho + l1 * np.abs(beta).sum(), rel=1e-13)
    assert c1["dual"] == pytest.approx(0.5 * y @ y - 0.5 * l1 ** 2 * np.sum((theta - y / l1) ** 2),
                                       rel=1e-12)


def test_dual_point_eq8_is_projection_on_span(orc):
    """Eq. (8): theta_k = alpha rho is the point of span(rho) in the dual
    feasible set closest to y/lambda (clipped 1-D projection)."""
    prob = _problem(13, 30, 50)
    X, y = _dense(prob), prob["y"]
    rng = np.random.default_rng(13)
    beta = 0.05 * rng.standard_normal(50)
    # the check takes (beta, rho) as given; the second residual points away
    # from y so that the clip at -1/||X^T rho||_inf is exercised
    for rho in (y - X @ beta, -0.7 * y + 0.1 * rng.standard_normal(30)):
        m = np.abs(X.T @ rho).max()
        for lam in (0.2 * m, 0.9 * m, 2.0 * m):
            res = orc.check(X, y, beta, rho, lam, dual_point=1)
            grid = np.linspace(-1 / m, 1 / m, 20001)
            d = [np.sum((a * rho - y / lam) ** 2) for a in grid]
            a_best = grid[int(np.argmin(d))]
            assert abs(res["alpha"] - a_best) <= 2 * (2 / m) / 20000
            assert np.abs(X.T @ (res["alpha"] * rho)).max() <= 1 + 1e-12


def test_gap_bounds_suboptimality(orc):
    """Sec. 3.2: G(beta, theta) <= eps implies P(beta) - P* <= eps."""
    prob = _problem(14, 14, 9, k=2, noise=0.3)
    X, y = _dense(prob), prob["y"]
    ratios = orc.lambda_ratios(5, 1.0)
    out = orc.lasso_path(X, y, ratios, gap_tol_rel=1e-3)
    lmax = out["lambda_max"]
    for t in range(len(ratios)):
        lam = lmax * ratios[t]
        _, Pstar = lasso_bruteforce(X, y, lam)
        Pb = primal(X, y, out["beta"][t], lam)
        assert Pb - Pstar <= out["stats"]["gap"][t] * (1 + 1e-9) + 1e-14
        assert out["stats"]["gap"][t] <= 1e-3 * out["ynorm2"]


def test_screening_never_changes_the_answer(orc):
    """Screening is safe: the path with checks every pass and the path with
    checks every 10 passes reach the same solutions (tight tolerance)."""
    prob = _problem(15, 40, 120, k=4)
    X, y = _dense(prob), prob["y"]
    ratios = orc.lambda_ratios(10, 2.0)
    a = orc.lasso_path(X, y, ratios, gap_tol_rel=1e-14, screen_period=1)
    b = orc.lasso_path(X, y, ratios, gap_tol_rel=1e-14, screen_period=10)
    np.testing.assert_allclose(a["beta"], b["beta"], atol=1e-6)
    np.testing.assert_array_equal(a["beta"] != 0, b["beta"] != 0)


def test_not_converged_status(orc):
    """The pass cap K of Algorithm 1: too small a K reports non-convergence."""
    prob = _problem(16, 40, 200, k=8)
    X, y = _dense(prob), prob["y"]
    out = orc.lasso_path(X, y, orc.lambda_ratios(5, 3.0), gap_tol_rel=1e-12, max_epochs=2)
    assert out["status"] == 5
    assert out["stats"]["converged"][-1] == 0
    assert np.all(out["stats"]["epochs"] <= 2)


def test_batch_equals_independent_paths(orc):
    """Row-subsampled problems: each batched solve equals the plain path on
    the gathered rows."""
    prob = _problem(17, 30, 40)
    X, y = _dense(prob), prob["y"]
    rng = np.random.default_rng(17)
    B = 3
    rm = (rng.random((B, 30)) < 0.7).astype(np.uint8)
    Y = np.stack([y * rm[b] for b in range(B)])
    ratios = orc.lambda_ratios(6, 1.5)
    out = orc.lasso_batch(X, Y, ratios, row_mask=rm, gap_tol_rel=1e-10)
    for b in range(B):
        rows = rm[b] != 0
        ref = orc.lasso_path(X[rows], y[rows], ratios, gap_tol_rel=1e-10)
        np.testing.assert_array_equal(out["beta"][b], ref["beta"])


def test_bad_warm_start_reaches_optimum(orc):
    """Remark 3: screening a feature whose coefficient is nonzero sets it to
    zero (with the residual updated); from a start where every coefficient
    is wrong and nonzero, the path still reaches the exact optimum."""
    prob = _problem(18, 14, 9, k=2, noise=0.2)
    X, y = _dense(prob), prob["y"]
    rng = np.random.default_rng(18)
    beta0 = rng.standard_normal(9)
    ratios = orc.lambda_ratios(4, 1.0)
    out = orc.lasso_path(X, y, ratios, beta0=beta0, gap_tol_rel=1e-14, screen_period=1)
    lmax = out["lambda_max"]
    for t in range(len(ratios)):
        bb, Pb = lasso_bruteforce(X, y, lmax * ratios[t])
        assert primal(X, y, out["beta"][t], lmax * ratios[t]) == pytest.approx(Pb, rel=1e-9)
        np.testing.assert_allclose(out["beta"][t], bb, atol=1e-6)


def test_screening_a_nonzero_coefficient(orc):
    """Remark 3 with the screening step exercised: start at the exact optimum
    plus a small coefficient on a clearly inactive feature.  The first check
    screens that feature while its coefficient is nonzero; removing it (and
    its contribution to the residual) must return the exact optimum."""
    prob = _problem(19, 20, 10, k=2, noise=0.2)
    X, y = _dense(prob), prob["y"]
    lmax = np.abs(X.T @ y).max()
    lam = 0.5 * lmax
    bb, Pb = lasso_bruteforce(X, y, lam)
    corr = np.abs(X.T @ (y - X @ bb)) / lam
    k = int(np.argmin(corr))
    assert corr[k] < 0.6 and bb[k] == 0
    beta0 = bb.copy()
    beta0[k] = 1e-3
    out = orc.lasso_path(X, y, [0.5], beta0=beta0, gap_tol_rel=1e-14)
    assert not orc.unpack_mask(out["mask"][0], 10)[k]
    np.testing.assert_allclose(out["beta"][0], bb, atol=1e-9)
    assert out["stats"]["primal"][0] == pytest.approx(Pb, rel=1e-12)


def test_gap_rounding_bound_holds(orc):
    """R7: the FP64 gap the check computes differs from the exact gap of the
    same (beta, rho, alpha) -- evaluated in rational arithmetic -- by at most
    the inflation tau the radius adds.  The cases include a nearly converged
    iterate, where the gap is far below its terms."""
    from fractions import Fraction as F
    prob = _problem(22, 20, 12, k=3, noise=0.2)
    X, y = _dense(prob), prob["y"]
    lmax = np.abs(X.T @ y).max()
    checked = 0
    for ratio in (0.6, 0.2):
        lam = ratio * lmax
        tight = orc.lasso_path(X, y, [1.0, ratio], gap_tol_rel=1e-15)["beta"][1]
        beta0 = np.zeros(12)
        for beta in (beta0, 0.5 * tight, tight):
            rho = y - X @ beta
            res = orc.check(X, y, beta, rho, lam)
            a = F(res["alpha"])
            L = F(lam)
            rr = sum(F(v) * F(v) for v in rho)
            l1 = sum(abs(F(v)) for v in beta)
            d2 = sum((L * (a * F(r)) - F(v)) ** 2 for r, v in zip(rho, y))
            yy = sum(F(v) * F(v) for v in y)
            G = (rr / 2 + L * l1) - (yy / 2 - d2 / 2)
            assert abs(F(res["gap"]) - G) <= F(res["tau"]), (float(G), res["gap"], res["tau"])
            checked += 1
    assert checked == 6
