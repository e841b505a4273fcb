"""Pins of the oracle's Elastic-Net (the paper's appendix: the Elastic-Net as
a Lasso on the augmented design [X; sqrt((1 - a) lambda) I], response [y; 0]
and penalty a lambda).

Each pin checks the Elastic-Net itself, not the reduction the oracle uses:
its closed form on an orthonormal design, its KKT conditions, lambda_max, the
first feature's entry, and the exact solution from support enumeration on
the augmented design.
"""
import numpy as np
import pytest

import gen
from oracle.bruteforce import lasso_bruteforce


def _dense(prob):
    return prob["XT"][:, :prob["n"]].T.astype(np.float64)


def enet_primal(X, y, b, lam, a):
    """1/2 ||X b - y||^2 + lam a ||b||_1 + lam (1 - a)/2 ||b||^2."""
    r = X @ b - y
    return 0.5 * r @ r + lam * a * np.abs(b).sum() + 0.5 * lam * (1 - a) * b @ b


@pytest.mark.parametrize("a", [0.3, 0.75])
def test_enet_orthonormal_closed_form(orc, a):
    """Orthonormal X: the problem decouples and beta_j = ST(a lam, x_j^T y) /
    (1 + (1 - a) lam); beta = 0 from lambda_max = ||X^T y||_inf / a on."""
    rng = np.random.default_rng(int(100 * a))
    n, p = 40, 16
    Q, _ = np.linalg.qr(rng.standard_normal((n, p)))
    y = rng.standard_normal(n) * 3
    c = Q.T @ y
    lmax = np.abs(c).max() / a
    ratios = orc.lambda_ratios(10, 2.0)
    out = orc.lasso_path(Q, y, ratios, gap_tol_rel=1e-14, enet_alpha=a)
    assert out["lambda_max"] == pytest.approx(lmax, rel=1e-14)
    for t, r in enumerate(ratios):
        lam = lmax * r
        expect = np.sign(c) * np.maximum(np.abs(c) - a * lam, 0.0) / (1 + (1 - a) * lam)
        np.testing.assert_allclose(out["beta"][t], expect, atol=1e-11 * np.abs(c).max())
        assert out["stats"]["lambda"][t] == pytest.approx(lam, rel=1e-14)
        assert out["stats"]["primal"][t] == pytest.approx(enet_primal(Q, y, out["beta"][t], lam, a),
                                                          rel=1e-12)
        assert out["stats"]["converged"][t] == 1


def test_enet_first_feature_enters(orc):
    """Just below lambda_max only j* = argmax |x_j^T y| is nonzero, with
    beta_j* = sign(c_j*) a (lambda_max - lambda) / (||x_j*||^2 + (1 - a) lambda)
    (KKT of the Elastic-Net with one active feature)."""
    a = 0.5
    prob = gen.small_problem(31, 40, 60, dtype=np.float64, k=3, noise=0.1)
    X, y = _dense(prob), prob["y"]
    c0 = X.T @ y
    js = int(np.argmax(np.abs(c0)))
    lmax = abs(c0[js]) / a
    ratio = 1.0 - 1e-4
    out = orc.lasso_path(X, y, [1.0, ratio], gap_tol_rel=1e-15, enet_alpha=a)
    assert np.all(out["beta"][0] == 0.0)
    lam = lmax * ratio
    expect = np.zeros(60)
    expect[js] = np.sign(c0[js]) * a * (lmax - lam) / (X[:, js] @ X[:, js] + (1 - a) * lam)
    np.testing.assert_allclose(out["beta"][1], expect, atol=1e-12 * lmax)


@pytest.mark.parametrize("seed,n,p,a", [(32, 20, 8, 0.5), (33, 9, 11, 0.2), (34, 14, 10, 0.9)])
def test_enet_bruteforce_agreement(orc, seed, n, p, a):
    """The exact Elastic-Net optimum from support-and-sign enumeration on the
    augmented design (a library-style exact Lasso solver on the paper's
    reduction): objective, support and coefficients agree; every screened
    feature is zero there."""
    prob = gen.small_problem(seed, n, p, dtype=np.float64, k=3, noise=0.3)
    X, y = _dense(prob), prob["y"]
    ratios = orc.lambda_ratios(7, 1.5)
    out = orc.lasso_path(X, y, ratios, gap_tol_rel=1e-15, max_epochs=200000, enet_alpha=a)
    lmax = out["lambda_max"]
    for t in range(1, len(ratios)):
        lam = lmax * ratios[t]
        Xa = np.vstack([X, np.sqrt((1 - a) * lam) * np.eye(p)])
        ya = np.concatenate([y, np.zeros(p)])
        bb, _ = lasso_bruteforce(Xa, ya, a * lam)
        b = out["beta"][t]
        assert enet_primal(X, y, b, lam, a) == pytest.approx(enet_primal(X, y, bb, lam, a), rel=1e-9)
        np.testing.assert_array_equal(b != 0, bb != 0)
        np.testing.assert_allclose(b, bb, atol=1e-6)
        kept = orc.unpack_mask(out["mask"][t], p)
        assert np.all(bb[~kept] == 0)


def test_enet_kkt_at_tight_solution(orc):
    """Elastic-Net optimality: x_j^T (y - X beta) - (1 - a) lam beta_j equals
    a lam sign(beta_j) on the support and is at most a lam in magnitude
    elsewhere."""
    a = 0.6
    prob = gen.small_problem(35, 50, 200, dtype=np.float64, k=5, noise=0.1, correlated=True)
    X, y = _dense(prob), prob["y"]
    ratios = orc.lambda_ratios(10, 2.0)
    out = orc.lasso_path(X, y, ratios, gap_tol_rel=1e-14, enet_alpha=a)
    for t in range(1, 10):
        lam = out["stats"]["lambda"][t]
        b = out["beta"][t]
        g = X.T @ (y - X @ b) - (1 - a) * lam * b
        tol = 1e-5 * a * lam
        assert np.all(np.abs(g) <= a * lam + tol)
        sup = b != 0
        assert sup.sum() > 0
        np.testing.assert_allclose(g[sup], a * lam * np.sign(b[sup]), atol=tol)


def test_enet_alpha_one_is_the_lasso(orc):
    prob = gen.small_problem(36, 30, 90, dtype=np.float64, k=4)
    X, y = _dense(prob), prob["y"]
    ratios = orc.lambda_ratios(6, 1.5)
    a = orc.lasso_path(X, y, ratios, gap_tol_rel=1e-10)
    b = orc.lasso_path(X, y, ratios, gap_tol_rel=1e-10, enet_alpha=1.0)
    np.testing.assert_array_equal(a["beta"], b["beta"])
    np.testing.assert_array_equal(a["mask"], b["mask"])


def test_enet_with_the_dome_is_safe(orc):
    """The dome test on the augmented design (Eq. (11) applied to the
    Elastic-Net's Lasso form): every feature it screens is zero at the exact
    Elastic-Net optimum, and the tight path equals the enumeration's."""
    a = 0.5
    prob = gen.small_problem(37, 14, 10, dtype=np.float64, k=3, noise=0.3)
    X, y = _dense(prob), prob["y"]
    ratios = orc.lambda_ratios(6, 1.5)
    out = orc.lasso_path(X, y, ratios, gap_tol_rel=1e-15, max_epochs=200000, enet_alpha=a, screen_rule=1,
                         screen_period=1)
    lmax = out["lambda_max"]
    screened = 0
    for t in range(1, len(ratios)):
        lam = lmax * ratios[t]
        Xa = np.vstack([X, np.sqrt((1 - a) * lam) * np.eye(10)])
        bb, _ = lasso_bruteforce(Xa, np.concatenate([y, np.zeros(10)]), a * lam)
        kept = orc.unpack_mask(out["mask"][t], 10)
        assert np.all(bb[~kept] == 0)
        screened += int((~kept).sum())
        np.testing.assert_allclose(out["beta"][t], bb, atol=1e-6)
    assert screened > 0


def test_enet_batch_equals_independent_paths(orc):
    """Row-subset Elastic-Net problems: each batched solve equals the plain
    Elastic-Net path on the gathered rows."""
    prob = gen.small_problem(38, 30, 40, dtype=np.float64, k=3)
    X, y = _dense(prob), prob["y"]
    rng = np.random.default_rng(38)
    B = 3
    rm = (rng.random((B, 30)) < 0.7).astype(np.uint8)
    Y = np.stack([y * rm[b] for b in range(B)])
    ratios = orc.lambda_ratios(5, 1.5)
    out = orc.lasso_batch(X, Y, ratios, row_mask=rm, gap_tol_rel=1e-10, enet_alpha=0.6)
    for b in range(B):
        rows = rm[b] != 0
        ref = orc.lasso_path(X[rows], y[rows], ratios, gap_tol_rel=1e-10, enet_alpha=0.6)
        np.testing.assert_array_equal(out["beta"][b], ref["beta"])


def test_enet_hand_examples(orc):
    """Hand-derived Elastic-Net cases (tests/golden/hand_examples.json):
    coefficients, primal and dual values at lambda, with lambda_max =
    ||X^T y||_inf / a."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")
    for case in json.load(open(path))["enet_cases"]:
        X = np.array(case["X"], dtype=np.float64)
        y = np.array(case["y"], dtype=np.float64)
        a = case["a"]
        ratio = case["lambda"] / (np.abs(X.T @ y).max() / a)
        out = orc.lasso_path(X, y, [1.0, ratio], gap_tol_rel=1e-15, enet_alpha=a)
        assert out["stats"]["lambda"][1] == pytest.approx(case["lambda"], rel=1e-15)
        np.testing.assert_allclose(out["beta"][1], case["beta"], atol=1e-12)
        assert out["stats"]["primal"][1] == pytest.approx(case["primal"], rel=1e-12)
        assert out["stats"]["dual"][1] == pytest.approx(case["dual"], rel=1e-12)


COMBOS = [
    dict(), dict(dual_point=1), dict(xtr_scope=1), dict(screen_rule=1), dict(refined_radius=1),
    dict(warm_start=False), dict(dual_point=1, xtr_scope=1, screen_rule=1, refined_radius=1),
    dict(enet_alpha=0.7), dict(enet_alpha=0.7, dual_point=1, xtr_scope=1),
    dict(enet_alpha=0.4, screen_rule=1, refined_radius=1), dict(enet_alpha=0.4, warm_start=False, screen_period=1),
]


@pytest.mark.parametrize("opt", COMBOS, ids=[",".join(f"{k}={v}" for k, v in c.items()) or "default" for c in COMBOS])
def test_every_option_combination_reaches_the_exact_solution(orc, opt):
    """Whatever the dual point, scope, safe region, radius, warm start and
    mixing, the screened path ends at the exact optimum (support enumeration
    on the augmented design; a = 1 is the Lasso) and screens only features
    that are zero there."""
    a = opt.get("enet_alpha", 1.0)
    prob = gen.small_problem(39, 16, 10, dtype=np.float64, k=3, noise=0.3, correlated=True)
    X, y = _dense(prob), prob["y"]
    ratios = orc.lambda_ratios(6, 1.5)
    out = orc.lasso_path(X, y, ratios, gap_tol_rel=1e-15, max_epochs=200000, **opt)
    assert out["status"] == 0
    lmax = out["lambda_max"]
    for t in range(1, len(ratios)):
        lam = lmax * ratios[t]
        Xa = np.vstack([X, np.sqrt((1 - a) * lam) * np.eye(10)])
        bb, _ = lasso_bruteforce(Xa, np.concatenate([y, np.zeros(10)]), a * lam)
        kept = orc.unpack_mask(out["mask"][t], 10)
        assert np.all(bb[~kept] == 0)
        np.testing.assert_array_equal(out["beta"][t] != 0, bb != 0)
        np.testing.assert_allclose(out["beta"][t], bb, atol=1e-6)
