"""Pins of the oracle's GAP SAFE dome test (Eq. (11), appendix "Dome test").

The dome's support function is checked against a sampled maximisation over
the dome itself, and the dome's parameters against the set they are derived
from: theta_hat lies in the ball with diameter [theta, y/lambda] (it is the
projection of y/lambda on the dual feasible set, and theta is feasible) and
at distance >= r(beta) from y/lambda (D(theta_hat) <= P(beta), Thm. 2).  The
maximum of x_j^T z over that set is sampled on its boundary and compared with
the oracle's test value.  None of these re-types the oracle's formulas.
"""
import numpy as np
import pytest

import gen
from oracle.bruteforce import lasso_bruteforce


def _dense(prob):
    return prob["XT"][:, :prob["n"]].T.astype(np.float64)


def _unit_sphere(rng, m, d):
    u = rng.standard_normal((m, d))
    return u / np.linalg.norm(u, axis=1, keepdims=True)


@pytest.mark.parametrize("alpha", [-1.0, -0.6, 0.0, 0.35, 0.8, 0.97])
def test_dome_support_matches_sampled_maximum(orc, alpha):
    """sigma_D(x) = max over the dome D(c, rad, alpha, nrm) of x^T z: the
    closed form equals the maximum over dense samples of the dome's boundary
    (its spherical cap and the circle where the hyperplane cuts the sphere),
    in R^3, for directions x on both sides of the hyperplane."""
    rng = np.random.default_rng(int(1000 * (alpha + 2)))
    c = rng.standard_normal(3)
    rad = 0.7
    nrm = _unit_sphere(rng, 1, 3)[0]
    u = _unit_sphere(rng, 400000, 3)
    cap = u[u @ nrm <= -alpha]
    # the rim: u = -alpha nrm + sqrt(1 - alpha^2) w, w a unit vector orthogonal to nrm
    w = _unit_sphere(rng, 20000, 3)
    w -= np.outer(w @ nrm, nrm)
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    rim = -alpha * nrm + np.sqrt(max(1 - alpha * alpha, 0.0)) * w
    pts = c + rad * np.vstack([cap, rim])
    for x in list(_unit_sphere(rng, 12, 3) * 2.5) + [2.0 * nrm, -1.5 * nrm]:
        sig = orc.dome_support(c @ x, rad, alpha, nrm @ x, np.linalg.norm(x))
        best = (pts @ x).max()
        assert best <= sig + 1e-12
        assert sig <= best + 2e-4 * rad * np.linalg.norm(x), (alpha, sig, best)


def _states(orc, X, y, lam, passes):
    """(beta, rho) after 0, 1, ... cyclic CD passes from beta = 0 at lam."""
    p = X.shape[1]
    beta, rho = np.zeros(p), y.copy()
    out = [(beta.copy(), rho.copy())]
    for k in range(max(passes)):
        beta, rho = orc.cd_pass(X, beta, rho, lam, np.arange(p))
        if k + 1 in passes:
            out.append((beta.copy(), rho.copy()))
    return out


@pytest.mark.parametrize("dual_point", [0, 1])
def test_dome_value_is_the_maximum_over_the_safe_set(orc, dual_point):
    """For three rows the set S = {z : (z - y/l)^T (z - theta) <= 0,
    ||z - y/l|| >= r(beta)} is sampled on its boundary (the part of the sphere
    with diameter [theta, y/l] outside the ball B(y/l, r), and the circle
    where the two spheres meet); max_{z in S} |x_j^T z| must equal the
    oracle's dome test value of every feature (S's convex hull is the dome,
    so the maxima agree)."""
    rng = np.random.default_rng(41)
    n, p = 3, 9
    X = rng.standard_normal((n, p))
    X /= np.linalg.norm(X, axis=0)
    y = rng.standard_normal(n) * 2
    lmax = np.abs(X.T @ y).max()
    lam = 0.45 * lmax
    u = _unit_sphere(rng, 400000, n)
    w0 = _unit_sphere(rng, 20000, n)
    checked = 0
    for beta, rho in _states(orc, X, y, lam, (1, 3)):
        res = orc.check(X, y, beta, rho, lam, screen_rule=1, dual_point=dual_point)
        theta = res["alpha"] * rho
        yl = y / lam
        R = np.linalg.norm(yl - theta)
        r2 = max(0.0, y @ y - 2 * res["primal"]) / lam ** 2
        z = 0.5 * (yl + theta) + 0.5 * R * u            # the sphere with diameter [theta, y/l]
        z = z[np.sum((z - yl) ** 2, axis=1) >= r2]      # at distance >= r from y/l
        assert len(z) > 1000
        if r2 > 0:
            # the circle where the two spheres meet: its plane is orthogonal to
            # e = (theta - y/l)/R at distance x = r^2/R from y/l (two-sphere
            # intersection with center distance R/2 and radii R/2, r)
            e = (theta - yl) / R
            x = r2 / R
            w = w0 - np.outer(w0 @ e, e)
            w /= np.linalg.norm(w, axis=1, keepdims=True)
            z = np.vstack([z, yl + x * e + np.sqrt(max(r2 - x * x, 0.0)) * w])
        best = np.abs(z @ X).max(axis=0)
        scale = np.linalg.norm(X, axis=0) * R
        assert np.all(best <= res["mu"] + 1e-9), (best, res["mu"])
        assert np.all(res["mu"] <= best + 2e-4 * scale), (best, res["mu"])
        assert res["dome_rad"] == pytest.approx(R / 2, rel=1e-9)
        checked += 1
    assert checked == 3


def test_dome_lies_inside_the_sphere(orc):
    """The dome is contained in the GAP SAFE sphere (Sec. 3, the convergence
    proof of the safe regions): its test value never exceeds the sphere's,
    and on a correlated design it screens strictly more features at some
    check."""
    prob = gen.small_problem(42, 40, 160, dtype=np.float64, k=5, noise=0.1, correlated=True)
    X, y = _dense(prob), prob["y"]
    lmax = np.abs(X.T @ y).max()
    more = 0
    for ratio in (0.8, 0.5, 0.2):
        lam = ratio * lmax
        for beta, rho in _states(orc, X, y, lam, (1, 2, 5, 20)):
            s = orc.check(X, y, beta, rho, lam)
            d = orc.check(X, y, beta, rho, lam, screen_rule=1)
            assert np.all(d["mu"] <= s["mu"] * (1 + 1e-12) + 1e-12)
            ks, kd = orc.unpack_mask(s["mask"], 160), orc.unpack_mask(d["mask"], 160)
            assert np.all(kd <= ks)
            more += int(ks.sum() - kd.sum())
            assert s["gap"] == d["gap"] and s["alpha"] == d["alpha"]
    assert more > 0


def test_every_dome_contains_dual_optimum(orc):
    """Thm. 2: at every check of a path run with the dome, theta_hat (from the
    exact brute-force beta) lies in the dome with the logged radius and
    ratio, center (y/l + theta_k)/2 and unit normal (y/l - theta_k)/R."""
    prob = gen.small_problem(43, 15, 10, dtype=np.float64, k=3, noise=0.2)
    X, y = _dense(prob), prob["y"]
    ratios = orc.lambda_ratios(6, 1.5)
    out = orc.lasso_path(X, y, ratios, gap_tol_rel=1e-13, log_checks=5000, screen_period=1,
                         screen_rule=1)
    lmax = out["lambda_max"]
    thetas = {t: (y - X @ lasso_bruteforce(X, y, lmax * ratios[t])[0]) / (lmax * ratios[t])
              for t in range(len(ratios))}
    log = out["log"]
    inner = 0
    for k in range(len(log["t"])):
        t = int(log["t"][k])
        lam = lmax * ratios[t]
        theta = log["alpha"][k] * log["rho"][k]
        R = np.linalg.norm(y / lam - theta)
        if log["dome_rad"][k] == 0.0:
            assert R == 0.0
            continue
        c = 0.5 * (y / lam + theta)
        nrm = (y / lam - theta) / R
        rad, al = log["dome_rad"][k], log["dome_alpha"][k]
        d = thetas[t] - c
        assert np.linalg.norm(d) <= rad * (1 + 1e-9) + 1e-12
        assert nrm @ d <= -al * rad + 1e-9 * rad + 1e-12
        inner += al > -1.0
    assert inner > 10


@pytest.mark.parametrize("seed,n,p", [(44, 20, 8), (45, 12, 11)])
def test_dome_path_reaches_the_exact_solution(orc, seed, n, p):
    """With the dome, every screened feature is zero at the exact optimum
    (Eq. (5)) and the tight path equals the brute-force solution."""
    prob = gen.small_problem(seed, n, p, dtype=np.float64, k=3, noise=0.3)
    X, y = _dense(prob), prob["y"]
    ratios = orc.lambda_ratios(8, 1.5)
    out = orc.lasso_path(X, y, ratios, gap_tol_rel=1e-15, max_epochs=200000, screen_rule=1)
    lmax = out["lambda_max"]
    for t in range(1, len(ratios)):
        bb, _ = lasso_bruteforce(X, y, lmax * ratios[t])
        kept = orc.unpack_mask(out["mask"][t], p)
        assert np.all(bb[~kept] == 0)
        np.testing.assert_array_equal(out["beta"][t] != 0, bb != 0)
        np.testing.assert_allclose(out["beta"][t], bb, atol=1e-6)
