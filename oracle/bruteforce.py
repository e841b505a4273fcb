"""Exact Lasso solution by exhaustive support-and-sign enumeration (p <= 12).

TEST INFRASTRUCTURE ONLY (part of the oracle package).

For a fixed support S and sign vector s, the stationarity condition of the
Lasso restricted to S (Eq. (3)-(4): x_j^T (y - X beta) = lambda s_j on S) is
the linear system X_S^T X_S beta_S = X_S^T y - lambda s.  A candidate is a
solution iff its signs agree with s and the off-support KKT inequality
|x_j^T (y - X beta)| <= lambda holds (Eq. (4)).  Among all candidates (the
empty support included) the one of least P_lambda (Eq. (1)) is returned.
Independent of coordinate descent; used to pin the oracle on tiny designs.
"""
from __future__ import annotations

import itertools

import numpy as np


def primal(X, y, beta, lam):
    """P_lambda(beta) = 1/2 ||X beta - y||^2 + lambda ||beta||_1 (Eq. (1))."""
    r = X @ beta - y
    return 0.5 * float(r @ r) + lam * float(np.abs(beta).sum())


def lasso_bruteforce(X, y, lam, kkt_rtol=1e-9):
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n, p = X.shape
    if p > 12:
        raise ValueError("brute force limited to p <= 12")
    best_beta = np.zeros(p)
    best_P = primal(X, y, best_beta, lam)
    c0 = X.T @ y
    best_ok = bool(np.all(np.abs(c0) <= lam * (1 + kkt_rtol)))
    for k in range(1, min(n, p) + 1):
        for S in itertools.combinations(range(p), k):
            S = list(S)
            XS = X[:, S]
            G = XS.T @ XS
            try:
                Ginv = np.linalg.inv(G)
            except np.linalg.LinAlgError:
                continue
            b = XS.T @ y
            for signs in itertools.product((-1.0, 1.0), repeat=k):
                s = np.array(signs)
                bS = Ginv @ (b - lam * s)
                if np.any(np.sign(bS) != s):
                    continue
                beta = np.zeros(p)
                beta[S] = bS
                corr = X.T @ (y - X @ beta)
                off = np.ones(p, dtype=bool)
                off[S] = False
                if np.any(np.abs(corr[off]) > lam * (1 + kkt_rtol)):
                    continue
                P = primal(X, y, beta, lam)
                if not best_ok or P < best_P:
                    best_P, best_beta, best_ok = P, beta, True
    if not best_ok:
        raise RuntimeError("no KKT-consistent candidate found")
    return best_beta, best_P
