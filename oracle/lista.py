"""FP64 CPU oracle of the learned warm start: an unrolled ISTA network.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the plain reference
the CUDA training and inference kernels are checked against.  It shares no
code with the CUDA library.  numpy FP64, no blocking or fusion: every line is
one step of the definitions below.

The paper has no learned component; this part only supplies a starting point
beta0 for the solver, whose safety never depends on it (any beta0 gives a
feasible dual point through the rescaling of Eq. (8), and every screening
test still uses an exactly computed duality gap).

Model.  For a response y (length n) let s = ||X^T y||_inf, the lambda_max of
y (Sec. 1.2), and ytil = y / s.  The Lasso solution is positively
homogeneous, beta_hat(c y, c lam) = c beta_hat(y, lam), so one network trained
on normalised responses serves every y at the fixed ratio lam / lambda_max.
With beta^0 = 0, layer l = 0 .. L-1 computes

    u_l       = ytil - X beta^l                  (residual)
    v_l       = W u_l                            (W: p x n, tied over layers)
    z_l       = beta^l + d_l * v_l               (d_l: length p, elementwise)
    beta^l+1  = ST(z_l, tau_l),  ST(z, t) = sign(z) max(|z| - t, 0)

and the warm start is s * beta^L.  With W = X^T, d_l = 1/Lip and
tau_l = r / Lip (Lip = ||X||_2^2) this is exactly L steps of ISTA on
min_b 1/2 ||ytil - X b||^2 + r ||b||_1, the special case the tests pin.

Training loss over a batch of B pairs (ytil_b, t_b), t_b = beta_hat_b / s_b:
    loss = 1/(2B) sum_b ||beta^L_b - t_b||^2.

Array layouts: X (n, p); Y, Ytil (B, n); beta and targets (B, p); W (p, n);
D (L, p); tau (L,).
"""
from __future__ import annotations

import numpy as np


def soft_threshold(z, t):
    """ST(z, t) = sign(z) max(|z| - t, 0)."""
    return np.sign(z) * np.maximum(np.abs(z) - t, 0.0)


def scales(X, Y):
    """s_b = ||X^T y_b||_inf for every row of Y (lambda_max of each response)."""
    return np.max(np.abs(Y @ X), axis=1)


def lipschitz(X):
    """Lip = ||X||_2^2, the largest eigenvalue of X^T X (LAPACK SVD)."""
    return float(np.linalg.norm(X, 2) ** 2)


def init_params(X, L, ratio):
    """ISTA initialisation: W = X^T, d_l = 1/Lip, tau_l = ratio/Lip."""
    lip = lipschitz(X)
    p = X.shape[1]
    W = X.T.copy()
    D = np.full((L, p), 1.0 / lip)
    tau = np.full(L, ratio / lip)
    return W, D, tau


def forward(X, W, D, tau, Ytil):
    """Returns beta^L (B, p) and the per-layer cache (u_l, v_l, z_l)."""
    B = Ytil.shape[0]
    p = X.shape[1]
    beta = np.zeros((B, p))
    cache = []
    for l in range(len(tau)):
        u = Ytil - beta @ X.T          # (B, n): ytil - X beta for every row
        v = u @ W.T                    # (B, p): W u
        z = beta + D[l] * v
        beta = soft_threshold(z, tau[l])
        cache.append((u, v, z))
    return beta, cache


def loss(betaL, Tgt):
    B = betaL.shape[0]
    return 0.5 * float(np.sum((betaL - Tgt) ** 2)) / B


def backward(X, W, D, tau, Ytil, Tgt, masks=None):
    """Loss and its gradients (dW, dD, dtau) by the chain rule through the L
    layers, taken from the last layer to the first.  The derivative of ST in
    z is the indicator [|z_l| > tau_l] (0 at the kink, a set of measure zero).
    masks, when given, is the list of per-layer indicators to use instead:
    a decision that floating point takes is then taken in the precision of
    the implementation under test (its own indicators), while every
    arithmetic step stays FP64."""
    betaL, cache = forward(X, W, D, tau, Ytil)
    B = Ytil.shape[0]
    g = (betaL - Tgt) / B                # d loss / d beta^L
    dW = np.zeros_like(W)
    dD = np.zeros_like(D)
    dtau = np.zeros_like(tau)
    for l in range(len(tau) - 1, -1, -1):
        u, v, z = cache[l]
        ind = (np.abs(z) > tau[l]) if masks is None else masks[l]
        gz = g * ind                     # through ST in z
        dtau[l] = -np.sum(np.sign(z) * gz)
        dD[l] = np.sum(gz * v, axis=0)
        gv = D[l] * gz
        dW += gv.T @ u                   # sum_b gv_b u_b^T
        gu = gv @ W                      # W^T gv for every row
        g = gz - gu @ X                  # d/d beta^l: direct term and through u = ytil - X beta
    return loss(betaL, Tgt), dW, dD, dtau


def adam_step(theta, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, 2015, Algorithm 1) at step t >= 1; returns
    the new (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def ista(X, ytil, r, lip, L):
    """L plain ISTA steps from 0 on 1/2 ||ytil - X b||^2 + r ||b||_1 (the
    textbook proximal-gradient iteration, step 1/Lip)."""
    b = np.zeros(X.shape[1])
    for _ in range(L):
        grad = X.T @ (X @ b - ytil)
        b = soft_threshold(b - grad / lip, r / lip)
    return b
