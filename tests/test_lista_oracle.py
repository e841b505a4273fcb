"""Pins of the FP64 learned-warm-start oracle (oracle/lista.py) against facts
that do not come from the oracle itself: finite differences of the forward
map, the textbook ISTA iteration, the soft-thresholding closed form on an
orthonormal design, Adam's first step, and the homogeneity of the Lasso
solution that the input normalisation relies on."""
import numpy as np
import pytest

from oracle import lista


def _problem(seed, n=7, p=12, L=3, B=4, ratio=0.3):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, p))
    X /= np.linalg.norm(X, axis=0)
    Y = rng.standard_normal((B, n))
    s = lista.scales(X, Y)
    Ytil = Y / s[:, None]
    W, D, tau = lista.init_params(X, L, ratio)
    # move away from the ISTA point so every parameter matters
    W = W + 0.2 * rng.standard_normal(W.shape)
    D = D * rng.uniform(0.5, 1.5, D.shape)
    tau = tau * rng.uniform(0.3, 0.9, tau.shape)
    Tgt = 0.3 * rng.standard_normal((B, p))
    return X, Ytil, W, D, tau, Tgt


def test_gradients_match_central_differences():
    """Every entry of dW, dD and dtau against central differences of the FP64
    forward loss (h = 1e-6), relative error <= 1e-6."""
    X, Ytil, W, D, tau, Tgt = _problem(1)
    f0, dW, dD, dtau = lista.backward(X, W, D, tau, Ytil, Tgt)
    h = 1e-6

    def fd(get, set_, shape):
        out = np.zeros(shape)
        for idx in np.ndindex(*shape):
            v = get(idx)
            set_(idx, v + h)
            fp = lista.loss(lista.forward(X, W, D, tau, Ytil)[0], Tgt)
            set_(idx, v - h)
            fm = lista.loss(lista.forward(X, W, D, tau, Ytil)[0], Tgt)
            set_(idx, v)
            out[idx] = (fp - fm) / (2 * h)
        return out

    gW = fd(lambda i: W[i], lambda i, v: W.__setitem__(i, v), W.shape)
    gD = fd(lambda i: D[i], lambda i, v: D.__setitem__(i, v), D.shape)
    gt = fd(lambda i: tau[i], lambda i, v: tau.__setitem__(i, v), tau.shape)
    for an, num in ((dW, gW), (dD, gD), (dtau, gt)):
        scale = max(np.abs(num).max(), 1e-12)
        assert np.abs(an - num).max() <= 1e-6 * scale, (np.abs(an - num).max(), scale)
    assert np.abs(dW).max() > 0 and np.abs(dD).max() > 0 and np.abs(dtau).max() > 0


def test_ista_initialisation_is_ista():
    """W = X^T, d = 1/Lip, tau = r/Lip: the network is L ISTA steps."""
    rng = np.random.default_rng(2)
    n, p, L, r = 20, 50, 8, 0.05
    X = rng.standard_normal((n, p))
    X /= np.linalg.norm(X, axis=0)
    Y = rng.standard_normal((5, n))
    Ytil = Y / lista.scales(X, Y)[:, None]
    W, D, tau = lista.init_params(X, L, r)
    beta, _ = lista.forward(X, W, D, tau, Ytil)
    lip = lista.lipschitz(X)
    for b in range(5):
        np.testing.assert_allclose(beta[b], lista.ista(X, Ytil[b], r, lip, L), rtol=0, atol=1e-13)
    # and ISTA itself decreases the Lasso objective monotonically
    P = lambda bb, y: 0.5 * np.sum((y - X @ bb) ** 2) + r * np.abs(bb).sum()
    prev = P(np.zeros(p), Ytil[0])
    for k in range(1, 6):
        cur = P(lista.ista(X, Ytil[0], r, lip, k), Ytil[0])
        assert cur <= prev + 1e-15
        prev = cur


def test_orthonormal_design_one_layer_is_exact():
    """X^T X = I: one ISTA step from 0 with step 1 is ST(X^T y, r), the exact
    Lasso solution, which every later layer leaves unchanged."""
    rng = np.random.default_rng(3)
    n, p, r = 40, 15, 0.1
    X, _ = np.linalg.qr(rng.standard_normal((n, p)))
    Y = rng.standard_normal((3, n))
    Ytil = Y / lista.scales(X, Y)[:, None]
    W, D, tau = X.T.copy(), np.ones((4, p)), np.full(4, r)
    beta, _ = lista.forward(X, W, D, tau, Ytil)
    exact = np.sign(Ytil @ X) * np.maximum(np.abs(Ytil @ X) - r, 0.0)
    np.testing.assert_allclose(beta, exact, rtol=0, atol=1e-14)
    assert np.count_nonzero(exact) > 0 and np.count_nonzero(exact) < exact.size


def test_adam_first_step_moves_by_lr_times_sign():
    """With m = v = 0 at t = 1 the bias-corrected step is g / (|g| + eps)."""
    rng = np.random.default_rng(4)
    th = rng.standard_normal(50)
    g = rng.standard_normal(50)
    new, m, v = lista.adam_step(th, g, np.zeros(50), np.zeros(50), 1, lr=1e-2, eps=1e-8)
    np.testing.assert_allclose(new, th - 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-14)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-14)


def test_normalisation_is_scale_free():
    """s(c y) = c s(y), so the normalised input and the network output do not
    depend on the scale of y, and s * beta^L scales with y like the Lasso
    solution at lambda = ratio * lambda_max."""
    X, Ytil, W, D, tau, _ = _problem(5)
    rng = np.random.default_rng(5)
    Y = rng.standard_normal((3, X.shape[0]))
    s = lista.scales(X, Y)
    np.testing.assert_allclose(lista.scales(X, 7.5 * Y), 7.5 * s, rtol=1e-15)
    b1, _ = lista.forward(X, W, D, tau, Y / s[:, None])
    b2, _ = lista.forward(X, W, D, tau, (7.5 * Y) / (7.5 * s)[:, None])
    np.testing.assert_allclose(b1, b2, rtol=1e-14, atol=1e-15)


def test_loss_zero_at_target_and_gradient_zero():
    X, Ytil, W, D, tau, _ = _problem(6)
    betaL, _ = lista.forward(X, W, D, tau, Ytil)
    f, dW, dD, dtau = lista.backward(X, W, D, tau, Ytil, betaL)
    assert f == 0.0
    assert not dW.any() and not dD.any() and not dtau.any()


@pytest.mark.parametrize("mutant", ["sign_u", "drop_direct", "no_mask", "tau_sign"])
def test_gradient_check_catches_planted_mistakes(mutant, monkeypatch):
    """A plausible slip in the backward pass (planted here in a copy, on the
    CPU) fails the finite-difference comparison."""
    X, Ytil, W, D, tau, Tgt = _problem(7)
    f0, dW, dD, dtau = lista.backward(X, W, D, tau, Ytil, Tgt)

    def bad_backward(X, W, D, tau, Ytil, Tgt):
        betaL, cache = lista.forward(X, W, D, tau, Ytil)
        B = Ytil.shape[0]
        g = (betaL - Tgt) / B
        dW_, dD_, dt_ = np.zeros_like(W), np.zeros_like(D), np.zeros_like(tau)
        for l in range(len(tau) - 1, -1, -1):
            u, v, z = cache[l]
            gz = g if mutant == "no_mask" else g * (np.abs(z) > tau[l])
            dt_[l] = (1 if mutant == "tau_sign" else -1) * np.sum(np.sign(z) * gz)
            dD_[l] = np.sum(gz * v, axis=0)
            gv = D[l] * gz
            dW_ += gv.T @ u
            gu = gv @ W
            if mutant == "sign_u":
                g = gz + gu @ X
            elif mutant == "drop_direct":
                g = -gu @ X
            else:
                g = gz - gu @ X
        return dW_, dD_, dt_

    bW, bD, bt = bad_backward(X, W, D, tau, Ytil, Tgt)
    err = max(np.abs(bW - dW).max() / np.abs(dW).max(), np.abs(bD - dD).max() / np.abs(dD).max(),
              np.abs(bt - dtau).max() / np.abs(dtau).max())
    assert err > 1e-3
