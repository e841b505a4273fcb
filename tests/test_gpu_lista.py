"""Learned warm start on the GPU against the FP64 oracle (oracle/lista.py):
normalisation, forward pass, every gradient, Adam, the ISTA initialisation,
and a test of what the trained network gains over the zero start.

The GPU computes in FP32.  Inputs are rounded to FP32 first and the oracle
runs on those values widened to FP64, so the differences are the FP32
arithmetic alone: tolerances are stated relative to the largest magnitude of
each quantity."""
import numpy as np
import pytest

import gen
import oracle
from oracle import lista as olista

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


DEV = "cuda:0"


def _case(seed, n, p, L, B, ratio=0.1):
    rng = np.random.default_rng(seed)
    XT = gen.gaussian_design(rng, n, p, dtype=np.float32)  # (p, ldx), unit-norm columns
    X = XT[:, :n].astype(np.float64).T
    Y = rng.standard_normal((B, n))
    W, D, tau = olista.init_params(X, L, ratio)
    W = (W + 0.2 * rng.standard_normal(W.shape)).astype(np.float32)
    D = (D * rng.uniform(0.5, 1.5, D.shape)).astype(np.float32)
    tau = (tau * rng.uniform(0.3, 0.9, tau.shape)).astype(np.float32)
    s = olista.scales(X, Y)
    Ytil = (Y / s[:, None]).astype(np.float32)
    Tgt = (0.05 * rng.standard_normal((B, p))).astype(np.float32)
    return dict(XT=XT, X=X, n=n, p=p, L=L, B=B, Y=Y, W=W, D=D, tau=tau, Ytil=Ytil, Tgt=Tgt)


def _net(pkg, c):
    XT = torch.from_numpy(c["XT"]).to(DEV)
    net = pkg.ListaNet(XT, c["n"], L=c["L"], init=False)
    net.W.copy_(torch.from_numpy(c["W"]))
    net.D.copy_(torch.from_numpy(c["D"]))
    net.tau.copy_(torch.from_numpy(c["tau"]))
    return net


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))


SIZES = [(401, 37, 300, 3, 21), (402, 130, 3000, 4, 200), (403, 64, 1000, 8, 64)]


@pytest.mark.parametrize("seed,n,p,L,B", SIZES)
def test_normalize(pkg, seed, n, p, L, B):
    c = _case(seed, n, p, L, B)
    net = _net(pkg, c)
    Ytil, s = net.normalize(torch.from_numpy(c["Y"]).to(DEV))
    torch.cuda.synchronize()
    s_ref = olista.scales(c["X"], c["Y"])
    np.testing.assert_allclose(s.cpu().numpy(), s_ref, rtol=2e-6)
    np.testing.assert_allclose(Ytil.cpu().numpy(), c["Y"] / s_ref[:, None], rtol=4e-6, atol=1e-7)


@pytest.mark.parametrize("seed,n,p,L,B", SIZES)
def test_forward(pkg, seed, n, p, L, B):
    """beta^L within 2e-5 of max |beta^L| (the sizes split K = p of X beta
    over several CTAs, and the feature counts leave ragged tiles)."""
    c = _case(seed, n, p, L, B)
    net = _net(pkg, c)
    out = net.forward(torch.from_numpy(c["Ytil"]).to(DEV)).cpu().numpy()
    ref, _ = olista.forward(c["X"], c["W"].astype(np.float64), c["D"].astype(np.float64),
                            c["tau"].astype(np.float64), c["Ytil"].astype(np.float64))
    assert np.abs(ref).max() > 0
    assert np.abs(out - ref).max() <= 2e-5 * np.abs(ref).max()
    # the support: agreement except where |z| sits within rounding of tau
    frac = np.mean((out != 0) != (ref != 0))
    assert frac <= 1e-3


@pytest.mark.parametrize("seed,n,p,L,B", SIZES)
def test_backward(pkg, seed, n, p, L, B):
    """Loss within 1e-5 relative; each gradient within 1e-4 of its largest
    entry.  The ST indicator [|z| > tau] is a decision floating point takes:
    the oracle takes the kernel's own decisions (read from the forward cache)
    and does all arithmetic in FP64.  Decisions that differ from the FP64
    forward's are those within FP32 rounding of the kink; they are counted and
    must be rare."""
    c = _case(seed, n, p, L, B)
    net = _net(pkg, c)
    betaL = net.forward(torch.from_numpy(c["Ytil"]).to(DEV), keep_cache=True)
    loss = net.backward(betaL, torch.from_numpy(c["Tgt"]).to(DEV))
    torch.cuda.synchronize()
    z_gpu = net.cache(B)[2].cpu().numpy()
    masks = [np.abs(z_gpu[l]) > c["tau"][l] for l in range(L)]
    args = (c["X"], c["W"].astype(np.float64), c["D"].astype(np.float64), c["tau"].astype(np.float64),
            c["Ytil"].astype(np.float64), c["Tgt"].astype(np.float64))
    f, dW, dD, dt = olista.backward(*args, masks=masks)
    np.testing.assert_allclose(float(loss.item()), f, rtol=1e-5)
    gW, gD, gt = (g.cpu().numpy() for g in net.grads)
    assert _rel(gW, dW) <= 1e-4, _rel(gW, dW)
    assert _rel(gD, dD) <= 1e-4, _rel(gD, dD)
    assert _rel(gt, dt) <= 1e-4, _rel(gt, dt)
    _, cache64 = olista.forward(*args[:5])
    flips = sum(int(np.sum(masks[l] != (np.abs(cache64[l][2]) > args[3][l]))) for l in range(L))
    assert flips <= 1e-5 * L * B * p + 2, flips


def test_backward_is_deterministic(pkg):
    c = _case(404, 90, 2000, 5, 128)
    net = _net(pkg, c)
    res = []
    for _ in range(2):
        betaL = net.forward(torch.from_numpy(c["Ytil"]).to(DEV), keep_cache=True)
        net.backward(betaL, torch.from_numpy(c["Tgt"]).to(DEV))
        res.append([g.cpu().numpy().copy() for g in net.grads] + [net.loss.cpu().numpy().copy()])
    for a, b in zip(*res):
        np.testing.assert_array_equal(a, b)


def test_adam_matches_oracle(pkg):
    rng = np.random.default_rng(405)
    c = _case(405, 20, 100, 2, 4)
    net = _net(pkg, c)
    th = c["W"].astype(np.float64)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    for t in range(1, 6):
        g = rng.standard_normal(th.shape).astype(np.float32)
        net.grads[0].copy_(torch.from_numpy(g))
        net.grads[1].zero_()
        net.grads[2].zero_()
        net.adam(1e-2, relative=False)
        th, m, v = olista.adam_step(th, g.astype(np.float64), m, v, t, 1e-2)
    torch.cuda.synchronize()
    np.testing.assert_allclose(net.W.cpu().numpy(), th, rtol=0, atol=2e-6)
    np.testing.assert_allclose(net.m[0].cpu().numpy(), m, rtol=1e-5, atol=1e-7)


def test_init_is_ista(pkg):
    """W = X^T exactly; d = 1/Lip, tau = ratio/Lip with Lip the power-method
    estimate of ||X||_2^2 raised by 1 %; the network then agrees with ISTA at
    that step size."""
    c = _case(406, 60, 500, 6, 16, ratio=0.08)
    XT = torch.from_numpy(c["XT"]).to(DEV)
    net = pkg.ListaNet(XT, 60, L=6, ratio=0.08)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(net.W.cpu().numpy(), c["XT"][:, :60])
    # the power method approaches ||X||_2^2 from below: the estimate, scaled
    # up by 1 %, lies in [Lip, 1.01 Lip] once it is within 1 %
    lip = olista.lipschitz(c["X"])
    est = float(net.lip.item())
    assert lip * (1 - 1e-6) <= est <= 1.01 * lip * (1 + 1e-6), (est, lip)
    np.testing.assert_allclose(net.D.cpu().numpy(), 1.0 / est, rtol=1e-6)
    np.testing.assert_allclose(net.tau.cpu().numpy(), 0.08 / est, rtol=1e-6)
    out = net.forward(torch.from_numpy(c["Ytil"]).to(DEV)).cpu().numpy()
    for b in range(4):
        ref = olista.ista(c["X"], c["Ytil"][b].astype(np.float64), 0.08, est, 6)
        assert np.abs(out[b] - ref).max() <= 1e-4 * max(np.abs(ref).max(), 1e-12)


def test_warm_start_is_scaled_forward(pkg):
    c = _case(407, 50, 700, 4, 33)
    net = _net(pkg, c)
    Yd = torch.from_numpy(c["Y"]).to(DEV)
    b0 = net.warm_start(Yd, max_nonzeros=0).cpu().numpy()
    Ytil, s = net.normalize(Yd)
    out = net.forward(Ytil).cpu().numpy()
    np.testing.assert_allclose(b0, s.cpu().numpy()[:, None].astype(np.float64) * out, rtol=1e-6, atol=0)
    # the cut to the K largest magnitudes of every row
    for K in (1, 7, 50, 699):
        bk = net.warm_start(Yd, max_nonzeros=K).cpu().numpy()
        for b in range(33):
            full = b0[b]
            nz = np.count_nonzero(full)
            keep = np.abs(full) >= np.sort(np.abs(full))[-K] if K <= nz else full != 0
            if K < nz and np.sort(np.abs(full))[-K] == np.sort(np.abs(full))[-K - 1]:
                continue  # a tie at the cut drops all tied entries
            np.testing.assert_array_equal(bk[b], np.where(keep, full, 0.0))
            assert np.count_nonzero(bk[b]) <= K
    ref, _ = olista.forward(c["X"], c["W"].astype(np.float64), c["D"].astype(np.float64),
                            c["tau"].astype(np.float64), Ytil.cpu().numpy().astype(np.float64))
    sref = olista.scales(c["X"], c["Y"])
    assert np.abs(b0 - sref[:, None] * ref).max() <= 3e-5 * np.abs(sref[:, None] * ref).max()


def test_learned_warm_start_saves_work(pkg):
    """Train on solver solutions at lambda = lambda_max / 20 of a fixed
    120 x 1200 design (beta* with k ~ U{2..20}, the sparsity-to-rows ratio of
    the 300 x 10000, k <= 50 workload), then solve held-out responses from the
    zero start and from the network's beta0.  Every solve is gap-certified
    either way; the learned start needs fewer passes on average and reads
    at least 5 % fewer columns of X; and a warm-started solve equals the
    oracle's from the same beta0."""
    w = gen.workload4(seed=1104, n=120, p=1200, k_range=(2, 20))
    XT = torch.from_numpy(w["XT"]).to(DEV)
    n, p = w["n"], w["p"]
    ratio = torch.tensor([w["lambda_ratio"]], dtype=torch.float64, device=DEV)
    opts = pkg.lasso_default_opts(gemm_dtype=pkg.LASSO_F32)

    def solve(Y, beta0=None):
        out = pkg.solve_batch(XT, Y, ratio, n=n, beta0=beta0, opts=opts)
        st = pkg.stats_to_numpy(out["stats"]).reshape(Y.shape[0])
        return out["beta"][:, 0, :], st

    Ytr = torch.from_numpy(w["sample"](8192, 1)).to(DEV)
    bh, st = solve(Ytr)
    assert np.all(st["status"] == 0)
    net = pkg.ListaNet(XT, n, L=8, ratio=w["lambda_ratio"])
    Ytil, s = net.normalize(Ytr)
    tgt = net.targets(bh.contiguous(), s)
    hist = net.fit(Ytil, tgt, epochs=30, batch=256, lr=1e-2, seed=7)
    assert hist[-1] < 0.7 * hist[0], hist

    Yev = torch.from_numpy(w["sample"](512, 2)).to(DEV)
    _, st0 = solve(Yev)
    beta0 = net.warm_start(Yev)
    bw, st1 = solve(Yev, beta0=beta0)
    torch.cuda.synchronize()
    assert np.all(st0["status"] == 0) and np.all(st1["status"] == 0)
    e0, e1 = st0["epochs"].mean(), st1["epochs"].mean()
    x0, x1 = st0["x_columns"].sum(), st1["x_columns"].sum()
    print(f"learned start: passes {e0:.1f} -> {e1:.1f}, columns read {x0:.3e} -> {x1:.3e}")
    assert e1 < e0, (e0, e1)
    assert x1 <= 0.95 * x0, (x0, x1)

    pick = [0, 1, 2, 3]
    Ynp = Yev.cpu().numpy()[pick]
    o = oracle.lasso_batch(w["XT"], Ynp, np.array([w["lambda_ratio"]]), n=n, beta0=beta0.cpu().numpy()[pick],
                           gap_tol_rel=1e-6)
    np.testing.assert_allclose(bw.cpu().numpy()[pick], o["beta"][:, 0, :], atol=1e-5, rtol=0)
    np.testing.assert_array_equal(st1["epochs"][pick], o["stats"]["epochs"][:, 0].astype(np.int64))
