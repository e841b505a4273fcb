"""The tensor-core batched correlations C = X^T R (tcgen05, BF16 in, FP32
accumulate) against an FP64 product of the same BF16 values, with the
rigorous bound of an FP32 sum of n exact products, on ragged sizes."""
import numpy as np
import pytest

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


def _colmajor_bf16(M, ld, dev):
    """(rows=n, cols) float64 numpy -> (cols, ld) BF16 CUDA tensor, zero padded."""
    n, cols = M.shape
    out = torch.zeros((cols, ld), dtype=torch.bfloat16, device=dev)
    out[:, :n] = torch.from_numpy(np.ascontiguousarray(M.T)).to(dev).to(torch.bfloat16)
    return out


@pytest.mark.parametrize("n,p,B", [(1000, 3000, 200), (64, 128, 128), (130, 257, 33), (2000, 1000, 300)])
def test_correlations_bf16(pkg, n, p, B):
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(n + p + B)
    X = rng.standard_normal((n, p))
    R = rng.standard_normal((n, B)) * rng.uniform(0.1, 10, size=B)
    ldx = (n + 7) // 8 * 8
    Xb = _colmajor_bf16(X, ldx, dev)
    Rb = _colmajor_bf16(R, ldx, dev)
    C = torch.full((B, p), float("nan"), dtype=torch.float32, device=dev)
    ws = torch.empty(256, dtype=torch.uint8, device=dev)
    pkg.lasso_correlations_bf16(Xb.data_ptr(), n, p, ldx, Rb.data_ptr(), ldx, B, C.data_ptr(), p, ws.data_ptr(),
                                256, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert int(ws[:4].view(torch.int32).item()) == 0
    Xf = Xb[:, :n].double().cpu().numpy()  # (p, n) exact BF16 values
    Rf = Rb[:, :n].double().cpu().numpy()  # (B, n)
    ref = Rf @ Xf.T                        # (B, p) in FP64
    bound = (n + 4) * 2.0 ** -24 * (np.abs(Rf) @ np.abs(Xf).T) + 1e-30
    got = C.double().cpu().numpy()
    assert np.all(np.isfinite(got))
    assert np.all(np.abs(got - ref) <= bound), np.max(np.abs(got - ref) / bound)


@pytest.mark.parametrize("n,p,ldx", [(500, 50000, 500), (37, 1001, 40), (130, 3000, 132), (1000, 20000, 1000),
                                     (2048, 777, 2048), (1, 5, 4), (129, 64, 132)])
def test_correlations_f32(pkg, n, p, ldx):
    """c = X^T r for an FP32 design: each c_j within (4 ceil(n/128) + 6) 2^-24
    sum_i |x_ij r_i| of the FP64 product of the same FP32 values, the maximum
    equal to max_j |c_j|, and padding rows of X ignored."""
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(n * 7 + p)
    X = rng.standard_normal((p, ldx)).astype(np.float32)
    X[:, n:] = np.nan  # padding rows must not be read into the sums
    r = rng.standard_normal(n).astype(np.float32)
    Xd = torch.from_numpy(X).to(dev)
    rd = torch.from_numpy(r).to(dev)
    c = torch.full((p,), float("nan"), dtype=torch.float32, device=dev)
    m = torch.zeros((1,), dtype=torch.float32, device=dev)
    pkg.lasso_correlations_f32(Xd.data_ptr(), n, p, ldx, rd.data_ptr(), c.data_ptr(), m.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    cg = c.cpu().numpy().astype(np.float64)
    X64 = X[:, :n].astype(np.float64)
    exact = X64 @ r.astype(np.float64)
    bound = (4 * ((n + 127) // 128) + 6) * 2.0 ** -24 * (np.abs(X64) @ np.abs(r.astype(np.float64)))
    assert np.all(np.abs(cg - exact) <= bound), float(np.max(np.abs(cg - exact) / bound))
    assert float(m.item()) == float(np.max(np.abs(cg)))
