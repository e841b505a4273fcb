"""Row a11 measured: with audit_bounds = 1 every check also computes each
x_j^T rho exactly and records the largest |c~_j - x_j^T rho| / E_j of the
reduced-precision correlations c~ (FP32 CUDA-core dots, or the split-BF16
tensor-core product of a lockstep batch) against the forward-error bounds
E_j that the safe test of Eq. (7) is tightened by.  Every bound must hold
(ratio <= 1), and the audit must not change any result."""
import numpy as np
import pytest

import gen
import oracle
from tests.test_gpu_batch import run_gpu_batch
from tests.test_gpu_path import run_gpu

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


def _same(g0, g1):
    np.testing.assert_array_equal(g0["beta"], g1["beta"])
    np.testing.assert_array_equal(g0["mask"], g1["mask"])
    for k in ("epochs", "checks", "n_active", "n_nonzero", "primal", "gap"):
        np.testing.assert_array_equal(g0["stats"][k], g1["stats"][k])


@pytest.mark.parametrize("dtype,enet", [(np.float32, 1.0), (np.float64, 1.0), (np.float32, 0.7)])
def test_single_path_bounds_hold(pkg, dtype, enet):
    prob = gen.small_problem(611, 300, 4000, dtype=dtype, k=25, noise=0.1, correlated=True)
    ratios = oracle.lambda_ratios(20, 2.5)
    g0 = run_gpu(pkg, prob, ratios, enet_alpha=enet)
    g1 = run_gpu(pkg, prob, ratios, enet_alpha=enet, audit_bounds=1)
    _same(g0, g1)
    r = g1["stats"]["bound_ratio"]
    assert np.all(g0["stats"]["bound_ratio"] == 0)
    assert np.all(r <= 1.0), r.max()
    assert r.max() > 0.0
    assert np.all(g1["stats"]["bound_ratio_tc"] == 0)


@pytest.mark.parametrize("gemm", [2, 1])
def test_batch_bounds_hold(pkg, gemm):
    w = gen.workload3(B=6)
    ratios = oracle.lambda_ratios(w["T"], w["delta"])[:10]
    opt = dict(gap_tol_rel=w["tol"], screen_period=w["f"], gemm_dtype=gemm)
    g0 = run_gpu_batch(pkg, w["XT"], w["n"], w["Y"], w["row_mask"], ratios, **opt)
    g1 = run_gpu_batch(pkg, w["XT"], w["n"], w["Y"], w["row_mask"], ratios, audit_bounds=1, **opt)
    _same(g0, g1)
    st = g1["stats"]
    assert np.all(st["bound_ratio"] <= 1.0) and np.all(st["bound_ratio_tc"] <= 1.0)
    if gemm == 2:
        # the first check of every lambda comes from the tensor-core product
        assert st["bound_ratio_tc"].max() > 0.0
    else:
        assert np.all(st["bound_ratio_tc"] == 0.0)
    assert st["bound_ratio"].max() > 0.0
