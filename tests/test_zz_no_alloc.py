"""lasso_path_static, the entry point for callers that cannot allocate device
memory (plug-ins under an application that owns the device heap, real-time
code whose hot path must not allocate): it must give the results of
lasso_path, call after call, although every call reuses the same static
scratch array.  This file is collected last on purpose."""
import numpy as np
import pytest

import gen

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


def _outputs(T, p, nbytes, dev):
    words = (p + 31) // 32
    return (torch.full((T, p), np.nan, dtype=torch.float64, device=dev),
            torch.zeros((T, words), dtype=torch.int32, device=dev),
            torch.zeros(T * nbytes, dtype=torch.uint8, device=dev))


def test_static_scratch_matches_workspace_entry(pkg):
    dev = torch.device("cuda:0")
    prob = gen.small_problem(301, 200, 3000, dtype=np.float32, k=10, noise=0.2, correlated=True)
    n, p = prob["n"], prob["p"]
    ratios_h = pkg.lasso_lambda_grid(20, 2.0)
    T = len(ratios_h)
    XT = torch.from_numpy(prob["XT"]).to(dev)
    y = torch.from_numpy(prob["y"]).to(dev)
    r = torch.from_numpy(ratios_h).to(dev)
    opts = pkg.lasso_default_opts(gap_tol_rel=1e-8)
    stream = torch.cuda.current_stream(dev).cuda_stream

    ref = pkg.solve_path(XT, y, r, n=n, opts=opts)
    torch.cuda.synchronize()
    ref_beta = ref["beta"].cpu().numpy()
    ref_mask = ref["mask"].cpu().numpy()
    ref_st = pkg.stats_to_numpy(ref["stats"])
    assert np.all(ref_st["status"] == 0)

    for call in range(2):
        beta, mask, stats = _outputs(T, p, pkg.STATS_DTYPE.itemsize, dev)
        pkg.lasso_path_static(XT.data_ptr(), pkg.LASSO_F32, n, p, prob["ldx"], y.data_ptr(), r.data_ptr(), T,
                              None, opts, beta.data_ptr(), mask.data_ptr(), stats.data_ptr(), stream)
        torch.cuda.synchronize()
        st = pkg.stats_to_numpy(stats)
        assert np.all(st["status"] == 0), (call, st["status"])
        np.testing.assert_allclose(beta.cpu().numpy(), ref_beta, atol=1e-5, rtol=0)
        np.testing.assert_allclose(st["primal"], ref_st["primal"], rtol=1e-9)
        np.testing.assert_array_equal(mask.cpu().numpy(), ref_mask)
        np.testing.assert_array_equal(st["epochs"], ref_st["epochs"])


def test_static_scratch_rejects_oversized_problems(pkg):
    """Problems whose workspace exceeds the static array are refused with a message."""
    opts = pkg.lasso_default_opts()
    with pytest.raises(pkg.LassoError) as e:
        pkg.lasso_path_static(0x10000, pkg.LASSO_F64, 500, 50000, 500, 0x20000, 0x30000, 10, None, opts,
                              0x40000, None, 0x50000, None)
    assert e.value.status == pkg.LASSO_ERR_INVALID_ARG
    assert "static" in pkg.lasso_last_error()


def test_static_scratch_reports_the_exact_reason(pkg):
    """An invalid option gets the same message from both entry points."""
    opts = pkg.lasso_default_opts(screen_period=0)
    with pytest.raises(pkg.LassoError) as e:
        pkg.lasso_path_static(0x10000, pkg.LASSO_F32, 64, 100, 64, 0x20000, 0x30000, 4, None, opts,
                              0x40000, None, 0x50000, None)
    assert e.value.status == pkg.LASSO_ERR_INVALID_ARG
    assert "screen_period" in pkg.lasso_last_error()
