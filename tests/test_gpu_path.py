"""GPU path vs the FP64 oracle, element by element on the same seeded inputs.

Tolerances (from the acceptance rule of the solver): at gap <= tol * ||y||^2
the objectives agree to 1e-9 relative, coefficients to 1e-5 absolute, and
supports and safe-active masks are identical.  Both sides run Algorithm 1
with the same options, so the iterates agree up to rounding; the per-lambda
pass counts are compared too.
"""
import numpy as np
import pytest

import gen
import oracle

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


def run_gpu(pkg, prob, ratios, beta0=None, **opt):
    dev = torch.device("cuda:0")
    XT = torch.from_numpy(np.ascontiguousarray(prob["XT"])).to(dev)
    y = torch.from_numpy(np.ascontiguousarray(prob["y"], dtype=np.float64)).to(dev)
    r = torch.from_numpy(np.ascontiguousarray(ratios, dtype=np.float64)).to(dev)
    b0 = None if beta0 is None else torch.from_numpy(np.ascontiguousarray(beta0, dtype=np.float64)).to(dev)
    out = pkg.solve_path(XT, y, r, n=prob["n"], beta0=b0, opts=pkg.lasso_default_opts(**opt))
    torch.cuda.synchronize()
    st = pkg.stats_to_numpy(out["stats"])
    return dict(beta=out["beta"].cpu().numpy(), mask=out["mask"].cpu().numpy().view(np.uint32), stats=st)


def run_orc(prob, ratios, beta0=None, **opt):
    return oracle.lasso_path(prob["XT"], prob["y"], ratios, n=prob["n"], beta0=beta0, **opt)


def assert_parity(g, o, check_epochs=True, rtol_obj=1e-9, atol_beta=1e-5):
    st, so = g["stats"], o["stats"]
    T = len(st)
    assert np.all(st["status"] == np.where(so["converged"] == 1, 0, 5)), (st["status"], so["converged"])
    # lambda_max is a sum of n products: the two sides round it differently
    np.testing.assert_allclose(st["lambda"], so["lambda"], rtol=1e-12)
    np.testing.assert_allclose(st["primal"], so["primal"], rtol=rtol_obj)
    np.testing.assert_allclose(g["beta"], o["beta"], atol=atol_beta, rtol=0)
    np.testing.assert_array_equal(g["beta"] != 0, o["beta"] != 0)
    np.testing.assert_array_equal(g["mask"], o["mask"])
    np.testing.assert_array_equal(st["n_active"], so["n_active"].astype(np.int64))
    np.testing.assert_array_equal(st["n_nonzero"], so["n_nonzero"].astype(np.int64))
    if check_epochs:
        np.testing.assert_array_equal(st["epochs"], so["epochs"].astype(np.int64))
        np.testing.assert_array_equal(st["checks"], so["checks"].astype(np.int64))
    assert T == len(so["lambda"])


CASES = [
    # (seed, n, p, dtype, correlated) -- ragged n and p, several CTA slices
    (101, 37, 300, np.float64, False),
    (102, 77, 1537, np.float32, False),
    (103, 130, 3000, np.float32, True),
    (104, 64, 5000, np.float64, True),
    (105, 500, 2500, np.float32, True),
    (106, 611, 900, np.float32, False),
    (107, 1100, 1300, np.float32, False),
    (108, 2048, 700, np.float32, False),
]


@pytest.mark.parametrize("seed,n,p,dtype,corr", CASES)
def test_path_parity(pkg, seed, n, p, dtype, corr):
    prob = gen.small_problem(seed, n, p, dtype=dtype, k=max(2, min(n, p) // 20), noise=0.2, correlated=corr)
    ratios = oracle.lambda_ratios(16, 2.0)
    g = run_gpu(pkg, prob, ratios, gap_tol_rel=1e-9)
    o = run_orc(prob, ratios, gap_tol_rel=1e-9)
    assert_parity(g, o)


def test_path_parity_workload1(pkg):
    """The full FP64 workload: Gaussian 100 x 1000, 100-point grid to
    lambda_max/1000, checks every 10 passes, gap <= 1e-6 ||y||^2."""
    w = gen.workload1()
    ratios = oracle.lambda_ratios(w["T"], w["delta"])
    g = run_gpu(pkg, w, ratios, screen_period=w["f"], gap_tol_rel=w["tol"])
    o = run_orc(w, ratios, screen_period=w["f"], gap_tol_rel=w["tol"])
    assert_parity(g, o)


@pytest.mark.parametrize("opt", [dict(dual_point=1), dict(xtr_scope=1), dict(warm_start=0),
                                 dict(screen_period=1), dict(screen_period=3, dual_point=1, xtr_scope=1)])
def test_options_parity(pkg, opt):
    prob = gen.small_problem(110, 90, 1200, dtype=np.float32, k=6, noise=0.2, correlated=True)
    ratios = oracle.lambda_ratios(12, 2.0)
    g = run_gpu(pkg, prob, ratios, gap_tol_rel=1e-8, **opt)
    o = run_orc(prob, ratios, gap_tol_rel=1e-8, **opt)
    assert_parity(g, o)


@pytest.mark.parametrize("seed,n,p,dtype,corr,opt", [
    (121, 77, 1537, np.float32, True, {}),
    (122, 37, 300, np.float64, False, {}),
    (123, 500, 2500, np.float32, True, {}),
    (124, 130, 3000, np.float32, True, dict(dual_point=1)),
    (125, 90, 1200, np.float32, True, dict(xtr_scope=1, screen_period=3)),
])
def test_dome_parity(pkg, seed, n, p, dtype, corr, opt):
    """GAP SAFE dome (Eq. (11), screen_rule = 1): masks, supports, pass and
    check counts, objectives and coefficients equal the oracle's run with the
    same rule, alone and with the other options."""
    prob = gen.small_problem(seed, n, p, dtype=dtype, k=max(2, min(n, p) // 20), noise=0.2, correlated=corr)
    ratios = oracle.lambda_ratios(14, 2.0)
    g = run_gpu(pkg, prob, ratios, gap_tol_rel=1e-9, screen_rule=1, **opt)
    o = run_orc(prob, ratios, gap_tol_rel=1e-9, screen_rule=1, **opt)
    assert_parity(g, o)


def test_dome_workload2_prefix(pkg):
    """The dome on the Toeplitz 500 x 50000 FP32 path in the benchmark's launch
    configuration: the first 20 lambdas match the oracle element by element."""
    w = gen.workload2()
    ratios = oracle.lambda_ratios(w["T"], w["delta"])[:20]
    g = run_gpu(pkg, w, ratios, screen_period=w["f"], gap_tol_rel=w["tol"], screen_rule=1)
    o = run_orc(w, ratios, screen_period=w["f"], gap_tol_rel=w["tol"], screen_rule=1)
    assert_parity(g, o)


@pytest.mark.parametrize("opt", [dict(refined_radius=1), dict(refined_radius=1, screen_rule=1)])
def test_refined_radius_parity(pkg, opt):
    """Thm. 2's radius (refined_radius = 1) from a poor start: P(beta0) is far
    above P(0) at every lambda and warm starts are off, so the first check of
    each lambda uses R = ||theta - y/lambda||, several times smaller than
    sqrt(2 gap)/lambda there."""
    prob = gen.small_problem(126, 80, 900, dtype=np.float64, k=4, noise=0.2)
    rng = np.random.default_rng(126)
    beta0 = 2.0 * rng.standard_normal(900) * (rng.random(900) < 0.05)
    ratios = oracle.lambda_ratios(8, 1.5)[1:]
    g = run_gpu(pkg, prob, ratios, beta0=beta0, warm_start=0, gap_tol_rel=1e-9, **opt)
    o = run_orc(prob, ratios, beta0=beta0, warm_start=0, gap_tol_rel=1e-9, **opt)
    assert_parity(g, o)


@pytest.mark.parametrize("seed,n,p,a,opt", [
    (131, 77, 1537, 0.5, {}),       # one-warp chain
    (132, 500, 1200, 0.8, {}),      # four chain warps, one granule per lane
    (133, 611, 900, 0.3, {}),       # two granules per lane
    (134, 1100, 1300, 0.6, {}),     # four granules per lane
    (135, 90, 1200, 0.5, dict(dual_point=1, xtr_scope=1, refined_radius=1)),
])
def test_enet_parity(pkg, seed, n, p, a, opt):
    """Elastic-Net (enet_alpha = a, the paper's appendix): the GPU keeps the
    augmented rows implicit, the oracle builds [X; sqrt((1 - a) lambda) I] at
    every lambda; masks, supports, pass and check counts, objectives and
    coefficients agree."""
    prob = gen.small_problem(seed, n, p, dtype=np.float32, k=max(2, min(n, p) // 20), noise=0.2, correlated=True)
    ratios = oracle.lambda_ratios(12, 2.0)
    g = run_gpu(pkg, prob, ratios, gap_tol_rel=1e-9, enet_alpha=a, **opt)
    o = run_orc(prob, ratios, gap_tol_rel=1e-9, enet_alpha=a, **opt)
    assert_parity(g, o)


@pytest.mark.parametrize("seed,n,p,dtype,a,opt", [
    (141, 90, 1100, np.float32, 0.5, dict(screen_rule=1)),          # the dome of the augmented problem
    (142, 400, 2500, np.float32, 0.7, dict(screen_rule=1, refined_radius=1)),
    (143, 64, 800, np.float64, 0.5, {}),                             # an FP64 design (two planes)
    (144, 300, 1500, np.float64, 0.3, dict(screen_rule=1)),
])
def test_enet_dome_and_fp64(pkg, seed, n, p, dtype, a, opt):
    """The Elastic-Net with the GAP SAFE dome (Eq. (11) on the augmented
    problem) and on FP64 designs, against the oracle, which forms the
    augmented design explicitly."""
    prob = gen.small_problem(seed, n, p, dtype=dtype, k=max(2, min(n, p) // 20), noise=0.2, correlated=True)
    ratios = oracle.lambda_ratios(12, 2.0)
    g = run_gpu(pkg, prob, ratios, gap_tol_rel=1e-9, enet_alpha=a, **opt)
    o = run_orc(prob, ratios, gap_tol_rel=1e-9, enet_alpha=a, **opt)
    assert_parity(g, o)


def test_enet_from_a_starting_point(pkg):
    """The Elastic-Net from an outside beta0 with warm starts off (every
    lambda restarts from it; the grid starts below lambda_max)."""
    prob = gen.small_problem(136, 80, 900, dtype=np.float32, k=4, noise=0.2)
    rng = np.random.default_rng(136)
    beta0 = 0.5 * rng.standard_normal(900) * (rng.random(900) < 0.03)
    ratios = oracle.lambda_ratios(8, 1.5)[1:]
    g = run_gpu(pkg, prob, ratios, beta0=beta0, warm_start=0, gap_tol_rel=1e-9, enet_alpha=0.4)
    o = run_orc(prob, ratios, beta0=beta0, warm_start=0, gap_tol_rel=1e-9, enet_alpha=0.4)
    assert_parity(g, o)


def test_beta0_and_screened_nonzero(pkg):
    """A warm start with nonzero coefficients on inactive features exercises
    the removal of screened nonzero coefficients (Remark 3)."""
    prob = gen.small_problem(111, 60, 800, dtype=np.float64, k=4, noise=0.2)
    rng = np.random.default_rng(111)
    beta0 = np.zeros(800)
    beta0[rng.choice(800, 40, replace=False)] = 1e-3 * rng.standard_normal(40)
    ratios = np.array([0.5, 0.3, 0.2])
    g = run_gpu(pkg, prob, ratios, beta0=beta0, gap_tol_rel=1e-10)
    o = run_orc(prob, ratios, beta0=beta0, gap_tol_rel=1e-10)
    assert_parity(g, o)


def test_not_converged_status(pkg):
    prob = gen.small_problem(112, 50, 600, dtype=np.float32, k=10, noise=0.1)
    ratios = oracle.lambda_ratios(6, 3.0)
    g = run_gpu(pkg, prob, ratios, gap_tol_rel=1e-12, max_epochs=3)
    o = run_orc(prob, ratios, gap_tol_rel=1e-12, max_epochs=3)
    assert (g["stats"]["status"] == 5).any()
    assert_parity(g, o)


def test_tiny_and_degenerate(pkg):
    # n = 1, p = 1; p < 32; an all-zero column (screened, never updated)
    for seed, n, p in [(113, 1, 1), (114, 3, 5), (115, 9, 31), (116, 16, 33)]:
        prob = gen.small_problem(seed, n, p, dtype=np.float64, k=1, noise=0.1)
        ratios = oracle.lambda_ratios(5, 1.0)
        assert_parity(run_gpu(pkg, prob, ratios, gap_tol_rel=1e-10), run_orc(prob, ratios, gap_tol_rel=1e-10))
    prob = gen.small_problem(117, 20, 70, dtype=np.float32, k=3, noise=0.1)
    prob["XT"][5] = 0.0
    ratios = oracle.lambda_ratios(6, 1.5)
    g = run_gpu(pkg, prob, ratios, gap_tol_rel=1e-10)
    assert_parity(g, run_orc(prob, ratios, gap_tol_rel=1e-10))
    assert np.all(g["beta"][:, 5] == 0)


def test_repeatable_with_empty_slices(pkg):
    """p = 3000 over the full grid leaves most CTAs without features (32-wide
    slices) and a ragged last mask word; three solves on fresh workspaces
    give bit-identical coefficients, masks and statistics, and the screening
    frequency 1 compares every pass with the oracle."""
    prob = gen.small_problem(103, 130, 3000, dtype=np.float32, k=6, noise=0.2, correlated=True)
    ratios = oracle.lambda_ratios(16, 2.0)[:5]
    opt = dict(gap_tol_rel=1e-9, screen_period=1)
    runs = [run_gpu(pkg, prob, ratios, **opt) for _ in range(3)]
    for r in runs[1:]:
        np.testing.assert_array_equal(r["beta"], runs[0]["beta"])
        np.testing.assert_array_equal(r["mask"], runs[0]["mask"])
        np.testing.assert_array_equal(r["stats"], runs[0]["stats"])
    assert_parity(runs[0], run_orc(prob, ratios, **opt))


def test_nonfinite_input_reported(pkg):
    prob = gen.small_problem(118, 20, 40, dtype=np.float32, k=2)
    prob["XT"][3, 4] = np.nan
    g = run_gpu(pkg, prob, oracle.lambda_ratios(3, 1.0))
    assert np.all(g["stats"]["status"] == pkg.LASSO_ERR_NONFINITE)


def test_workload2_full_size_prefix(pkg):
    """Toeplitz 500 x 50000 FP32 at full size: the first 40 lambdas of the
    100-point grid (the oracle finishes them in seconds) match element by
    element; the launch configuration is the benchmark's."""
    w = gen.workload2()
    ratios = oracle.lambda_ratios(w["T"], w["delta"])[:40]
    g = run_gpu(pkg, w, ratios, screen_period=w["f"], gap_tol_rel=w["tol"])
    o = run_orc(w, ratios, screen_period=w["f"], gap_tol_rel=w["tol"])
    assert_parity(g, o)


@pytest.mark.parametrize("n,p,dtype", [(77, 1537, np.float32), (130, 3000, np.float32), (37, 300, np.float64),
                                       (501, 2000, np.float32)])
def test_workspace_contents_do_not_matter(pkg, n, p, dtype):
    """The workspace is the caller's uninitialised memory: filled with NaN bit
    patterns before the call, it must give the oracle's path (rows past n, the
    padding of the residual's planes, included)."""
    prob = gen.small_problem(700 + n, n, p, dtype=dtype, k=max(2, min(n, p) // 20), noise=0.2)
    ratios = oracle.lambda_ratios(12, 2.0)
    opt = dict(gap_tol_rel=1e-9)
    dev = torch.device("cuda:0")
    xt = pkg.LASSO_F32 if dtype == np.float32 else pkg.LASSO_F64
    need = pkg.lasso_path_workspace_size(n, p, xt, pkg.lasso_default_opts(**opt))
    ws = torch.full((need,), 0xFF, dtype=torch.uint8, device=dev)
    XT = torch.from_numpy(prob["XT"]).to(dev)
    y = torch.from_numpy(prob["y"]).to(dev)
    r = torch.from_numpy(np.ascontiguousarray(ratios)).to(dev)
    out = pkg.solve_path(XT, y, r, n=n, opts=pkg.lasso_default_opts(**opt), workspace=ws)
    torch.cuda.synchronize()
    g = dict(beta=out["beta"].cpu().numpy(), mask=out["mask"].cpu().numpy().view(np.uint32),
             stats=pkg.stats_to_numpy(out["stats"]))
    assert_parity(g, run_orc(prob, ratios, **opt))
