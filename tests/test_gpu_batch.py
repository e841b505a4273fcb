"""lasso_batch vs the FP64 oracle: B independent paths over one design, each on
its own row subset (stability-selection replicates) or its own response
(multi right-hand side).  Each problem is compared element by element with
the oracle's path on the gathered rows, with the tolerances of the single
path (objective 1e-9 relative, beta 1e-5, supports, masks and pass counts)."""
import numpy as np
import pytest

import gen
import oracle
from tests.test_gpu_path import assert_parity

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


def run_gpu_batch(pkg, XT, n, Y, rmask, ratios, beta0=None, **opt):
    dev = torch.device("cuda:0")
    Xd = torch.from_numpy(np.ascontiguousarray(XT, dtype=np.float32)).to(dev)
    Yd = torch.from_numpy(np.ascontiguousarray(Y, dtype=np.float64)).to(dev)
    Md = None if rmask is None else torch.from_numpy(np.ascontiguousarray(rmask, dtype=np.uint8)).to(dev)
    r = torch.from_numpy(np.ascontiguousarray(ratios, dtype=np.float64)).to(dev)
    b0 = None if beta0 is None else torch.from_numpy(np.ascontiguousarray(beta0, dtype=np.float64)).to(dev)
    if opt.get("gemm_dtype") == PASS:
        opt = dict(opt, gemm_dtype=pkg.LASSO_BF16, lockstep_pass=1)
    out = pkg.solve_batch(Xd, Yd, r, n=n, row_mask=Md, beta0=b0, opts=pkg.lasso_default_opts(**opt))
    torch.cuda.synchronize()
    B, T = Y.shape[0], len(ratios)
    st = pkg.stats_to_numpy(out["stats"]).reshape(B, T)
    return dict(beta=out["beta"].cpu().numpy(), mask=out["mask"].cpu().numpy().view(np.uint32), stats=st)


def check_batch(g, o):
    B = g["beta"].shape[0]
    for b in range(B):
        gb = dict(beta=g["beta"][b], mask=g["mask"][b], stats=g["stats"][b])
        ob = dict(beta=o["beta"][b], mask=o["mask"][b], stats={k: v[b] for k, v in o["stats"].items()})
        assert_parity(gb, ob)


def _subsample_problem(seed, n, p, B, frac_lo=0.4, k=5, correlated=False):
    prob = gen.small_problem(seed, n, p, dtype=np.float32, k=k, noise=0.2, correlated=correlated)
    rng = np.random.default_rng(seed)
    rmask = np.zeros((B, n), dtype=np.uint8)
    Y = np.empty((B, n))
    for b in range(B):
        m = int(rng.integers(max(1, int(frac_lo * n)), n + 1))
        rmask[b, rng.choice(n, size=m, replace=False)] = 1
        Y[b] = prob["y"] + 0.05 * rng.standard_normal(n)
    return prob, Y, rmask


# gemm_dtype 1 (LASSO_F32): every CTA runs whole paths, its checks are FP32
# CUDA-core passes; 2 (LASSO_BF16): lockstep over lambda, the first check of
# every lambda comes from one split-BF16 tensor-core product for all problems;
# PASS: lockstep over coordinate passes (LASSO_BF16 with lockstep_pass = 1),
# a product before every pass serving its check and its certificates
PASS = 3
GEMM = [1, 2, PASS]


@pytest.mark.parametrize("gemm", GEMM)
@pytest.mark.parametrize("seed,n,p,B,corr", [(201, 120, 900, 7, False), (202, 333, 1500, 5, True),
                                             (203, 64, 640, 3, False)])
def test_batch_row_subsets(pkg, seed, n, p, B, corr, gemm):
    prob, Y, rmask = _subsample_problem(seed, n, p, B, correlated=corr)
    ratios = oracle.lambda_ratios(12, 2.0)
    opt = dict(gap_tol_rel=1e-9, xtr_scope=1)
    g = run_gpu_batch(pkg, prob["XT"], n, Y, rmask, ratios, gemm_dtype=gemm, **opt)
    o = oracle.lasso_batch(prob["XT"], Y * rmask, ratios, row_mask=rmask, n=n, **opt)
    check_batch(g, o)


@pytest.mark.parametrize("gemm", GEMM)
def test_batch_multi_rhs_no_mask(pkg, gemm):
    prob = gen.small_problem(204, 90, 1100, dtype=np.float32, k=6)
    rng = np.random.default_rng(204)
    B = 6
    Y = np.stack([prob["y"] * rng.uniform(0.5, 2.0) + 0.3 * rng.standard_normal(90) for _ in range(B)])
    ratios = oracle.lambda_ratios(10, 2.0)
    g = run_gpu_batch(pkg, prob["XT"], 90, Y, None, ratios, gap_tol_rel=1e-9, gemm_dtype=gemm)
    o = oracle.lasso_batch(prob["XT"], Y, ratios, n=90, gap_tol_rel=1e-9)
    check_batch(g, o)


@pytest.mark.parametrize("gemm", GEMM)
def test_batch_more_problems_than_resident_ctas(pkg, gemm):
    """B larger than the number of resident CTAs: the queue hands out every
    problem exactly once."""
    prob, Y, rmask = _subsample_problem(205, 40, 200, 500, k=3)
    ratios = oracle.lambda_ratios(5, 1.5)
    g = run_gpu_batch(pkg, prob["XT"], 40, Y, rmask, ratios, gap_tol_rel=1e-9, gemm_dtype=gemm)
    pick = [0, 1, 151, 152, 303, 304, 305, 499]
    o = oracle.lasso_batch(prob["XT"], (Y * rmask)[pick], ratios, row_mask=rmask[pick], n=40, gap_tol_rel=1e-9)
    check_batch(dict(beta=g["beta"][pick], mask=g["mask"][pick], stats=g["stats"][pick]), o)
    assert np.all(g["stats"]["status"] == 0)


@pytest.mark.parametrize("gemm", GEMM)
def test_batch_bad_problem_is_isolated(pkg, gemm):
    """A problem with a NaN response reports NONFINITE; the others solve."""
    prob, Y, rmask = _subsample_problem(206, 50, 300, 4)
    Y[2, int(np.nonzero(rmask[2])[0][0])] = np.nan
    ratios = oracle.lambda_ratios(4, 1.0)
    g = run_gpu_batch(pkg, prob["XT"], 50, Y, rmask, ratios, gap_tol_rel=1e-9, gemm_dtype=gemm)
    assert np.all(g["stats"]["status"][2] == pkg.LASSO_ERR_NONFINITE)
    keep = [0, 1, 3]
    o = oracle.lasso_batch(prob["XT"], (Y * rmask)[keep], ratios, row_mask=rmask[keep], n=50, gap_tol_rel=1e-9)
    check_batch(dict(beta=g["beta"][keep], mask=g["mask"][keep], stats=g["stats"][keep]), o)


@pytest.mark.parametrize("gemm", GEMM)
def test_batch_workload3_full_size_prefix(pkg, gemm):
    """Stability-selection workload at full size (Gaussian 1000 x 20000, row
    subsets of U{400..1000}) for 4 problems on the first 15 lambdas of the
    50-point grid to lambda_max/100."""
    w = gen.workload3(B=4)
    ratios = oracle.lambda_ratios(w["T"], w["delta"])[:15]
    opt = dict(gap_tol_rel=w["tol"], xtr_scope=1, screen_period=w["f"])
    g = run_gpu_batch(pkg, w["XT"], w["n"], w["Y"], w["row_mask"], ratios, gemm_dtype=gemm, **opt)
    o = oracle.lasso_batch(w["XT"], w["Y"], ratios, row_mask=w["row_mask"], n=w["n"], **opt)
    check_batch(g, o)


@pytest.mark.parametrize("gemm", GEMM)
@pytest.mark.parametrize("warm", [1, 0])
def test_batch_beta0(pkg, gemm, warm):
    """Per-problem starting points (Sec. 3.3 warm start taken from outside,
    e.g. a learned initialiser): rho = y - X beta0 on the problem's rows;
    with warm_start = 0 every lambda restarts from beta0.  The grid starts
    below lambda_max: there, from a nonzero start, the update of the feature
    attaining lambda_max lands exactly on the soft-threshold boundary and its
    sign of rounding (+-1e-16 or 0) is not a property of the method."""
    prob, Y, rmask = _subsample_problem(207, 150, 1200, 6, correlated=True)
    rng = np.random.default_rng(207)
    beta0 = np.zeros((6, 1200))
    for b in range(6):
        idx = rng.choice(1200, size=int(rng.integers(0, 40)), replace=False)
        beta0[b, idx] = rng.standard_normal(idx.size) * 0.3
    beta0[3] = 0.0  # one problem from zero
    ratios = oracle.lambda_ratios(9, 1.5)[1:]
    opt = dict(gap_tol_rel=1e-9, warm_start=warm)
    g = run_gpu_batch(pkg, prob["XT"], 150, Y, rmask, ratios, beta0=beta0, gemm_dtype=gemm, **opt)
    o = oracle.lasso_batch(prob["XT"], Y * rmask, ratios, row_mask=rmask, n=150, beta0=beta0, **opt)
    check_batch(g, o)


def test_batch_captured_in_cuda_graph(pkg):
    """The lockstep solver allocates nothing and never waits on the host, so
    a whole lasso_batch call (per lambda: residual packing, tensor-core
    product, solver launch) can be captured in a CUDA graph once and replayed
    on new responses; replays equal direct calls."""
    prob, Y, rmask = _subsample_problem(208, 160, 1400, 12, correlated=True)
    ratios = oracle.lambda_ratios(10, 2.0)
    dev = torch.device("cuda:0")
    opts = pkg.lasso_default_opts(gap_tol_rel=1e-9, gemm_dtype=pkg.LASSO_BF16)
    Xd = torch.from_numpy(np.ascontiguousarray(prob["XT"], dtype=np.float32)).to(dev)
    Yd = torch.from_numpy(Y).to(dev)
    Md = torch.from_numpy(rmask).to(dev)
    r = torch.from_numpy(ratios).to(dev)
    B, T, p = Y.shape[0], len(ratios), prob["XT"].shape[0]
    words = (p + 31) // 32
    beta = torch.empty((B, T, p), dtype=torch.float64, device=dev)
    mask = torch.empty((B, T, words), dtype=torch.int32, device=dev)
    stats = torch.empty(B * T * pkg.STATS_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    need = pkg.lasso_batch_workspace_size(160, p, B, opts)
    ws = torch.empty(need, dtype=torch.uint8, device=dev)

    def call(stream):
        pkg.lasso_batch(Xd.data_ptr(), 160, p, Xd.shape[1], Yd.data_ptr(), Yd.shape[1], Md.data_ptr(), Md.shape[1],
                        B, r.data_ptr(), T, None, 0, opts, beta.data_ptr(), mask.data_ptr(), stats.data_ptr(),
                        ws.data_ptr(), need, stream)

    side = torch.cuda.Stream(dev)
    with torch.cuda.stream(side):
        call(side.cuda_stream)  # warm-up outside the capture (lazy module and attribute set-up)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        call(side.cuda_stream)
    results = []
    for k in range(2):
        Yd.copy_(torch.from_numpy(Y * (1.0 + 0.5 * k)))
        g.replay()
        torch.cuda.synchronize()
        gr = dict(beta=beta.cpu().numpy().copy(), mask=mask.cpu().numpy().view(np.uint32).copy(),
                  stats=pkg.stats_to_numpy(stats).reshape(B, T).copy())
        direct = run_gpu_batch(pkg, prob["XT"], 160, Y * (1.0 + 0.5 * k), rmask, ratios, gap_tol_rel=1e-9,
                               gemm_dtype=pkg.LASSO_BF16)
        np.testing.assert_array_equal(gr["beta"], direct["beta"])
        np.testing.assert_array_equal(gr["mask"], direct["mask"])
        np.testing.assert_array_equal(gr["stats"], direct["stats"])
        results.append(gr)
    o = oracle.lasso_batch(prob["XT"], Y * rmask * 1.5, ratios, row_mask=rmask, n=160, gap_tol_rel=1e-9)
    check_batch(results[1], o)


def test_autotuner_picks_a_shape_and_keeps_results(pkg):
    """lasso_batch_tune times its eleven launch shapes and returns the fastest;
    solving with the tuned options gives the masks and pass counts of the
    default shape (every shape makes the FP64 test's decisions) and the same
    coefficients up to rounding (a group of CTAs may run the chain in Gram
    form, which orders the double-float sums differently), and both match
    the oracle."""
    prob, Y, rmask = _subsample_problem(209, 200, 2000, 40, correlated=False)
    ratios = oracle.lambda_ratios(8, 1.5)
    dev = torch.device("cuda:0")
    Xd = torch.from_numpy(np.ascontiguousarray(prob["XT"], dtype=np.float32)).to(dev)
    Yd = torch.from_numpy(Y).to(dev)
    Md = torch.from_numpy(rmask).to(dev)
    r = torch.from_numpy(ratios).to(dev)
    base = pkg.lasso_default_opts(gap_tol_rel=1e-9)
    tuned, times = pkg.tune_batch(Xd, Yd, r, n=200, row_mask=Md, opts=base, sample=16, lambdas=4)
    assert np.all((times > 0) | (times == -1)) and np.any(times > 0)
    k = int(np.argmin(np.where(times > 0, times, np.inf)))
    shapes = [(pkg.LASSO_F32, 2, 0, 1, 0), (pkg.LASSO_F32, 1, 0, 1, 0), (pkg.LASSO_BF16, 2, 128, 1, 0),
              (pkg.LASSO_BF16, 1, 128, 1, 0), (pkg.LASSO_BF16, 2, 256, 1, 0), (pkg.LASSO_BF16, 1, 256, 1, 0),
              (pkg.LASSO_F32, 2, 0, 8, 0), (pkg.LASSO_F32, 2, 0, 32, 0), (pkg.LASSO_F32, 1, 0, 16, 0),
              (pkg.LASSO_BF16, 2, 128, 1, 1), (pkg.LASSO_BF16, 1, 128, 1, 1)]
    assert len(times) == len(shapes)
    assert (tuned.gemm_dtype, tuned.batch_ctas_per_sm, tuned.gemm_tile_n, tuned.batch_group,
            tuned.lockstep_pass) == shapes[k]
    assert tuned.gap_tol_rel == 1e-9
    outs = {}
    for name, o in (("default", base), ("tuned", tuned)):
        out = pkg.solve_batch(Xd, Yd, r, n=200, row_mask=Md, opts=o)
        torch.cuda.synchronize()
        st = pkg.stats_to_numpy(out["stats"]).reshape(40, len(ratios))
        outs[name] = (out["beta"].cpu().numpy(), out["mask"].cpu().numpy(), st)
    np.testing.assert_allclose(outs["default"][0], outs["tuned"][0], rtol=0, atol=1e-10)
    np.testing.assert_array_equal(outs["default"][0] != 0, outs["tuned"][0] != 0)
    np.testing.assert_array_equal(outs["default"][1], outs["tuned"][1])
    np.testing.assert_array_equal(outs["default"][2]["epochs"], outs["tuned"][2]["epochs"])
    pick = [0, 17, 39]
    o = oracle.lasso_batch(prob["XT"], (Y * rmask)[pick], ratios, row_mask=rmask[pick], n=200, gap_tol_rel=1e-9)
    g = dict(beta=outs["tuned"][0][pick], mask=outs["tuned"][1][pick].view(np.uint32), stats=outs["tuned"][2][pick])
    check_batch(g, o)


@pytest.mark.parametrize("per_sm,tile", [(1, 64), (1, 256), (2, 64)])
def test_batch_launch_shapes(pkg, per_sm, tile):
    """One CTA per SM (no register cap) and every tensor-core N tile give the
    oracle's results."""
    prob, Y, rmask = _subsample_problem(210, 333, 1500, 9, correlated=True)
    ratios = oracle.lambda_ratios(10, 2.0)
    opt = dict(gap_tol_rel=1e-9, xtr_scope=1)
    g = run_gpu_batch(pkg, prob["XT"], 333, Y, rmask, ratios, gemm_dtype=pkg.LASSO_BF16, batch_ctas_per_sm=per_sm,
                      gemm_tile_n=tile, **opt)
    o = oracle.lasso_batch(prob["XT"], Y * rmask, ratios, row_mask=rmask, n=333, **opt)
    check_batch(g, o)
    g1 = run_gpu_batch(pkg, prob["XT"], 333, Y, rmask, ratios, gemm_dtype=pkg.LASSO_F32, batch_ctas_per_sm=per_sm,
                       **opt)
    check_batch(g1, o)


@pytest.mark.parametrize("group", [2, 8, 32])
def test_batch_groups_of_ctas(pkg, group):
    """Several CTAs per problem (feature slices and a barrier per group) give
    the oracle's results, with row subsets, starting points and a problem
    whose response holds a NaN."""
    prob, Y, rmask = _subsample_problem(211, 150, 3001, 11, correlated=True)
    rng = np.random.default_rng(211)
    beta0 = np.zeros((11, 3001))
    for b in range(0, 11, 3):
        idx = rng.choice(3001, size=15, replace=False)
        beta0[b, idx] = 0.2 * rng.standard_normal(15)
    Y[5, int(np.nonzero(rmask[5])[0][0])] = np.nan
    ratios = oracle.lambda_ratios(9, 1.5)[1:]
    opt = dict(gap_tol_rel=1e-9, xtr_scope=1)
    g = run_gpu_batch(pkg, prob["XT"], 150, Y, rmask, ratios, beta0=beta0, gemm_dtype=pkg.LASSO_F32,
                      batch_group=group, **opt)
    assert np.all(g["stats"]["status"][5] == pkg.LASSO_ERR_NONFINITE)
    keep = [b for b in range(11) if b != 5]
    o = oracle.lasso_batch(prob["XT"], (Y * rmask)[keep], ratios, row_mask=rmask[keep], n=150, beta0=beta0[keep],
                           **opt)
    check_batch(dict(beta=g["beta"][keep], mask=g["mask"][keep], stats=g["stats"][keep]), o)


@pytest.mark.parametrize("gemm,group", [(1, 1), (2, 1), (1, 8), (PASS, 1)])
def test_batch_dome(pkg, gemm, group):
    """GAP SAFE dome (Eq. (11)) in every batched mode: per-CTA FP32 checks,
    lockstep split-BF16 first checks and groups of CTAs; x_j^T y is taken on
    each problem's own rows."""
    prob, Y, rmask = _subsample_problem(207, 150, 1100, 6, correlated=True)
    ratios = oracle.lambda_ratios(10, 2.0)
    opt = dict(gap_tol_rel=1e-9, screen_rule=1)
    g = run_gpu_batch(pkg, prob["XT"], 150, Y, rmask, ratios, gemm_dtype=gemm, batch_group=group, **opt)
    o = oracle.lasso_batch(prob["XT"], Y * rmask, ratios, row_mask=rmask, n=150, **opt)
    check_batch(g, o)


@pytest.mark.parametrize("gemm,group,a,rule", [(1, 1, 0.5, 0), (2, 1, 0.5, 0), (1, 8, 0.7, 0), (2, 1, 0.6, 1),
                                                (1, 1, 0.4, 1), (PASS, 1, 0.5, 0), (PASS, 1, 0.6, 1)])
def test_batch_enet(pkg, gemm, group, a, rule):
    """The Elastic-Net in every batched mode (per-CTA FP32 checks, lockstep
    split-BF16 first checks, groups of CTAs), with the sphere or the dome:
    each problem is the augmented Lasso on its own rows, with its own
    lambda_max = ||X_b^T y_b||_inf / a."""
    prob, Y, rmask = _subsample_problem(208, 140, 1300, 6, correlated=True)
    ratios = oracle.lambda_ratios(10, 2.0)
    opt = dict(gap_tol_rel=1e-9, enet_alpha=a, screen_rule=rule)
    g = run_gpu_batch(pkg, prob["XT"], 140, Y, rmask, ratios, gemm_dtype=gemm, batch_group=group, **opt)
    o = oracle.lasso_batch(prob["XT"], Y * rmask, ratios, row_mask=rmask, n=140, **opt)
    check_batch(g, o)


@pytest.mark.parametrize("gemm", GEMM)
def test_batch_refined_radius(pkg, gemm):
    """Thm. 2's radius in the batched modes, from poor per-problem starting
    points (warm starts off, grids below lambda_max)."""
    prob, Y, rmask = _subsample_problem(208, 120, 700, 4)
    rng = np.random.default_rng(208)
    beta0 = 2.0 * rng.standard_normal((4, 700)) * (rng.random((4, 700)) < 0.05)
    ratios = oracle.lambda_ratios(7, 1.5)[1:]
    opt = dict(gap_tol_rel=1e-9, refined_radius=1, warm_start=0)
    g = run_gpu_batch(pkg, prob["XT"], 120, Y, rmask, ratios, beta0=beta0, gemm_dtype=gemm, **opt)
    o = oracle.lasso_batch(prob["XT"], Y * rmask, ratios, row_mask=rmask, n=120, beta0=beta0, **opt)
    check_batch(g, o)


@pytest.mark.parametrize("warm,a", [(1, 1.0), (0, 1.0), (1, 0.6)])
def test_batch_pass_tail_on_single_path(pkg, warm, a):
    """Lockstep per pass on a batch without row subsets: once at most 8
    problems are unfinished, each stops at its next lambda boundary and the
    rest of its path runs on the single path.  Every (problem, lambda) still
    equals the oracle: passes, checks, masks, objectives, coefficients; with
    warm starts off the single path restarts every lambda from beta0 too."""
    prob = gen.small_problem(212, 120, 1500, dtype=np.float32, k=8, correlated=True)
    rng = np.random.default_rng(212)
    B = 7
    Y = np.stack([prob["y"] * rng.uniform(0.5, 2.0) + 0.3 * rng.standard_normal(120) for _ in range(B)])
    beta0 = np.zeros((B, 1500))
    for b in range(0, B, 2):
        idx = rng.choice(1500, size=12, replace=False)
        beta0[b, idx] = 0.2 * rng.standard_normal(12)
    ratios = oracle.lambda_ratios(12, 2.0)[1:]
    opt = dict(gap_tol_rel=1e-9, warm_start=warm, enet_alpha=a)
    g = run_gpu_batch(pkg, prob["XT"], 120, Y, None, ratios, beta0=beta0, gemm_dtype=PASS, **opt)
    o = oracle.lasso_batch(prob["XT"], Y, ratios, n=120, beta0=beta0, **opt)
    check_batch(g, o)
