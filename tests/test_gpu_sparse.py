"""The sparse CSC variant of the solver (Sec. 4.1: the implementation runs on
a dense or a sparse compressed-column design) against the FP64 oracle on the
same matrix stored densely: masks, supports, pass and check counts,
objectives to 1e-9 relative and coefficients to 1e-5, with every option."""
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


def run_csc(pkg, prob, ratios, beta0=None, **opt):
    dev = torch.device("cuda:0")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    out = pkg.solve_path_csc(t(prob["colptr"]), t(prob["rowidx"]), t(prob["values"]), t(prob["y"]),
                             t(np.asarray(ratios, dtype=np.float64)), prob["n"],
                             beta0=None if beta0 is None else t(np.asarray(beta0, dtype=np.float64)),
                             opts=pkg.lasso_default_opts(**opt))
    torch.cuda.synchronize()
    return dict(beta=out["beta"].cpu().numpy(), mask=out["mask"].cpu().numpy().view(np.uint32),
                stats=pkg.stats_to_numpy(out["stats"]))


CASES = [
    # (seed, n, p, density, options)
    (901, 80, 600, 0.10, {}),
    (902, 300, 3000, 0.03, {}),
    (903, 1000, 2000, 0.02, {}),
    (904, 2500, 800, 0.04, {}),                                      # more rows than the dense path takes
    (905, 150, 1500, 0.05, dict(screen_rule=1)),                     # the dome
    (906, 200, 1200, 0.05, dict(enet_alpha=0.6)),                    # the Elastic-Net
    (907, 120, 900, 0.08, dict(enet_alpha=0.5, screen_rule=1)),
    (908, 160, 1400, 0.05, dict(dual_point=1, xtr_scope=1, refined_radius=1)),
    (909, 64, 500, 0.12, dict(screen_period=1)),
]


@pytest.mark.parametrize("seed,n,p,d,opt", CASES)
def test_csc_parity(pkg, seed, n, p, d, opt):
    prob = gen.sparse_problem(seed, n, p, density=d, k=max(2, min(n, p) // 20), noise=0.2, empty_cols=3)
    ratios = oracle.lambda_ratios(12, 2.0)
    g = run_csc(pkg, prob, ratios, gap_tol_rel=1e-9, **opt)
    o = oracle.lasso_path(prob["XT"], prob["y"], ratios, n=n, gap_tol_rel=1e-9, **opt)
    assert_parity(g, o)


def test_csc_from_a_starting_point(pkg):
    """An outside beta0 with every lambda restarting from it (the grid starts
    below lambda_max)."""
    prob = gen.sparse_problem(910, 100, 800, density=0.06, k=5, noise=0.2)
    rng = np.random.default_rng(910)
    beta0 = 0.5 * rng.standard_normal(800) * (rng.random(800) < 0.03)
    ratios = oracle.lambda_ratios(8, 1.5)[1:]
    g = run_csc(pkg, prob, ratios, beta0=beta0, warm_start=0, gap_tol_rel=1e-9)
    o = oracle.lasso_path(prob["XT"], prob["y"], ratios, beta0=beta0, n=100, warm_start=0, gap_tol_rel=1e-9)
    assert_parity(g, o)


def test_csc_bad_row_index_is_reported(pkg):
    """A row index out of range is found on the device: every record gets
    LASSO_ERR_INVALID_ARG and nothing is read out of bounds."""
    prob = gen.sparse_problem(911, 50, 200, density=0.1)
    prob["rowidx"] = prob["rowidx"].copy()
    prob["rowidx"][7] = 50
    g = run_csc(pkg, prob, oracle.lambda_ratios(4, 1.0))
    assert np.all(g["stats"]["status"] == pkg.LASSO_ERR_INVALID_ARG)
