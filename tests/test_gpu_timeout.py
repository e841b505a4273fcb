"""The bounded waits of the path kernel (the GPU's counterpart of Algorithm
1's pass cap K: a launch never runs unbounded).  Every grid-barrier wait gives
up after a time limit, records LASSO_ERR_TIMEOUT and unwinds.  The limit is
20 s; the library reads a shorter one from LASSOGS_WAIT_LIMIT_NS, which these
tests set so that the waits of the CTAs that idle at the grid barrier while
CTA 0 runs a coordinate chain run out.  Nothing faults: the kernel returns,
its records carry the status, and the next call on the same context runs
normally."""
import time

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


def _run(pkg, prob, ratios, **opt):
    dev = torch.device("cuda:0")
    XT = torch.from_numpy(prob["XT"]).to(dev)
    y = torch.from_numpy(prob["y"]).to(dev)
    r = torch.from_numpy(np.ascontiguousarray(ratios)).to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = pkg.solve_path(XT, y, r, n=prob["n"], opts=pkg.lasso_default_opts(**opt))
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return out, pkg.stats_to_numpy(out["stats"]), dt


def test_grid_barrier_wait_runs_out(pkg, monkeypatch):
    # long coordinate chains: a correlated design whose supports reach a few
    # hundred features on the lower part of the grid
    prob = gen.small_problem(511, 400, 6000, dtype=np.float32, k=80, noise=0.05, correlated=True)
    ratios = oracle.lambda_ratios(40, 3.0)
    monkeypatch.setenv("LASSOGS_WAIT_LIMIT_NS", "2000")
    _, st, dt = _run(pkg, prob, ratios)
    assert np.all(st["status"] == pkg.LASSO_ERR_TIMEOUT), st["status"]
    assert np.all(st["converged"] == 0)
    assert dt < 10.0, dt  # the launch unwinds instead of running the path
    # the context is intact: the same call with the default limit succeeds
    # and matches the oracle
    monkeypatch.delenv("LASSOGS_WAIT_LIMIT_NS")
    out, st2, _ = _run(pkg, prob, ratios[:12])
    assert np.all(st2["status"] == 0), st2["status"]
    o = oracle.lasso_path(prob["XT"], prob["y"], ratios[:12], n=prob["n"])
    np.testing.assert_array_equal(st2["epochs"], o["stats"]["epochs"].astype(np.int64))
    np.testing.assert_allclose(st2["primal"], o["stats"]["primal"], rtol=1e-9)
    np.testing.assert_array_equal(out["beta"].cpu().numpy() != 0, o["beta"] != 0)


def test_wait_limit_variable_is_validated(pkg, monkeypatch):
    """Values below 1000 ns or not numbers fall back to the 20 s limit."""
    prob = gen.small_problem(512, 60, 400, dtype=np.float32, k=5, noise=0.1)
    ratios = oracle.lambda_ratios(6, 2.0)
    for v in ("10", "abc", ""):
        monkeypatch.setenv("LASSOGS_WAIT_LIMIT_NS", v)
        _, st, _ = _run(pkg, prob, ratios)
        assert np.all(st["status"] == 0), (v, st["status"])
