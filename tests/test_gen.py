"""The seeded input generators match the recipes the workloads are stated
with: shapes, storage layout, column normalisation, the Toeplitz correlation,
the sparsity of beta*, the noise level, the row subsets, and determinism."""
import numpy as np
import pytest

import gen


def _cols(w):
    return w["XT"][:, :w["n"]].astype(np.float64)


def test_workload1_recipe():
    w = gen.workload1()
    X = _cols(w)
    assert X.shape == (1000, 100) and w["XT"].dtype == np.float64
    np.testing.assert_allclose(X.mean(axis=1), 0.0, atol=1e-15)
    np.testing.assert_allclose(np.linalg.norm(X, axis=1), 1.0, rtol=1e-14)
    b = w["beta_star"]
    assert np.count_nonzero(b) == 10 and set(np.unique(b[b != 0])) <= {-1.0, 1.0}
    assert (w["T"], w["delta"], w["f"], w["tol"]) == (100, 3.0, 10, 1e-6)
    noise = w["y"] - X.T @ b
    assert 0.05 < noise.std() < 0.15  # y = X beta* + 0.1 N(0, 1)
    w2 = gen.workload1()
    np.testing.assert_array_equal(w["XT"], w2["XT"])
    np.testing.assert_array_equal(w["y"], w2["y"])


def test_workload2_recipe_on_a_slice():
    """The Toeplitz design (here 500 x 4000 of the 50000 columns' recipe):
    unit-norm FP32 columns, neighbouring columns correlated 0.5 and 0.25 two
    apart; beta* 50-sparse; noise sigma = ||X beta*|| / (5 sqrt(n))."""
    w = gen.workload2(n=500, p=4000)
    X = _cols(w)
    assert w["XT"].dtype == np.float32 and w["XT"].shape == (4000, 500)
    np.testing.assert_allclose(np.linalg.norm(X, axis=1), 1.0, rtol=1e-6)
    c1 = np.mean(np.sum(X[1:] * X[:-1], axis=1))
    c2 = np.mean(np.sum(X[2:] * X[:-2], axis=1))
    assert abs(c1 - 0.5) < 0.02 and abs(c2 - 0.25) < 0.02
    b = w["beta_star"]
    assert np.count_nonzero(b) == 50
    signal = X.T @ b
    sigma = np.linalg.norm(signal) / (5.0 * np.sqrt(500))
    assert 0.85 < np.std(w["y"] - signal) / sigma < 1.15
    assert (w["T"], w["delta"], w["f"]) == (100, 3.0, 10)


def test_workload3_recipe_on_a_slice():
    """Row subsets of size U{400..1000}, responses zero outside them, one
    shared 30-sparse beta*, T = 50 and delta = 2."""
    w = gen.workload3(n=1000, p=600, B=24)
    m = w["row_mask"].sum(axis=1)
    assert np.all((m >= 400) & (m <= 1000))
    assert np.all(w["Y"][w["row_mask"] == 0] == 0.0)
    assert np.count_nonzero(w["beta_star"]) == 30
    assert (w["T"], w["delta"]) == (50, 2.0)
    np.testing.assert_allclose(np.linalg.norm(_cols(w), axis=1), 1.0, rtol=1e-6)


def test_workload4_sampler_is_seeded():
    w = gen.workload4(n=60, p=500)
    a, b = w["sample"](5, 1), w["sample"](5, 1)
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, w["sample"](5, 2))
    assert a.shape == (5, 60) and w["lambda_ratio"] == 1.0 / 20.0


@pytest.mark.parametrize("n,p,dtype", [(37, 300, np.float64), (130, 77, np.float32)])
def test_small_problem_layout(n, p, dtype):
    """Column-major storage with leading dimension a multiple of 4 and zero
    padding rows."""
    w = gen.small_problem(3, n, p, dtype=dtype)
    assert w["XT"].shape == (p, w["ldx"]) and w["ldx"] % 4 == 0 and w["ldx"] >= n
    assert np.all(w["XT"][:, n:] == 0)
    assert w["XT"].flags["C_CONTIGUOUS"] and w["XT"].dtype == dtype


@pytest.mark.parametrize("name", ["workload2_sphere", "workload3_batch"])
def test_workloads_match_the_stored_fingerprints(name):
    """The full-size workloads regenerate to the bytes the stored oracle
    results were computed from (the GPU tests compare against those)."""
    import os
    from tests.golden.oracle_paths import fingerprint
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name + ".npz")
    if not os.path.exists(path):
        pytest.skip(f"{path} not written yet")
    gold = np.load(path)
    w = gen.workload2() if name.startswith("workload2") else gen.workload3()
    assert fingerprint(w["XT"]) == str(gold["x_sha256"])
    assert fingerprint(w["y" if "y" in w else "Y"]) == str(gold["y_sha256"])
