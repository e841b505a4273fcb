"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds input generation only: designs X, responses y, row
subsets and noise, drawn with numpy's PCG64 generator.  It contains none of
the method's arithmetic (no lambda_max, no grid, no screening).

Storage convention: a design is returned column-major as a C-contiguous
array ``XT`` of shape (p, ldx); column j is ``XT[j, :n]`` and rows n..ldx-1
are zero padding, so ``XT`` is exactly the column-major block with leading
dimension ``ldx`` that the library and the oracle take.

The five workloads mirror the shapes of the paper's experiments (dense p >> n
designs, a 100-point geometric grid from lambda_max to lambda_max/1000, a
check every f = 10 passes, Sec. 4) -- the paper's own datasets (Leukemia,
20newsgroups, RCV1) are not used; these synthetic designs stand in for them.
"""
from __future__ import annotations

import numpy as np

__all__ = ["round_up", "gaussian_design", "toeplitz_design", "sparse_truth", "WORKLOADS",
           "workload1", "workload2", "workload3", "workload4", "workload5", "small_problem", "sparse_problem"]


def round_up(n, m):
    return (n + m - 1) // m * m


def _finish(cols, n, ldx, dtype, center):
    """cols: (p, n) float64 columns -> centered (optional), unit-norm,
    stored in the requested dtype and padded to ldx."""
    if center:
        cols = cols - cols.mean(axis=1, keepdims=True)
    nrm = np.sqrt((cols * cols).sum(axis=1, keepdims=True))
    nrm[nrm == 0] = 1.0
    cols = cols / nrm
    p = cols.shape[0]
    XT = np.zeros((p, ldx), dtype=dtype)
    XT[:, :n] = cols.astype(dtype)
    return XT


def gaussian_design(rng, n, p, dtype=np.float32, center=False, ldx=None):
    """i.i.d. N(0,1) design with unit-norm columns (optionally centered)."""
    ldx = ldx or round_up(n, 4)
    cols = rng.standard_normal((p, n))
    return _finish(cols, n, ldx, dtype, center)


def toeplitz_design(rng, n, p, corr=0.5, dtype=np.float32, ldx=None):
    """Columns with corr(x_j, x_k) = corr^|j-k| (AR(1) along the feature
    index: x_j = corr x_{j-1} + sqrt(1-corr^2) z_j), then unit-norm."""
    ldx = ldx or round_up(n, 4)
    cols = np.empty((p, n))
    cols[0] = rng.standard_normal(n)
    s = np.sqrt(1.0 - corr * corr)
    for j in range(1, p):
        cols[j] = corr * cols[j - 1] + s * rng.standard_normal(n)
    return _finish(cols, n, ldx, dtype, center=False)


def sparse_truth(rng, p, k, kind="normal"):
    beta = np.zeros(p)
    pos = rng.choice(p, size=k, replace=False)
    if kind == "sign":
        beta[pos] = rng.choice([-1.0, 1.0], size=k)
    else:
        beta[pos] = rng.standard_normal(k)
    return beta


def _matvec(XT, n, beta):
    """X beta in float64 from the stored (possibly float32) columns, summed
    column by column in ascending order with plain elementwise operations, so
    that the result does not depend on the host's BLAS (the inputs must be
    the same bytes on every machine the tests run on)."""
    acc = np.zeros(n)
    for j in np.nonzero(beta)[0]:
        acc = acc + XT[j, :n].astype(np.float64) * beta[j]
    return acc


def _norm(v):
    """Euclidean norm by numpy's pairwise sum (no BLAS)."""
    return float(np.sqrt(np.sum(v * v)))


def small_problem(seed, n, p, dtype=np.float64, k=None, noise=0.1, ldx=None, center=False,
                  correlated=False):
    """A generic small Gaussian (or Toeplitz) problem for tests."""
    rng = np.random.default_rng(seed)
    XT = (toeplitz_design(rng, n, p, dtype=dtype, ldx=ldx) if correlated
          else gaussian_design(rng, n, p, dtype=dtype, center=center, ldx=ldx))
    k = k if k is not None else max(1, min(p // 10, n // 2))
    bstar = sparse_truth(rng, p, k)
    y = _matvec(XT, n, bstar) + noise * rng.standard_normal(n)
    return dict(XT=XT, n=n, p=p, ldx=XT.shape[1], y=y, beta_star=bstar)


def sparse_problem(seed, n, p, density=0.05, k=None, noise=0.1, empty_cols=0):
    """A sparse design with about density * n * p nonzeros (N(0,1) values at
    uniform positions; every column unit-norm except `empty_cols` all-zero
    columns), y = X beta* + noise.  Returns the dense column-major block XT
    (p, n) float64 and the same matrix in compressed sparse column storage:
    colptr (p+1,) int64, rowidx (nnz,) int32 ascending within each column,
    values (nnz,) float64."""
    rng = np.random.default_rng(seed)
    XT = np.zeros((p, n))
    nz = rng.random((p, n)) < density
    XT[nz] = rng.standard_normal(int(nz.sum()))
    for j in range(p):
        if not XT[j].any():
            XT[j, rng.integers(n)] = 1.0
    if empty_cols:
        XT[rng.choice(p, size=empty_cols, replace=False)] = 0.0
    nrm = np.sqrt((XT * XT).sum(axis=1, keepdims=True))
    nrm[nrm == 0] = 1.0
    XT = XT / nrm
    k = k if k is not None else max(1, min(p // 10, n // 2))
    bstar = sparse_truth(rng, p, k)
    y = _matvec(XT, n, bstar) + noise * rng.standard_normal(n)
    counts = (XT != 0).sum(axis=1)
    colptr = np.zeros(p + 1, dtype=np.int64)
    colptr[1:] = np.cumsum(counts)
    rows = [np.flatnonzero(XT[j]) for j in range(p)]
    rowidx = np.concatenate(rows).astype(np.int32) if p else np.zeros(0, np.int32)
    values = np.concatenate([XT[j, r] for j, r in enumerate(rows)]) if p else np.zeros(0)
    return dict(XT=XT, n=n, p=p, ldx=n, y=y, beta_star=bstar, colptr=colptr, rowidx=rowidx, values=values)


def workload1(seed=1001):
    """Single path, FP64: Gaussian 100 x 1000, columns centered then unit-norm;
    beta* 10-sparse with +-1 at uniform positions; y = X beta* + 0.1 N(0,1);
    T = 100, delta = 3, f = 10, gap <= 1e-6 ||y||^2."""
    rng = np.random.default_rng(seed)
    n, p = 100, 1000
    XT = gaussian_design(rng, n, p, dtype=np.float64, center=True)
    bstar = sparse_truth(rng, p, 10, kind="sign")
    y = _matvec(XT, n, bstar) + 0.1 * rng.standard_normal(n)
    return dict(name="gaussian-100x1000-f64", XT=XT, n=n, p=p, ldx=XT.shape[1], y=y,
                beta_star=bstar, T=100, delta=3.0, f=10, tol=1e-6)


def workload2(seed=1002, n=500, p=50000):
    """Single path at scale, FP32 storage: Toeplitz-correlated design
    (corr 0.5^|i-j|) 500 x 50000, unit-norm columns; beta* 50-sparse N(0,1);
    SNR 5 read as noise sigma = ||X beta*|| / (5 sqrt(n)); T = 100,
    delta = 3, f = 10, gap <= 1e-6 ||y||^2."""
    rng = np.random.default_rng(seed)
    XT = toeplitz_design(rng, n, p, corr=0.5, dtype=np.float32)
    bstar = sparse_truth(rng, p, 50)
    signal = _matvec(XT, n, bstar)
    sigma = _norm(signal) / (5.0 * np.sqrt(n))
    y = signal + sigma * rng.standard_normal(n)
    return dict(name=f"toeplitz-{n}x{p}-f32", XT=XT, n=n, p=p, ldx=XT.shape[1], y=y,
                beta_star=bstar, T=100, delta=3.0, f=10, tol=1e-6)


def workload3(seed=1003, n=1000, p=20000, B=256, k=30):
    """Batched stability selection: Gaussian 1000 x 20000 FP32 unit-norm;
    B = 256 problems, each a uniform random row subset of size U{400..1000};
    beta* 30-sparse N(0,1) shared by all problems; each problem has its own
    noise at SNR 5; T = 50, delta = 2."""
    rng = np.random.default_rng(seed)
    XT = gaussian_design(rng, n, p, dtype=np.float32)
    bstar = sparse_truth(rng, p, k)
    signal = _matvec(XT, n, bstar)
    sigma = _norm(signal) / (5.0 * np.sqrt(n))
    Y = np.empty((B, n))
    row_mask = np.zeros((B, n), dtype=np.uint8)
    for b in range(B):
        m = int(rng.integers(min(400, n), n + 1))
        rows = rng.choice(n, size=m, replace=False)
        row_mask[b, rows] = 1
        Y[b] = (signal + sigma * rng.standard_normal(n)) * row_mask[b]
    return dict(name=f"stability-{n}x{p}-B{B}-f32", XT=XT, n=n, p=p, ldx=XT.shape[1], Y=Y,
                row_mask=row_mask, beta_star=bstar, T=50, delta=2.0, f=10, tol=1e-6)


def workload4(seed=1004, n=300, p=10000, n_train=200000, n_eval=4096, k_range=(5, 50)):
    """Learned warm start on a fixed design: Gaussian 300 x 10000 FP32
    unit-norm; each y from its own beta* with k ~ U{5..50} N(0,1) entries and
    SNR ~ U[2,10].  Returns the design and a response sampler."""
    rng = np.random.default_rng(seed)
    XT = gaussian_design(rng, n, p, dtype=np.float32)

    def sample(count, seed_offset):
        r = np.random.default_rng(seed * 1000 + seed_offset)
        Y = np.empty((count, n))
        for i in range(count):
            k = int(r.integers(k_range[0], k_range[1] + 1))
            bstar = sparse_truth(r, p, k)
            signal = _matvec(XT, n, bstar)
            snr = r.uniform(2.0, 10.0)
            sigma = _norm(signal) / (snr * np.sqrt(n))
            Y[i] = signal + sigma * r.standard_normal(n)
        return Y

    return dict(name=f"learned-start-{n}x{p}-f32", XT=XT, n=n, p=p, ldx=XT.shape[1],
                sample=sample, n_train=n_train, n_eval=n_eval, lambda_ratio=1.0 / 20.0)


def workload5(seed=1005, n=2000, p=100000, B=1024):
    """Full tuned form at large size: Gaussian 2000 x 100000 FP32; B = 1024
    right-hand sides with beta* sparsity k ~ U{10..200}, SNR ~ U[1,10];
    T = 30, delta = 2."""
    rng = np.random.default_rng(seed)
    XT = gaussian_design(rng, n, p, dtype=np.float32)
    Y = np.empty((B, n))
    for b in range(B):
        k = int(rng.integers(10, 201))
        bstar = sparse_truth(rng, p, k)
        signal = _matvec(XT, n, bstar)
        snr = rng.uniform(1.0, 10.0)
        sigma = _norm(signal) / (snr * np.sqrt(n))
        Y[b] = signal + sigma * rng.standard_normal(n)
    return dict(name=f"multi-rhs-{n}x{p}-B{B}-f32", XT=XT, n=n, p=p, ldx=XT.shape[1], Y=Y,
                T=30, delta=2.0, f=10, tol=1e-6)


WORKLOADS = {1: workload1, 2: workload2, 3: workload3, 4: workload4, 5: workload5}
