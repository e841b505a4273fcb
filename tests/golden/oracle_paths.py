"""Stored oracle results for the full benchmark workloads.

The FP64 oracle needs minutes for a whole 100-lambda path at 500 x 50000 and
over an hour of CPU for the 256-problem batch, too long to run inside a GPU
test.  This script runs it once (calling only ``oracle``) and writes what the
GPU path must reproduce into compressed ``.npz`` files beside it:

* ``workload2_sphere.npz`` / ``workload2_dome.npz`` -- the Toeplitz
  500 x 50000 path, all 100 lambdas of the grid to lambda_max/1000 (Sec. 3.3,
  Algorithm 1), with the GAP SAFE sphere (Eq. (10)) or sphere and dome
  (Eq. (11));
* ``workload3_batch.npz`` -- the 256 row-subset problems of the stability
  selection workload over their 50 lambdas.

Per (problem, lambda) the files hold the pass and check counts, |A|, the
number of nonzeros, the primal value, the gap, the support (ascending
indices with their coefficients rounded to FP32, well inside the 1e-5
coefficient tolerance) and a digest of the safe-active mask words.  The
inputs are fingerprinted so that a test run on another machine first checks
that it regenerated the same seeded arrays (``gen`` avoids BLAS for that).

Usage: ``python tests/golden/oracle_paths.py [workload2_sphere|workload2_dome|workload3_batch ...] [--jobs N]``
"""
from __future__ import annotations

import argparse
import hashlib
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# problems of the 256-problem batch whose coefficients are stored (the others
# keep counts, objectives and digests of their supports and masks)
W3_VALUES = tuple(int(b) for b in np.linspace(0, 255, 16).astype(int))


def fingerprint(a) -> str:
    """sha256 of an array's bytes (C order)."""
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def digest64(words) -> np.uint64:
    """First 8 bytes of the sha256 of uint32 words (little endian)."""
    b = np.ascontiguousarray(words, dtype="<u4").tobytes()
    return np.frombuffer(hashlib.sha256(b).digest()[:8], dtype="<u8")[0]


def support_digest(beta_row) -> np.uint64:
    """Digest of the support and the signs of one coefficient vector."""
    nz = np.flatnonzero(beta_row).astype("<u4")
    sg = (beta_row[nz] > 0).astype("<u4")
    return digest64(np.concatenate([nz, sg]))


def pack_paths(beta, mask, stats, keep_values=True):
    """beta (T, p), mask (T, words), stats dict of (T,) arrays -> arrays."""
    T = beta.shape[0]
    out = {
        "epochs": stats["epochs"].astype(np.int64), "checks": stats["checks"].astype(np.int64),
        "n_active": stats["n_active"].astype(np.int64), "n_nonzero": stats["n_nonzero"].astype(np.int64),
        "converged": stats["converged"].astype(np.int8), "primal": stats["primal"].astype(np.float64),
        "dual": stats["dual"].astype(np.float64), "gap": stats["gap"].astype(np.float64),
        "lambda": stats["lambda"].astype(np.float64),
        "mask_digest": np.array([digest64(mask[t]) for t in range(T)], dtype=np.uint64),
        "support_digest": np.array([support_digest(beta[t]) for t in range(T)], dtype=np.uint64),
    }
    if keep_values:
        idx, val, ptr = [], [], [0]
        for t in range(T):
            nz = np.flatnonzero(beta[t])
            idx.append(nz.astype(np.int32))
            val.append(beta[t, nz].astype(np.float32))
            ptr.append(ptr[-1] + nz.size)
        out["sup_idx"] = np.concatenate(idx) if idx else np.zeros(0, np.int32)
        out["sup_val"] = np.concatenate(val) if val else np.zeros(0, np.float32)
        out["sup_ptr"] = np.asarray(ptr, dtype=np.int64)
    return out


def _w2(screen_rule):
    import gen
    import oracle
    w = gen.workload2()
    ratios = oracle.lambda_ratios(w["T"], w["delta"])
    t0 = time.time()
    o = oracle.lasso_path(w["XT"], w["y"], ratios, n=w["n"], screen_period=w["f"], gap_tol_rel=w["tol"],
                          screen_rule=screen_rule)
    out = pack_paths(o["beta"], o["mask"], o["stats"])
    out.update(x_sha256=np.array(fingerprint(w["XT"])), y_sha256=np.array(fingerprint(w["y"])),
               ratios=ratios, oracle_seconds=np.array(time.time() - t0))
    return out


def _w3_problem(b):
    import gen
    import oracle
    w = gen.workload3()
    ratios = oracle.lambda_ratios(w["T"], w["delta"])
    o = oracle.lasso_batch(w["XT"], w["Y"][b:b + 1], ratios, row_mask=w["row_mask"][b:b + 1], n=w["n"],
                           screen_period=w["f"], gap_tol_rel=w["tol"])
    st = {k: v[0] for k, v in o["stats"].items()}
    return b, pack_paths(o["beta"][0], o["mask"][0], st, keep_values=b in W3_VALUES)


def make_workload3(jobs):
    import gen
    import oracle
    w = gen.workload3()
    B = w["Y"].shape[0]
    t0 = time.time()
    with mp.get_context("spawn").Pool(jobs) as pool:
        res = dict(pool.imap_unordered(_w3_problem, range(B)))
    out = {}
    for key in ("epochs", "checks", "n_active", "n_nonzero", "converged", "primal", "dual", "gap", "lambda",
                "mask_digest", "support_digest"):
        out[key] = np.stack([res[b][key] for b in range(B)])
    for b in W3_VALUES:
        for key in ("sup_idx", "sup_val", "sup_ptr"):
            out[f"{key}_{b}"] = res[b][key]
    out.update(x_sha256=np.array(fingerprint(w["XT"])), y_sha256=np.array(fingerprint(w["Y"])),
               row_mask_sha256=np.array(fingerprint(w["row_mask"])),
               ratios=oracle.lambda_ratios(w["T"], w["delta"]), values_for=np.array(W3_VALUES),
               oracle_seconds=np.array(time.time() - t0))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("which", nargs="*", default=["workload2_sphere", "workload2_dome", "workload3_batch"])
    ap.add_argument("--jobs", type=int, default=max(1, (os.cpu_count() or 2) - 2))
    args = ap.parse_args()
    for name in args.which:
        if name == "workload2_sphere":
            out = _w2(0)
        elif name == "workload2_dome":
            out = _w2(1)
        elif name == "workload3_batch":
            out = make_workload3(args.jobs)
        else:
            raise SystemExit(f"unknown golden {name}")
        path = os.path.join(HERE, name + ".npz")
        np.savez_compressed(path, **out)
        print(f"{path}: {os.path.getsize(path)} bytes, oracle {float(out['oracle_seconds']):.1f} s", flush=True)


if __name__ == "__main__":
    main()
