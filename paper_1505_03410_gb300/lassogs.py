"""ctypes binding of liblassogs (include/lassogs.h).

The functions below carry the C names and only marshal arguments: every step
of the solver runs in the CUDA library.  There is no CPU fallback -- if the
library is missing, loading it raises.

``solve_path`` is a convenience wrapper that allocates the outputs and the
workspace as torch CUDA tensors (PyTorch supplies device memory and streams)
and calls ``lasso_path`` on the current stream.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblassogs.so")

LASSO_OK = 0
LASSO_ERR_INVALID_ARG = 1
LASSO_ERR_NONFINITE = 2
LASSO_ERR_WORKSPACE = 3
LASSO_ERR_CUDA = 4
LASSO_ERR_NOT_CONVERGED = 5
LASSO_ERR_TIMEOUT = 6
LASSO_F64, LASSO_F32, LASSO_BF16 = 0, 1, 2

# every symbol include/lassogs.h declares
EXPORTED = ("lasso_default_opts", "lasso_lambda_grid", "lasso_path_workspace_size", "lasso_path",
            "lasso_last_error", "lasso_path_static", "lasso_batch_workspace_size", "lasso_batch",
            "lasso_correlations_bf16", "lasso_correlations_f32", "lasso_batch_tune_candidates",
            "lasso_batch_tune_workspace_size", "lasso_batch_tune", "lasso_path_phase_cycles",
            "lasso_path_csc_workspace_size", "lasso_path_csc")


class LassoError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"lasso status {status}: {msg}")
        self.status = status


class LassoOpts(ctypes.Structure):
    _fields_ = [("screen_period", ctypes.c_int32), ("dual_point", ctypes.c_int32),
                ("xtr_scope", ctypes.c_int32), ("warm_start", ctypes.c_int32),
                ("max_epochs", ctypes.c_int64), ("gap_tol_rel", ctypes.c_double),
                ("gemm_dtype", ctypes.c_int32), ("batch_ctas_per_sm", ctypes.c_int32),
                ("gemm_tile_n", ctypes.c_int32), ("batch_group", ctypes.c_int32),
                ("screen_rule", ctypes.c_int32), ("refined_radius", ctypes.c_int32),
                ("enet_alpha", ctypes.c_double), ("audit_bounds", ctypes.c_int32),
                ("lockstep_pass", ctypes.c_int32)]


class LassoPathStats(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("primal", ctypes.c_double), ("dual", ctypes.c_double),
                ("gap", ctypes.c_double), ("radius", ctypes.c_double), ("alpha", ctypes.c_double),
                ("epochs", ctypes.c_int64), ("checks", ctypes.c_int64), ("n_active", ctypes.c_int64),
                ("n_nonzero", ctypes.c_int64), ("x_columns", ctypes.c_int64), ("converged", ctypes.c_int32),
                ("status", ctypes.c_int32), ("bound_ratio", ctypes.c_double), ("bound_ratio_tc", ctypes.c_double)]


STATS_DTYPE = np.dtype([("lambda", "<f8"), ("primal", "<f8"), ("dual", "<f8"), ("gap", "<f8"),
                        ("radius", "<f8"), ("alpha", "<f8"), ("epochs", "<i8"), ("checks", "<i8"),
                        ("n_active", "<i8"), ("n_nonzero", "<i8"), ("x_columns", "<i8"), ("converged", "<i4"),
                        ("status", "<i4"), ("bound_ratio", "<f8"), ("bound_ratio_tc", "<f8")])
assert STATS_DTYPE.itemsize == ctypes.sizeof(LassoPathStats)

_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load liblassogs.so (built by paper_1505_03410_gb300.build)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"{p} is missing: build it with paper_1505_03410_gb300.build.build()")
            lib = ctypes.CDLL(p)
            V, I32, I64, D, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
            lib.lasso_default_opts.argtypes = [ctypes.POINTER(LassoOpts)]
            lib.lasso_default_opts.restype = None
            lib.lasso_lambda_grid.argtypes = [I32, D, V]
            lib.lasso_lambda_grid.restype = ctypes.c_int
            lib.lasso_path_workspace_size.argtypes = [I64, I64, ctypes.c_int, ctypes.POINTER(LassoOpts)]
            lib.lasso_path_workspace_size.restype = SZ
            lib.lasso_path.argtypes = [V, ctypes.c_int, I64, I64, I64, V, V, I32, V, ctypes.POINTER(LassoOpts),
                                       V, V, V, V, SZ, V]
            lib.lasso_path.restype = ctypes.c_int
            lib.lasso_path_static.argtypes = [V, ctypes.c_int, I64, I64, I64, V, V, I32, V,
                                              ctypes.POINTER(LassoOpts), V, V, V, V]
            lib.lasso_path_static.restype = ctypes.c_int
            lib.lasso_batch_workspace_size.argtypes = [I64, I64, I64, ctypes.POINTER(LassoOpts)]
            lib.lasso_batch_workspace_size.restype = SZ
            lib.lasso_batch.argtypes = [V, I64, I64, I64, V, I64, V, I64, I64, V, I32, V, I64,
                                        ctypes.POINTER(LassoOpts), V, V, V, V, SZ, V]
            lib.lasso_batch.restype = ctypes.c_int
            lib.lasso_correlations_bf16.argtypes = [V, I64, I64, I64, V, I64, I64, V, I64, V, SZ, V]
            lib.lasso_correlations_bf16.restype = ctypes.c_int
            lib.lasso_correlations_f32.argtypes = [V, I64, I64, I64, V, V, V, V]
            lib.lasso_correlations_f32.restype = ctypes.c_int
            lib.lasso_batch_tune_candidates.argtypes = []
            lib.lasso_batch_tune_candidates.restype = I32
            lib.lasso_batch_tune_workspace_size.argtypes = [I64, I64, I64, I32]
            lib.lasso_batch_tune_workspace_size.restype = SZ
            lib.lasso_batch_tune.argtypes = [V, I64, I64, I64, V, I64, V, I64, I64, V, I32, V, I64,
                                             ctypes.POINTER(LassoOpts), I32, I32, ctypes.POINTER(LassoOpts), V, V, SZ,
                                             V]
            lib.lasso_batch_tune.restype = ctypes.c_int
            lib.lasso_path_csc_workspace_size.argtypes = [I64, I64, ctypes.POINTER(LassoOpts)]
            lib.lasso_path_csc_workspace_size.restype = SZ
            lib.lasso_path_csc.argtypes = [V, V, V, I64, I64, V, V, I32, V, ctypes.POINTER(LassoOpts), V, V, V, V, SZ, V]
            lib.lasso_path_csc.restype = ctypes.c_int
            lib.lasso_path_phase_cycles.argtypes = [V, V, V]
            lib.lasso_path_phase_cycles.restype = ctypes.c_int
            lib.lasso_last_error.argtypes = []
            lib.lasso_last_error.restype = ctypes.c_char_p
            _lib = lib
    return _lib


def lasso_last_error() -> str:
    return load().lasso_last_error().decode()


def _check(status):
    if status != LASSO_OK:
        raise LassoError(status, lasso_last_error())
    return status


def lasso_default_opts(**overrides) -> LassoOpts:
    o = LassoOpts()
    load().lasso_default_opts(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def lasso_lambda_grid(T: int, delta: float) -> np.ndarray:
    out = np.empty(int(T), dtype=np.float64)
    _check(load().lasso_lambda_grid(int(T), float(delta), out.ctypes.data_as(ctypes.c_void_p)))
    return out


def lasso_path_workspace_size(n: int, p: int, x_dtype: int, opts: LassoOpts | None = None) -> int:
    return int(load().lasso_path_workspace_size(int(n), int(p), int(x_dtype),
                                                ctypes.byref(opts) if opts is not None else None))


def lasso_path(X, x_dtype, n, p, ldx, y, lambda_ratios, T, beta0, opts, beta_out, mask_out, stats,
               workspace, workspace_bytes, stream) -> int:
    """Direct call of the C entry point; pointer arguments are integers
    (device addresses) or None.  Raises LassoError on a non-zero status."""
    def vp(x):
        return None if x is None or x == 0 else ctypes.c_void_p(int(x))
    return _check(load().lasso_path(vp(X), int(x_dtype), int(n), int(p), int(ldx), vp(y), vp(lambda_ratios),
                                    int(T), vp(beta0), ctypes.byref(opts) if opts is not None else None,
                                    vp(beta_out), vp(mask_out), vp(stats), vp(workspace), int(workspace_bytes),
                                    vp(stream)))


def lasso_path_static(X, x_dtype, n, p, ldx, y, lambda_ratios, T, beta0, opts, beta_out, mask_out, stats,
                      stream) -> int:
    """The workspace-free entry point (scratch in a static 32 MiB device array
    owned by the library): for callers that cannot allocate device memory.
    Calls that overlap on the GPU race on that array."""
    def vp(x):
        return None if x is None or x == 0 else ctypes.c_void_p(int(x))
    return _check(load().lasso_path_static(vp(X), int(x_dtype), int(n), int(p), int(ldx), vp(y),
                                           vp(lambda_ratios), int(T), vp(beta0),
                                           ctypes.byref(opts) if opts is not None else None, vp(beta_out),
                                           vp(mask_out), vp(stats), vp(stream)))


def lasso_batch_workspace_size(n: int, p: int, B: int, opts: LassoOpts | None = None) -> int:
    return int(load().lasso_batch_workspace_size(int(n), int(p), int(B),
                                                 ctypes.byref(opts) if opts is not None else None))


def lasso_batch(X, n, p, ldx, Y, ldy, row_mask, ldm, B, lambda_ratios, T, beta0, ldb0, opts, beta_out, mask_out,
                stats, workspace, workspace_bytes, stream) -> int:
    """Direct call of the batched C entry point (pointers as integers)."""
    def vp(x):
        return None if x is None or x == 0 else ctypes.c_void_p(int(x))
    return _check(load().lasso_batch(vp(X), int(n), int(p), int(ldx), vp(Y), int(ldy), vp(row_mask), int(ldm),
                                     int(B), vp(lambda_ratios), int(T), vp(beta0), int(ldb0),
                                     ctypes.byref(opts) if opts is not None else None, vp(beta_out),
                                     vp(mask_out), vp(stats), vp(workspace), int(workspace_bytes), vp(stream)))


def solve_batch(XT, Y, ratios, n=None, row_mask=None, beta0=None, opts=None, workspace=None, stream=None,
                want_mask=True):
    """Allocate outputs as torch CUDA tensors and run lasso_batch.

    XT: (p, ldx) float32 CUDA tensor (column-major design); Y: (B, ldy) float64
    CUDA tensor (row b = problem b's responses); row_mask: (B, ldm) uint8 or
    None; beta0: (B, ldb0) float64 starting points or None; ratios: (T,)
    float64.  Returns beta (B, T, p), mask (B, T, words), stats (uint8 bytes
    of B*T records)."""
    import torch
    assert XT.is_cuda and XT.is_contiguous() and XT.dtype == torch.float32
    p, ldx = XT.shape
    B, ldy = Y.shape
    n = int(n if n is not None else ldy)
    T = int(ratios.shape[0])
    dev = XT.device
    opts = opts or lasso_default_opts()
    words = (p + 31) // 32
    beta_out = torch.empty((B, T, p), dtype=torch.float64, device=dev)
    mask_out = torch.empty((B, T, words), dtype=torch.int32, device=dev) if want_mask else None
    stats = torch.empty(B * T * STATS_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    need = lasso_batch_workspace_size(n, p, B, opts)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    if beta0 is not None:
        assert beta0.is_cuda and beta0.is_contiguous() and beta0.dtype == torch.float64 and beta0.shape[0] == B
    lasso_batch(XT.data_ptr(), n, p, ldx, Y.data_ptr(), ldy, row_mask.data_ptr() if row_mask is not None else None,
                row_mask.shape[1] if row_mask is not None else 0, B, ratios.data_ptr(), T,
                beta0.data_ptr() if beta0 is not None else None, beta0.shape[1] if beta0 is not None else 0,
                opts, beta_out.data_ptr(),
                mask_out.data_ptr() if mask_out is not None else None, stats.data_ptr(), workspace.data_ptr(),
                workspace.numel(), s.cuda_stream)
    return dict(beta=beta_out, mask=mask_out, stats=stats, workspace=workspace)


def lasso_correlations_bf16(X_bf16, n, p, ldx, R_bf16, ldr, B, C, ldc, workspace, workspace_bytes, stream) -> int:
    """C = X^T R on the tensor cores (pointers as integers)."""
    def vp(x):
        return None if x is None or x == 0 else ctypes.c_void_p(int(x))
    return _check(load().lasso_correlations_bf16(vp(X_bf16), int(n), int(p), int(ldx), vp(R_bf16), int(ldr), int(B),
                                                 vp(C), int(ldc), vp(workspace), int(workspace_bytes), vp(stream)))


def lasso_correlations_f32(X, n, p, ldx, r, c, cmax, stream) -> int:
    """c = X^T r and cmax = ||c||_inf (pointers as integers)."""
    def vp(x):
        return None if x is None or x == 0 else ctypes.c_void_p(int(x))
    return _check(load().lasso_correlations_f32(vp(X), int(n), int(p), int(ldx), vp(r), vp(c), vp(cmax),
                                                vp(stream)))


def lasso_batch_tune_candidates() -> int:
    return int(load().lasso_batch_tune_candidates())


def lasso_batch_tune_workspace_size(n, p, sample, lambdas) -> int:
    return int(load().lasso_batch_tune_workspace_size(int(n), int(p), int(sample), int(lambdas)))


def lasso_batch_tune(X, n, p, ldx, Y, ldy, row_mask, ldm, B, lambda_ratios, T, beta0, ldb0, opts, sample, lambdas,
                     tuned, times_ms, workspace, workspace_bytes, stream) -> int:
    """Direct call of the launch-shape autotuner (pointers as integers; tuned
    a LassoOpts to fill; times_ms a float32 numpy array or None)."""
    def vp(x):
        return None if x is None or x == 0 else ctypes.c_void_p(int(x))
    return _check(load().lasso_batch_tune(vp(X), int(n), int(p), int(ldx), vp(Y), int(ldy), vp(row_mask), int(ldm),
                                          int(B), vp(lambda_ratios), int(T), vp(beta0), int(ldb0),
                                          ctypes.byref(opts) if opts is not None else None, int(sample),
                                          int(lambdas), ctypes.byref(tuned),
                                          times_ms.ctypes.data_as(ctypes.c_void_p) if times_ms is not None else None,
                                          vp(workspace), int(workspace_bytes), vp(stream)))


def tune_batch(XT, Y, ratios, n=None, row_mask=None, beta0=None, opts=None, sample=None, lambdas=None, stream=None):
    """Run lasso_batch_tune on torch CUDA tensors (the layouts of solve_batch).
    Defaults: one resident wave of problems (2 x SMs) over the first quarter of
    the grid (at least 5 lambdas).  Returns (tuned LassoOpts, per-candidate
    times in ms as a numpy array)."""
    import torch
    p, ldx = XT.shape
    B, ldy = Y.shape
    n = int(n if n is not None else ldy)
    T = int(ratios.shape[0])
    opts = opts or lasso_default_opts()
    sample = int(sample if sample is not None else min(B, 2 * torch.cuda.get_device_properties(XT.device)
                                                       .multi_processor_count))
    # the first lambdas are check-dominated (where the tensor-core product
    # helps most); a quarter of the grid weighs the passes of the later ones
    lambdas = int(lambdas if lambdas is not None else min(T, max(5, T // 4)))
    need = lasso_batch_tune_workspace_size(n, p, sample, lambdas)
    ws = torch.empty(need, dtype=torch.uint8, device=XT.device)
    times = np.zeros(lasso_batch_tune_candidates(), dtype=np.float32)
    tuned = LassoOpts()
    s = stream if stream is not None else torch.cuda.current_stream(XT.device)

    def vp(x):
        return None if x is None or x == 0 else ctypes.c_void_p(int(x))
    _check(load().lasso_batch_tune(vp(XT.data_ptr()), n, p, ldx, vp(Y.data_ptr()), ldy,
                                   vp(row_mask.data_ptr() if row_mask is not None else None),
                                   row_mask.shape[1] if row_mask is not None else 0, B, vp(ratios.data_ptr()), T,
                                   vp(beta0.data_ptr() if beta0 is not None else None),
                                   beta0.shape[1] if beta0 is not None else 0, ctypes.byref(opts), sample, lambdas,
                                   ctypes.byref(tuned), times.ctypes.data_as(ctypes.c_void_p), vp(ws.data_ptr()),
                                   need, vp(s.cuda_stream)))
    return tuned, times


def lasso_path_csc_workspace_size(n: int, p: int, opts: LassoOpts | None = None) -> int:
    return int(load().lasso_path_csc_workspace_size(int(n), int(p), ctypes.byref(opts) if opts is not None else None))


def lasso_path_csc(colptr, rowidx, values, n, p, y, lambda_ratios, T, beta0, opts, beta_out, mask_out, stats,
                   workspace, workspace_bytes, stream) -> int:
    """Direct call of the C entry point (pointer arguments are device addresses
    or None).  Raises LassoError on a non-zero status."""
    def vp(x):
        return None if x is None else ctypes.c_void_p(int(x))
    return _check(load().lasso_path_csc(vp(colptr), vp(rowidx), vp(values), int(n), int(p), vp(y),
                                        vp(lambda_ratios), int(T), vp(beta0),
                                        ctypes.byref(opts) if opts is not None else None, vp(beta_out),
                                        vp(mask_out), vp(stats), vp(workspace), int(workspace_bytes),
                                        ctypes.c_void_p(int(stream) if stream else 0)))


def solve_path_csc(colptr, rowidx, values, y, ratios, n, beta0=None, opts=None, stream=None, want_mask=True):
    """Allocate outputs and the workspace as torch CUDA tensors and run
    lasso_path_csc.  colptr: (p+1,) int64, rowidx: (nnz,) int32, values:
    (nnz,) float64, y: (n,) float64, ratios: (T,) float64 CUDA tensors."""
    import torch
    p = int(colptr.shape[0]) - 1
    T = int(ratios.shape[0])
    dev = colptr.device
    opts = opts or lasso_default_opts()
    words = (p + 31) // 32
    beta_out = torch.empty((T, p), dtype=torch.float64, device=dev)
    mask_out = torch.empty((T, words), dtype=torch.int32, device=dev) if want_mask else None
    stats = torch.empty(T * STATS_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    need = lasso_path_csc_workspace_size(n, p, opts)
    workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    lasso_path_csc(colptr.data_ptr(), rowidx.data_ptr(), values.data_ptr(), n, p, y.data_ptr(), ratios.data_ptr(), T,
                   beta0.data_ptr() if beta0 is not None else None, opts, beta_out.data_ptr(),
                   mask_out.data_ptr() if mask_out is not None else None, stats.data_ptr(), workspace.data_ptr(),
                   workspace.numel(), s.cuda_stream)
    return dict(beta=beta_out, mask=mask_out, stats=stats, workspace=workspace)


PHASES = ("check", "chain", "verify", "round_end", "pass_end", "chain_entries", "rollbacks", "other")


def lasso_path_phase_cycles(workspace, stream) -> dict:
    """Phase counters of the last lasso_path run on `workspace` (a device
    address): SM cycles per phase and the chain-entry and rollback counts."""
    out = (ctypes.c_uint64 * 8)()
    _check(load().lasso_path_phase_cycles(ctypes.c_void_p(int(workspace)), ctypes.cast(out, ctypes.c_void_p),
                                          ctypes.c_void_p(int(stream) if stream else 0)))
    return dict(zip(PHASES, (int(v) for v in out)))


def stats_to_numpy(stats_tensor) -> np.ndarray:
    """A uint8 torch tensor of T * sizeof(stats) bytes -> structured numpy array."""
    return stats_tensor.cpu().numpy().view(STATS_DTYPE)


def solve_path(XT, y, ratios, n=None, beta0=None, opts=None, workspace=None, stream=None, want_mask=True):
    """Allocate outputs as torch CUDA tensors and run lasso_path.

    XT: (p, ldx) contiguous CUDA tensor (float32 or float64) -- the column-major
    design; y: (n,) float64 CUDA tensor; ratios: (T,) float64 CUDA tensor.
    Returns a dict with beta (T, p) float64, mask (T, words) int32 view of the
    uint32 words, stats (uint8 bytes; see stats_to_numpy)."""
    import torch
    assert XT.is_cuda and XT.is_contiguous() and XT.dim() == 2
    p, ldx = XT.shape
    n = int(n if n is not None else y.shape[0])
    xt = LASSO_F32 if XT.dtype == torch.float32 else LASSO_F64
    if XT.dtype not in (torch.float32, torch.float64):
        raise TypeError("XT must be float32 or float64")
    T = int(ratios.shape[0])
    dev = XT.device
    opts = opts or lasso_default_opts()
    words = (p + 31) // 32
    beta_out = torch.empty((T, p), dtype=torch.float64, device=dev)
    mask_out = torch.empty((T, words), dtype=torch.int32, device=dev) if want_mask else None
    stats = torch.empty(T * STATS_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    need = lasso_path_workspace_size(n, p, xt, opts)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    lasso_path(XT.data_ptr(), xt, n, p, ldx, y.data_ptr(), ratios.data_ptr(), T,
               beta0.data_ptr() if beta0 is not None else None, opts, beta_out.data_ptr(),
               mask_out.data_ptr() if mask_out is not None else None, stats.data_ptr(),
               workspace.data_ptr(), workspace.numel(), s.cuda_stream)
    return dict(beta=beta_out, mask=mask_out, stats=stats, workspace=workspace)
