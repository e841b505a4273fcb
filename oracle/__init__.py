"""FP64 CPU oracle for Lasso coordinate descent with GAP SAFE screening.

TEST INFRASTRUCTURE ONLY: the slow, plain reference that the CUDA library is
checked against (Fercoq, Gramfort, Salmon, ICML 2015, Algorithm 1).  Only the
test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import it.  It shares no code with the CUDA library and never imports it.

The C part (``lasso_oracle.c``) is compiled on first use with gcc
(``-O2 -ffp-contract=off``); this module only marshals numpy arrays.

Pins (checked by the ``not gpu`` tests): beta = 0 for lambda >= lambda_max
(Sec. 1.2), soft-thresholding closed form on orthonormal designs, brute-force
support enumeration for p <= 12 (``oracle.bruteforce``), KKT conditions
(Eq. (4)), safety of every sphere (Thm. 2 + Prop. 1), the sequential identity
of Prop. 3, finite identification (Thm. 1); for the options: the dome's
support function and parameters against sampled maxima over the sets they come
from (Eq. (11)), Thm. 2's refined radius recomputed from its definition, and
the Elastic-Net's closed form, KKT conditions and exact solution (appendix).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lasso_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblasso_oracle.so")
_lock = threading.Lock()
_lib = None

# per-lambda record fields (same order as the C enum)
STAT_FIELDS = ("lambda", "primal", "dual", "gap", "radius", "alpha", "epochs",
               "checks", "n_active", "n_nonzero", "converged")
NF = len(STAT_FIELDS)


def build(force: bool = False) -> str:
    """Compile the C oracle into oracle/_build (plain gcc, no BLAS)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Opts(ctypes.Structure):
    _fields_ = [("screen_period", ctypes.c_int32), ("dual_point", ctypes.c_int32),
                ("xtr_scope", ctypes.c_int32), ("warm_start", ctypes.c_int32),
                ("max_epochs", ctypes.c_int64), ("gap_tol_rel", ctypes.c_double),
                ("screen_rule", ctypes.c_int32), ("refined_radius", ctypes.c_int32),
                ("enet_alpha", ctypes.c_double)]


class _CheckResult(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("xtr_inf", ctypes.c_double),
                ("primal", ctypes.c_double), ("dual", ctypes.c_double),
                ("gap", ctypes.c_double), ("radius", ctypes.c_double),
                ("tau", ctypes.c_double), ("n_kept", ctypes.c_int64),
                ("dome_rad", ctypes.c_double), ("dome_alpha", ctypes.c_double)]


class _Log(ctypes.Structure):
    _fields_ = [("cap", ctypes.c_int64), ("count", ctypes.c_int64),
                ("t", ctypes.c_void_p), ("gap", ctypes.c_void_p), ("radius", ctypes.c_void_p),
                ("alpha", ctypes.c_void_p), ("rho", ctypes.c_void_p),
                ("dome_rad", ctypes.c_void_p), ("dome_alpha", ctypes.c_void_p)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(build())
    return _lib


def _bind(path):
    """Load a compiled oracle library and declare its C signatures."""
    lib = ctypes.CDLL(path)
    P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    lib.orc_precompute.argtypes = [P, I64, I64, I64, P, P, P, P]
    lib.orc_precompute.restype = None
    lib.orc_lambda_ratios.argtypes = [I32, D, P]
    lib.orc_lambda_ratios.restype = None
    lib.orc_check.argtypes = [P, I64, I64, I64, P, D, P, P, P, P, P, D, P, P, P, P, P]
    lib.orc_check.restype = None
    lib.orc_dome_support.argtypes = [D, D, D, D, D]
    lib.orc_dome_support.restype = D
    lib.orc_cd_pass.argtypes = [P, I64, I64, P, I64, P, D, P, P]
    lib.orc_cd_pass.restype = None
    lib.orc_lasso_path.argtypes = [P, I64, I64, I64, P, P, I32, P, P, P, P, P, P]
    lib.orc_lasso_path.restype = ctypes.c_int
    lib.orc_lasso_batch.argtypes = [P, I64, I64, I64, P, P, I64, P, I32, P, P, P, P, P]
    lib.orc_lasso_batch.restype = ctypes.c_int
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _colmajor64(X, n=None):
    """Return (Xc, n, p, ldx) with Xc a C-contiguous (p, ldx) float64 array,
    i.e. column-major storage.  X may be given as an (n, p) array (any order)
    or already as a (p, ldx) column-major block via n=..."""
    if n is not None:
        Xc = np.ascontiguousarray(X, dtype=np.float64)
        p, ldx = Xc.shape
        return Xc, int(n), p, ldx
    X = np.asarray(X)
    nn, p = X.shape
    Xc = np.ascontiguousarray(X.T, dtype=np.float64)
    return Xc, nn, p, nn


def _opts(screen_period=10, dual_point=0, xtr_scope=0, warm_start=True, max_epochs=100000,
          gap_tol_rel=1e-6, screen_rule=0, refined_radius=0, enet_alpha=1.0):
    return _Opts(int(screen_period), int(dual_point), int(xtr_scope), int(bool(warm_start)),
                 int(max_epochs), float(gap_tol_rel), int(screen_rule), int(refined_radius),
                 float(enet_alpha))


def mask_words(p):
    return (p + 31) // 32


def unpack_mask(words, p):
    """uint32 words -> bool array of length p (bit j%32 of word j//32)."""
    w = np.asarray(words, dtype=np.uint32)
    bits = np.unpackbits(w.view(np.uint8).reshape(-1, 4)[:, ::-1], axis=1)[:, ::-1]
    return bits.reshape(-1)[:p].astype(bool) if w.ndim == 1 else None


def precompute(X, y, n=None):
    """||x_j||^2, X^T y, lambda_max = ||X^T y||_inf, ||y||^2 (Sec. 1.2)."""
    lib = _load()
    Xc, n, p, ldx = _colmajor64(X, n)
    y = np.ascontiguousarray(y, dtype=np.float64)
    norms2 = np.empty(p)
    c0 = np.empty(p)
    scal = np.empty(3)
    lib.orc_precompute(_ptr(Xc), n, p, ldx, _ptr(y), _ptr(norms2), _ptr(c0), _ptr(scal))
    return dict(norms2=norms2, c0=c0, lambda_max=scal[0], ynorm2=scal[1], argmax=int(scal[2]))


def lambda_ratios(T, delta):
    """lambda_t / lambda_max = 10^(-delta t/(T-1)), t = 0..T-1 (Sec. 3.3)."""
    lib = _load()
    out = np.empty(int(T))
    lib.orc_lambda_ratios(int(T), float(delta), _ptr(out))
    return out


def dome_support(cx, rad, alpha, nx, xnorm):
    """Support function of the dome D(c, rad, alpha, nrm) at x, from c^T x,
    nrm^T x and ||x|| (appendix, dome test)."""
    return _load().orc_dome_support(float(cx), float(rad), float(alpha), float(nx), float(xnorm))


def check(X, y, beta, rho, lam, mask_in=None, n=None, **opt):
    """One GAP SAFE check on given (beta, rho): returns dict with c, mu (the
    test value per feature), alpha, xtr_inf, primal, dual, gap, radius, tau,
    n_kept, dome_rad, dome_alpha and mask (uint32 words)."""
    lib = _load()
    Xc, n, p, ldx = _colmajor64(X, n)
    y = np.ascontiguousarray(y, dtype=np.float64)
    pre = precompute(Xc, y, n=n)
    W = mask_words(p)
    if mask_in is None:
        mask_in = np.full(W, 0xFFFFFFFF, dtype=np.uint32)
        if p % 32:
            mask_in[-1] = (1 << (p % 32)) - 1
    mask_in = np.ascontiguousarray(mask_in, dtype=np.uint32)
    mask_out = np.empty(W, dtype=np.uint32)
    c = np.empty(p)
    mu = np.empty(p)
    res = _CheckResult()
    o = _opts(**opt)
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    lib.orc_check(_ptr(Xc), n, p, ldx, _ptr(y), pre["ynorm2"], _ptr(pre["norms2"]), _ptr(pre["c0"]),
                  _ptr(beta), _ptr(rho), _ptr(mask_in), float(lam), ctypes.byref(o), _ptr(mask_out),
                  _ptr(c), _ptr(mu), ctypes.byref(res))
    out = {f: getattr(res, f) for f, _ in _CheckResult._fields_}
    out.update(c=c, mu=mu, mask=mask_out)
    return out


def cd_pass(X, beta, rho, lam, active, n=None):
    """One cyclic pass over the ascending index list `active` (updates copies)."""
    lib = _load()
    Xc, n, p, ldx = _colmajor64(X, n)
    beta = np.array(beta, dtype=np.float64)
    rho = np.array(rho, dtype=np.float64)
    lst = np.ascontiguousarray(active, dtype=np.int64)
    norms2 = precompute(Xc, np.zeros(n), n=n)["norms2"]
    lib.orc_cd_pass(_ptr(Xc), n, ldx, _ptr(lst), len(lst), _ptr(norms2), float(lam), _ptr(beta),
                    _ptr(rho))
    return beta, rho


def lasso_path(X, y, ratios, beta0=None, n=None, log_checks=0, **opt):
    """Algorithm 1 along lambda_t = lambda_max * ratios[t].

    Returns dict(beta=(T, p), mask=(T, words) uint32, stats=dict of (T,)
    arrays, status=int, lambda_max, ynorm2) and, when log_checks > 0, a check
    log (t, gap, radius, alpha, rho per check)."""
    lib = _load()
    Xc, n, p, ldx = _colmajor64(X, n)
    y = np.ascontiguousarray(y, dtype=np.float64)
    ratios = np.ascontiguousarray(ratios, dtype=np.float64)
    T = len(ratios)
    W = mask_words(p)
    beta_out = np.empty((T, p))
    mask_out = np.empty((T, W), dtype=np.uint32)
    stats = np.empty((T, NF))
    b0 = None if beta0 is None else np.ascontiguousarray(beta0, dtype=np.float64)
    o = _opts(**opt)
    log = None
    logbufs = None
    if log_checks:
        cap = int(log_checks)
        logbufs = dict(t=np.zeros(cap, dtype=np.int32), gap=np.zeros(cap), radius=np.zeros(cap),
                       alpha=np.zeros(cap), rho=np.zeros((cap, n)), dome_rad=np.zeros(cap),
                       dome_alpha=np.zeros(cap))
        log = _Log(cap, 0, *(_ptr(logbufs[k]).value
                             for k in ("t", "gap", "radius", "alpha", "rho", "dome_rad", "dome_alpha")))
    rc = lib.orc_lasso_path(_ptr(Xc), n, p, ldx, _ptr(y), _ptr(ratios), T, _ptr(b0), ctypes.byref(o),
                            _ptr(beta_out), _ptr(mask_out), _ptr(stats),
                            ctypes.byref(log) if log is not None else None)
    pre = precompute(Xc, y, n=n)
    out = dict(beta=beta_out, mask=mask_out, stats={f: stats[:, i] for i, f in enumerate(STAT_FIELDS)},
               status=int(rc), lambda_max=pre["lambda_max"] / float(opt.get("enet_alpha", 1.0)),
               ynorm2=pre["ynorm2"])
    if log is not None:
        k = log.count
        out["log"] = {key: v[:k] for key, v in logbufs.items()}
    return out


def lasso_batch(X, Y, ratios, row_mask=None, n=None, beta0=None, **opt):
    """Independent paths over one design: problem b uses rows with
    row_mask[b, i] != 0, response Y[b] (shape (B, n)) and starting point
    beta0[b] (shape (B, p), zeros when None).  Returns
    beta (B, T, p), mask (B, T, words), stats dict of (B, T) arrays."""
    lib = _load()
    Xc, n, p, ldx = _colmajor64(X, n)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    B = Y.shape[0]
    assert Y.shape[1] == n
    rm = None if row_mask is None else np.ascontiguousarray(row_mask, dtype=np.uint8)
    ratios = np.ascontiguousarray(ratios, dtype=np.float64)
    T = len(ratios)
    W = mask_words(p)
    beta_out = np.empty((B, T, p))
    mask_out = np.empty((B, T, W), dtype=np.uint32)
    stats = np.empty((B, T, NF))
    o = _opts(**opt)
    b0 = None if beta0 is None else np.ascontiguousarray(beta0, dtype=np.float64).reshape(B, p)
    rc = lib.orc_lasso_batch(_ptr(Xc), n, p, ldx, _ptr(Y), _ptr(rm), B, _ptr(ratios), T, _ptr(b0),
                             ctypes.byref(o), _ptr(beta_out), _ptr(mask_out), _ptr(stats))
    return dict(beta=beta_out, mask=mask_out,
                stats={f: stats[:, :, i] for i, f in enumerate(STAT_FIELDS)}, status=int(rc))
