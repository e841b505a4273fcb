"""ctypes binding of the learned warm start (include/lista.h).

The functions carry the C names and only marshal arguments; the forward and
backward passes, the optimiser and the data preparation all run in the CUDA
library.  ``ListaNet`` holds the parameters, gradients and Adam moments as
torch CUDA tensors (PyTorch supplies device memory and streams) and strings
the C calls together for training and inference.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import lassogs as _lg

EXPORTED = ("lista_workspace_size", "lista_cache_layout", "lista_init", "lista_normalize", "lista_forward",
            "lista_backward", "lista_adam", "lista_gather", "lista_targets", "lista_warm_start")

_bound = False


def _lib():
    global _bound
    lib = _lg.load()
    if not _bound:
        V, I32, I64, F, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_size_t
        lib.lista_workspace_size.argtypes = [I64, I64, I32, I64]
        lib.lista_workspace_size.restype = SZ
        lib.lista_cache_layout.argtypes = [I64, I64, I32, I64, V, V, V]
        lib.lista_init.argtypes = [V, I64, I64, I64, I32, F, V, V, V, V, V, SZ, V]
        lib.lista_normalize.argtypes = [V, I64, I64, I64, V, I64, I64, V, I64, V, V, SZ, V]
        lib.lista_forward.argtypes = [V, I64, I64, I64, V, V, V, I32, V, I64, I64, V, I32, V, SZ, V]
        lib.lista_backward.argtypes = [V, I64, I64, I64, V, V, V, I32, I64, V, V, V, V, V, V, V, SZ, V]
        lib.lista_adam.argtypes = [V, V, V, V, I64, I32, F, F, F, F, V]
        lib.lista_gather.argtypes = [V, I64, V, I64, I64, V, I64, V]
        lib.lista_targets.argtypes = [V, I64, V, I64, I64, V, V]
        lib.lista_warm_start.argtypes = [V, I64, I64, I64, V, V, V, I32, V, I64, I64, V, I64, I64, V, SZ, V]
        for name in EXPORTED[1:]:
            getattr(lib, name).restype = ctypes.c_int
        _bound = True
    return lib


def _vp(x):
    return None if x is None or x == 0 else ctypes.c_void_p(int(x))


def lista_workspace_size(n, p, L, B) -> int:
    return int(_lib().lista_workspace_size(int(n), int(p), int(L), int(B)))


def lista_cache_layout(n, p, L, B):
    """Byte offsets (u, v, z) of the per-layer forward cache in the workspace."""
    o = [ctypes.c_int64(0) for _ in range(3)]
    _lg._check(_lib().lista_cache_layout(int(n), int(p), int(L), int(B), *(ctypes.cast(ctypes.byref(x), ctypes.c_void_p)
                                                                          for x in o)))
    return tuple(int(x.value) for x in o)


def lista_init(X, n, p, ldx, L, ratio, W, D, tau, lip_out, workspace, workspace_bytes, stream):
    return _lg._check(_lib().lista_init(_vp(X), int(n), int(p), int(ldx), int(L), float(ratio), _vp(W), _vp(D),
                                        _vp(tau), _vp(lip_out), _vp(workspace), int(workspace_bytes), _vp(stream)))


def lista_normalize(X, n, p, ldx, Y, ldy, B, Ytil, ldyt, s, workspace, workspace_bytes, stream):
    return _lg._check(_lib().lista_normalize(_vp(X), int(n), int(p), int(ldx), _vp(Y), int(ldy), int(B), _vp(Ytil),
                                             int(ldyt), _vp(s), _vp(workspace), int(workspace_bytes), _vp(stream)))


def lista_forward(X, n, p, ldx, W, D, tau, L, Ytil, ldyt, B, beta_out, keep_cache, workspace, workspace_bytes, stream):
    return _lg._check(_lib().lista_forward(_vp(X), int(n), int(p), int(ldx), _vp(W), _vp(D), _vp(tau), int(L),
                                           _vp(Ytil), int(ldyt), int(B), _vp(beta_out), int(keep_cache),
                                           _vp(workspace), int(workspace_bytes), _vp(stream)))


def lista_backward(X, n, p, ldx, W, D, tau, L, B, betaL, targets, gW, gD, gtau, loss_out, workspace,
                   workspace_bytes, stream):
    return _lg._check(_lib().lista_backward(_vp(X), int(n), int(p), int(ldx), _vp(W), _vp(D), _vp(tau), int(L),
                                            int(B), _vp(betaL), _vp(targets), _vp(gW), _vp(gD), _vp(gtau),
                                            _vp(loss_out), _vp(workspace), int(workspace_bytes), _vp(stream)))


def lista_adam(theta, grad, m, v, count, t, lr, b1, b2, eps, stream):
    return _lg._check(_lib().lista_adam(_vp(theta), _vp(grad), _vp(m), _vp(v), int(count), int(t), float(lr),
                                        float(b1), float(b2), float(eps), _vp(stream)))


def lista_gather(src, ld_src, idx, B, width, dst, ld_dst, stream):
    return _lg._check(_lib().lista_gather(_vp(src), int(ld_src), _vp(idx), int(B), int(width), _vp(dst),
                                          int(ld_dst), _vp(stream)))


def lista_targets(beta_hat, ldbh, s, B, p, targets, stream):
    return _lg._check(_lib().lista_targets(_vp(beta_hat), int(ldbh), _vp(s), int(B), int(p), _vp(targets),
                                           _vp(stream)))


def lista_warm_start(X, n, p, ldx, W, D, tau, L, Y, ldy, B, beta0, ldb0, max_nonzeros, workspace, workspace_bytes,
                     stream):
    return _lg._check(_lib().lista_warm_start(_vp(X), int(n), int(p), int(ldx), _vp(W), _vp(D), _vp(tau), int(L),
                                              _vp(Y), int(ldy), int(B), _vp(beta0), int(ldb0), int(max_nonzeros),
                                              _vp(workspace), int(workspace_bytes), _vp(stream)))


class ListaNet:
    """The unrolled ISTA network for one design X (a (p, ldx) float32 CUDA
    tensor, column-major) with L layers, trained for lambda = ratio *
    lambda_max(y).  Parameters W (p, n), D (L, p), tau (L,), their gradients
    and Adam moments are float32 CUDA tensors."""

    def __init__(self, XT, n, L=8, ratio=0.05, init=True):
        import torch
        assert XT.is_cuda and XT.dtype == torch.float32 and XT.is_contiguous()
        self.XT, self.n, self.L, self.ratio = XT, int(n), int(L), float(ratio)
        self.p, self.ldx = XT.shape
        dev = XT.device
        f32 = dict(dtype=torch.float32, device=dev)
        self.W = torch.zeros((self.p, self.n), **f32)
        self.D = torch.zeros((self.L, self.p), **f32)
        self.tau = torch.zeros((self.L,), **f32)
        self.lip = torch.zeros((1,), **f32)
        self.grads = [torch.zeros_like(t) for t in (self.W, self.D, self.tau)]
        self.m = [torch.zeros_like(t) for t in (self.W, self.D, self.tau)]
        self.v = [torch.zeros_like(t) for t in (self.W, self.D, self.tau)]
        self.loss = torch.zeros((1,), dtype=torch.float64, device=dev)
        self.step = 0
        self._ws = {}
        # scale of each parameter group at the ISTA point (W = X^T with unit
        # columns, d = 1/Lip, tau = ratio/Lip): Adam steps are relative to it
        self.pscale = (1.0 / np.sqrt(self.n), 1.0, self.ratio)
        if init:
            ws = self.workspace(1)
            lista_init(self.XT.data_ptr(), self.n, self.p, self.ldx, self.L, self.ratio, self.W.data_ptr(),
                       self.D.data_ptr(), self.tau.data_ptr(), self.lip.data_ptr(), ws.data_ptr(), ws.numel(),
                       self._stream())
            lip = float(self.lip.item())
            self.pscale = (1.0 / np.sqrt(self.n), 1.0 / lip, self.ratio / lip)

    def _stream(self):
        import torch
        return torch.cuda.current_stream(self.XT.device).cuda_stream

    def workspace(self, B):
        import torch
        B = int(B)
        if B not in self._ws:
            need = lista_workspace_size(self.n, self.p, self.L, B)
            self._ws[B] = torch.empty(need, dtype=torch.uint8, device=self.XT.device)
        return self._ws[B]

    def params(self):
        return (self.W, self.D, self.tau)

    def normalize(self, Y):
        """Y (B, ldy) float64 CUDA tensor -> (Ytil (B, n) float32, s (B,) float32)."""
        import torch
        B, ldy = Y.shape
        Ytil = torch.empty((B, self.n), dtype=torch.float32, device=Y.device)
        s = torch.empty((B,), dtype=torch.float32, device=Y.device)
        ws = self.workspace(B)
        lista_normalize(self.XT.data_ptr(), self.n, self.p, self.ldx, Y.data_ptr(), ldy, B, Ytil.data_ptr(),
                        self.n, s.data_ptr(), ws.data_ptr(), ws.numel(), self._stream())
        return Ytil, s

    def forward(self, Ytil, keep_cache=False):
        import torch
        B, ldyt = Ytil.shape
        out = torch.empty((B, self.p), dtype=torch.float32, device=Ytil.device)
        ws = self.workspace(B)
        lista_forward(self.XT.data_ptr(), self.n, self.p, self.ldx, self.W.data_ptr(), self.D.data_ptr(),
                      self.tau.data_ptr(), self.L, Ytil.data_ptr(), ldyt, B, out.data_ptr(), int(keep_cache),
                      ws.data_ptr(), ws.numel(), self._stream())
        return out

    def cache(self, B):
        """(u, v, z) of the last forward(keep_cache=True) on B samples, as
        float32 views of the workspace: shapes (L, B, n), (L, B, p), (L, B, p)."""
        import torch
        ou, ov, oz = lista_cache_layout(self.n, self.p, self.L, B)
        ws = self.workspace(B)

        def view(off, width):
            cnt = self.L * B * width
            return ws[off:off + 4 * cnt].view(torch.float32).view(self.L, B, width)
        return view(ou, self.n), view(ov, self.p), view(oz, self.p)

    def backward(self, betaL, targets):
        """Gradients of the batch of the preceding forward(keep_cache=True)
        into self.grads; the loss (FP64) into self.loss."""
        B = betaL.shape[0]
        ws = self.workspace(B)
        gW, gD, gt = self.grads
        lista_backward(self.XT.data_ptr(), self.n, self.p, self.ldx, self.W.data_ptr(), self.D.data_ptr(),
                       self.tau.data_ptr(), self.L, B, betaL.data_ptr(), targets.data_ptr(), gW.data_ptr(),
                       gD.data_ptr(), gt.data_ptr(), self.loss.data_ptr(), ws.data_ptr(), ws.numel(), self._stream())
        return self.loss

    def adam(self, lr, b1=0.9, b2=0.999, eps=1e-8, relative=True):
        """One Adam step on W, D and tau.  relative: the step of each group is
        lr times the group's scale at the ISTA point (pscale), so one rate
        fits parameters of very different magnitudes."""
        self.step += 1
        for k, (th, g, m, v) in enumerate(zip(self.params(), self.grads, self.m, self.v)):
            rate = lr * self.pscale[k] if relative else lr
            lista_adam(th.data_ptr(), g.data_ptr(), m.data_ptr(), v.data_ptr(), th.numel(), self.step, rate, b1, b2,
                       eps, self._stream())

    def train_step(self, Ytil_all, T_all, idx, lr, **adam_kw):
        """One minibatch step: rows idx (int32 CUDA tensor) of the normalised
        responses Ytil_all (N, n) and targets T_all (N, p)."""
        import torch
        B = idx.numel()
        yb = torch.empty((B, self.n), dtype=torch.float32, device=idx.device)
        tb = torch.empty((B, self.p), dtype=torch.float32, device=idx.device)
        st = self._stream()
        lista_gather(Ytil_all.data_ptr(), Ytil_all.shape[1], idx.data_ptr(), B, self.n, yb.data_ptr(), self.n, st)
        lista_gather(T_all.data_ptr(), T_all.shape[1], idx.data_ptr(), B, self.p, tb.data_ptr(), self.p, st)
        betaL = self.forward(yb, keep_cache=True)
        loss = self.backward(betaL, tb)
        self.adam(lr, **adam_kw)
        return loss

    def fit(self, Ytil_all, T_all, epochs, batch=256, lr=1e-3, seed=0, **adam_kw):
        """Minibatch Adam over the training pairs; returns the per-epoch mean
        losses (read back once per epoch)."""
        import torch
        N = Ytil_all.shape[0]
        rng = np.random.default_rng(seed)
        hist = []
        for _ in range(int(epochs)):
            perm = torch.from_numpy(rng.permutation(N).astype(np.int32)).to(Ytil_all.device)
            acc = torch.zeros((1,), dtype=torch.float64, device=Ytil_all.device)
            nb = 0
            for k in range(0, N - batch + 1, batch):
                acc += self.train_step(Ytil_all, T_all, perm[k:k + batch], lr, **adam_kw)
                nb += 1
            hist.append(float(acc.item()) / max(nb, 1))
        return hist

    def targets(self, beta_hat, s):
        """t_b = beta_hat_b / s_b as float32 (B, p) from FP64 solver output (B, ldbh)."""
        import torch
        B, ldbh = beta_hat.shape
        t = torch.empty((B, self.p), dtype=torch.float32, device=beta_hat.device)
        lista_targets(beta_hat.data_ptr(), ldbh, s.data_ptr(), B, self.p, t.data_ptr(), self._stream())
        return t

    def warm_start(self, Y, max_nonzeros=None):
        """beta0 (B, p) float64 for responses Y (B, ldy) float64: the starting
        points lasso_batch takes, each row cut to its max_nonzeros largest
        entries (default n; 0 keeps all)."""
        import torch
        B, ldy = Y.shape
        K = self.n if max_nonzeros is None else int(max_nonzeros)
        beta0 = torch.empty((B, self.p), dtype=torch.float64, device=Y.device)
        ws = self.workspace(B)
        lista_warm_start(self.XT.data_ptr(), self.n, self.p, self.ldx, self.W.data_ptr(), self.D.data_ptr(),
                         self.tau.data_ptr(), self.L, Y.data_ptr(), ldy, B, beta0.data_ptr(), self.p, K,
                         ws.data_ptr(), ws.numel(), self._stream())
        return beta0
