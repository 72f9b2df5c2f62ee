"""Thin Python binding of the C ABI (include/gp.h): the same entry points, taking torch CUDA tensors.

Every function only checks and marshals arguments and calls libgp; all computation happens in the
library's CUDA kernels. Tensors must be float64, contiguous and on the context's device. Errors raise
GPError(status, info).
"""
from __future__ import annotations

import ctypes

import torch

from . import _native as N


class GPError(RuntimeError):
    def __init__(self, status: int, info: int = 0, where: str = ""):
        lib = N.load()
        msg = lib.gp_status_string(status).decode()
        super().__init__(f"{where}: {msg} (status {status}, info {info})")
        self.status = status
        self.info = info


def _check(status: int, where: str):
    if status != N.GP_OK:
        raise GPError(status, 0, where)


def _dev(t: torch.Tensor, name: str, shape=None) -> int:
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda" or t.dtype != torch.float64:
        raise TypeError(f"{name} must be a float64 CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t.data_ptr()


class Hyper(tuple):
    """(l, v, s2) in the textbook SE form v*exp(-r^2/(2 l^2)) + s2*delta."""

    def __new__(cls, l=1.0, v=1.0, s2=0.1):
        return super().__new__(cls, (float(l), float(v), float(s2)))

    @property
    def c(self):
        return N.gp_hyper(self[0], self[1], self[2])


class Context:
    """Owns a gp_ctx (device, stream, configuration) and the factors created through it."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None, tile: int = 0,
                 precision: str = "fp64", ir_tol: float = 0.0, ir_maxit: int = 0, noisy_prior: bool = False,
                 timeout_s: float = 0.0, grid: int = 0, withhold_task: int | None = None):
        self.lib = N.load()
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        cfg = N.gp_config()
        cfg.tile = tile
        cfg.precision = {"fp64": N.GP_FP64, "fp32": N.GP_FP32}[precision]
        cfg.ir_tol = ir_tol
        cfg.ir_maxit = ir_maxit
        cfg.noisy_prior = int(noisy_prior)
        cfg.timeout_ns = int(timeout_s * 1e9)
        cfg.grid = grid
        if withhold_task is not None:  # test hook: never publish this task's completion
            cfg.withhold_task = withhold_task
            cfg.withhold_enable = 1
        h = ctypes.c_void_p()
        _check(self.lib.gp_create(ctypes.byref(h), device, ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(cfg)),
               "gp_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.gp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def launch_count(self) -> int:
        return int(self.lib.gp_launch_count(self.h))

    def set_stream(self, stream: torch.cuda.Stream):
        self.stream = stream
        _check(self.lib.gp_set_stream(self.h, ctypes.c_void_p(stream.cuda_stream)), "gp_set_stream")


class Factor:
    """A gp_factor: the tiled K (then L) of one training set, plus the solve workspace."""

    def __init__(self, ctx: Context, X: torch.Tensor):
        self.ctx = ctx
        self.h = ctypes.c_void_p()
        self.X = X  # keeps the caller's training inputs alive: the library reads them later
        self.n, self.D = X.shape

    def free(self):
        if self.h and self.h.value:
            self.ctx.lib.gp_factor_free(self.ctx.h, self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def gp_sync(ctx: Context) -> None:
    info = ctypes.c_int64(0)
    s = ctx.lib.gp_sync(ctx.h, ctypes.byref(info))
    if s != N.GP_OK:
        raise GPError(s, info.value, "gp_sync")


def gp_assemble(ctx: Context, X: torch.Tensor, hyper: Hyper, factor: Factor | None = None) -> Factor:
    n, D = X.shape
    _dev(X, "X")
    f = factor if factor is not None else Factor(ctx, X)
    f.X = X
    _check(ctx.lib.gp_assemble(ctx.h, X.data_ptr(), n, D, Hyper(*hyper).c, ctypes.byref(f.h)), "gp_assemble")
    f.n, f.D = n, D
    return f


def gp_cholesky(ctx: Context, f: Factor) -> None:
    _check(ctx.lib.gp_cholesky(ctx.h, f.h), "gp_cholesky")


def gp_predict_mean(ctx: Context, f: Factor, y: torch.Tensor, Xs: torch.Tensor, out: torch.Tensor | None = None,
                    want_iters: bool = False):
    m = Xs.shape[0]
    _dev(y, "y", (f.n,))
    _dev(Xs, "Xs", (m, f.D))
    if out is None:
        out = torch.empty(m, dtype=torch.float64, device=Xs.device)
    _dev(out, "mean_out", (m,))
    it = ctypes.c_int32(0)
    _check(ctx.lib.gp_predict_mean(ctx.h, f.h, y.data_ptr(), Xs.data_ptr(), m, out.data_ptr(),
                                   ctypes.byref(it) if want_iters else None), "gp_predict_mean")
    return (out, it.value) if want_iters else out


def gp_predict_full_cov(ctx: Context, f: Factor, Xs: torch.Tensor, out: torch.Tensor | None = None):
    m = Xs.shape[0]
    _dev(Xs, "Xs", (m, f.D))
    if out is None:
        out = torch.empty((m, m), dtype=torch.float64, device=Xs.device)
    _dev(out, "cov_out", (m, m))
    _check(ctx.lib.gp_predict_full_cov(ctx.h, f.h, Xs.data_ptr(), m, out.data_ptr()), "gp_predict_full_cov")
    return out


def gp_factor_rows(ctx: Context, f: Factor, row0: int = 0, nrows: int | None = None) -> torch.Tensor:
    nrows = f.n - row0 if nrows is None else nrows
    out = torch.empty((nrows, f.n), dtype=torch.float64, device=ctx.device)
    _check(ctx.lib.gp_factor_rows(ctx.h, f.h, row0, nrows, out.data_ptr()), "gp_factor_rows")
    return out


def gp_alpha(ctx: Context, f: Factor) -> torch.Tensor:
    out = torch.empty(f.n, dtype=torch.float64, device=ctx.device)
    _check(ctx.lib.gp_alpha(ctx.h, f.h, out.data_ptr()), "gp_alpha")
    return out


def gp_logdet(ctx: Context, f: Factor) -> float:
    out = ctypes.c_double(0.0)
    _check(ctx.lib.gp_logdet(ctx.h, f.h, ctypes.byref(out)), "gp_logdet")
    return out.value


def gp_nlml_grad(ctx: Context, X: torch.Tensor, y: torch.Tensor, hyper: Hyper):
    n, D = X.shape
    _dev(X, "X")
    _dev(y, "y", (n,))
    nl = ctypes.c_double(0.0)
    g = (ctypes.c_double * 3)()
    _check(ctx.lib.gp_nlml_grad(ctx.h, X.data_ptr(), y.data_ptr(), n, D, Hyper(*hyper).c, ctypes.byref(nl), g),
           "gp_nlml_grad")
    return nl.value, [g[0], g[1], g[2]]


def predict(X, y, Xs, hyper=Hyper(), ctx: Context | None = None, full_cov: bool = True):
    """Convenience: assemble, factor, and predict mean (and full covariance) in one call."""
    ctx = ctx or Context(X.device.index or 0)
    f = gp_assemble(ctx, X, hyper)
    gp_cholesky(ctx, f)
    mean = gp_predict_mean(ctx, f, y, Xs)
    cov = gp_predict_full_cov(ctx, f, Xs) if full_cov else None
    gp_sync(ctx)
    return mean, cov
