"""Thin Python binding of the C ABI (include/gp.h): the same entry points, taking torch CUDA tensors.

Every function only checks and marshals arguments and calls libgp; all computation happens in the
library's CUDA kernels. Tensors must be float64, contiguous and on the context's device. Errors raise
GPError(status, info).
"""
from __future__ import annotations

import ctypes
import warnings

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
                 timeout_s: float = 0.0, grid: int = 0, withhold_task: int | None = None,
                 withhold_solve_block: int | None = None, tensor_cores: bool = True, trace: bool = False, batch_order: int = 0, batch_ctas_per_sm: int = 0,
                 locality_order: bool | None = None, shift: float = 0.0, tile_variant: str = "right"):
        self.lib = N.load()
        self.precision = precision
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        cfg = N.gp_config()
        cfg.tile = tile
        cfg.precision = N.PRECISIONS[precision]
        cfg.ir_tol = ir_tol
        cfg.ir_maxit = ir_maxit
        cfg.noisy_prior = int(noisy_prior)
        cfg.timeout_ns = int(timeout_s * 1e9)
        cfg.grid = grid
        cfg.tensor_cores = 0 if tensor_cores else -1
        cfg.trace = int(trace)
        cfg.batch_order = batch_order
        cfg.batch_ctas_per_sm = batch_ctas_per_sm
        cfg.locality_order = 0 if locality_order is None else (1 if locality_order else -1)
        cfg.shift = shift
        cfg.tile_variant = {"right": 0, "left": 1, "top": 2}[tile_variant]
        if withhold_task is not None:  # test hook: never publish this task's completion
            cfg.withhold_task = withhold_task
            cfg.withhold_enable = 1
        elif withhold_solve_block is not None:  # test hook: never publish this forward block of the mean solve
            cfg.withhold_task = withhold_solve_block
            cfg.withhold_enable = 2
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


TASK_NAMES = ["POTRF", "TRSM", "UPDATE", "VTRSM", "VGEMM", "WSYRK", "FSOLVE", "FGEMV", "BSOLVE", "BGEMV",
              "RUPD", "RTRSM", "RDIAG", "RPOTRF", "TRTRI", "VGEMM_G", "WSYRK_G",
              "FSOLVE_C", "BSOLVE_C", "UPDATE2"]


def gp_trace(ctx: Context):
    """Per-task trace of the last persistent-kernel launch (Context(trace=True)): an int64 array of
    rows {kind, p, q, r, cta, t_taken, t_ready, t_done} (ns)."""
    import numpy as np
    n = ctx.lib.gp_trace(ctx.h, None, 0)
    if n < 0:
        raise RuntimeError("no trace: create the context with trace=True and run a factorisation first")
    out = np.zeros((n, 8), dtype=np.int64)
    ctx.lib.gp_trace(ctx.h, out.ctypes.data, n)
    return out


def trace_to_chrome(rows, path: str):
    """Writes a trace from gp_trace as Chrome-trace JSON (one row per CTA; wait and run slices)."""
    import json
    t0 = int(rows[:, 5].min())
    ev = []
    for kind, p, q, r, cta, tt, tr, td in rows.tolist():
        name = f"{TASK_NAMES[kind & 31]}({p},{q},{r})" + (f" gp{kind >> 5}" if kind >> 5 else "")
        ev.append({"name": "wait", "ph": "X", "pid": 0, "tid": cta, "ts": (tt - t0) / 1e3, "dur": (tr - tt) / 1e3})
        ev.append({"name": name, "ph": "X", "pid": 0, "tid": cta, "ts": (tr - t0) / 1e3, "dur": (td - tr) / 1e3})
    with open(path, "w") as fh:
        json.dump({"traceEvents": ev}, fh)


def debug_fail_alloc(k: int) -> None:
    """Test hook: the k-th device allocation of the library from now on fails (GP_ERR_OOM); 0 = off."""
    N.load().gp_debug_fail_alloc(int(k))


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
    s = ctx.lib.gp_predict_mean(ctx.h, f.h, y.data_ptr(), Xs.data_ptr(), m, out.data_ptr(),
                                ctypes.byref(it) if want_iters else None)
    if s == N.GP_ERR_NO_CONVERGENCE:  # the refined result is still returned
        warnings.warn("gp_predict_mean: iterative refinement stopped above its tolerance", RuntimeWarning)
    else:
        _check(s, "gp_predict_mean")
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


def debug_exp_neg(ctx: Context, x: torch.Tensor) -> torch.Tensor:
    """Test hook: the covariance assembly's exponential of each entry of x (float64 CUDA tensor)."""
    _dev(x, "x")
    out = torch.empty_like(x)
    _check(ctx.lib.gp_debug_exp_neg(ctx.h, x.data_ptr(), x.numel(), out.data_ptr()), "gp_debug_exp_neg")
    return out


def gp_solve(ctx: Context, f: Factor, b: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
    """x = (L L^T)^{-1} b with the stored factor, no refinement (FP32 arithmetic for the refined forms at
    tile edges 128 and 256, FP64 otherwise). Asynchronous: errors are reported by gp_sync."""
    _dev(b, "b", (f.n,))
    if out is None:
        out = torch.empty(f.n, dtype=torch.float64, device=b.device)
    _dev(out, "out", (f.n,))
    _check(ctx.lib.gp_solve(ctx.h, f.h, b.data_ptr(), out.data_ptr()), "gp_solve")
    return out


def gp_predict_var(ctx: Context, f: Factor, Xs: torch.Tensor, out: torch.Tensor | None = None):
    m = Xs.shape[0]
    _dev(Xs, "Xs", (m, f.D))
    if out is None:
        out = torch.empty(m, dtype=torch.float64, device=Xs.device)
    _dev(out, "var_out", (m,))
    _check(ctx.lib.gp_predict_var(ctx.h, f.h, Xs.data_ptr(), m, out.data_ptr()), "gp_predict_var")
    return out


def gp_factor_stats(ctx: Context, f: Factor) -> dict:
    """The factor's refinement record: diagonal shift, backward error and steps of the last mean solve."""
    out = (ctypes.c_double * 4)()
    _check(ctx.lib.gp_factor_stats(ctx.h, f.h, out), "gp_factor_stats")
    return {"shift": out[0], "eta": out[1], "iterations": int(out[2]), "precision": int(out[3])}


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


def debug_tile_product(ctx: Context, precision: str, A: torch.Tensor, B: torch.Tensor, C: torch.Tensor,
                       store: bool = False, lower: bool = False, reps: int = 1) -> torch.Tensor:
    """Test hook gp_debug_tile_product: C (128 x 128) -= A B^T (store: C = A B^T) with A, B 128 x K
    through the tensor-core products of `precision`, in place on C."""
    K = A.shape[1]
    _dev(A, "A", (128, K))
    _dev(B, "B", (128, K))
    _dev(C, "C", (128, 128))
    _check(ctx.lib.gp_debug_tile_product(ctx.h, N.PRECISIONS[precision], A.data_ptr(), B.data_ptr(), C.data_ptr(),
                                         K, int(store), int(lower), reps), "gp_debug_tile_product")
    return C


def gp_predict_mean_noalloc(X: torch.Tensor, y: torch.Tensor, Xs: torch.Tensor, hyper: Hyper, out: torch.Tensor,
                            stream: torch.cuda.Stream | None = None) -> torch.Tensor:
    """Mean of a small GP (n <= 1024) through the allocation-free entry point; `out` is caller-owned."""
    n, D = X.shape
    m = Xs.shape[0]
    _dev(X, "X")
    _dev(y, "y", (n,))
    _dev(Xs, "Xs", (m, D))
    _dev(out, "mean_out", (m,))
    for t, name in ((y, "y"), (Xs, "Xs"), (out, "mean_out")):
        if t.device != X.device:
            raise ValueError(f"{name} is on {t.device}, X on {X.device}: all arrays must share one device")
    if stream is not None and stream.device != X.device:
        raise ValueError(f"stream belongs to {stream.device}, the arrays to {X.device}")
    lib = N.load()
    # the C entry point works on the current device: make it the arrays' device for the call
    with torch.cuda.device(X.device):
        stream = stream if stream is not None else torch.cuda.current_stream(X.device)
        info = ctypes.c_int64(0)
        s = lib.gp_predict_mean_noalloc(X.data_ptr(), y.data_ptr(), n, D, Hyper(*hyper).c, Xs.data_ptr(), m,
                                        out.data_ptr(), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(info))
    if s != N.GP_OK:
        raise GPError(s, info.value, "gp_predict_mean_noalloc")
    return out


def _batch_descs(gps, want_cov: bool):
    """gp_batch_desc array for entries (X, y, Xs, hyper[, tile]), with freshly allocated outputs."""
    descs = (N.gp_batch_desc * len(gps))()
    inputs, means, covs = [], [], []
    for g, e in enumerate(gps):
        X, y, Xs, hyper = e[:4]
        tile = e[4] if len(e) > 4 else 0
        n, D = X.shape
        m = Xs.shape[0]
        _dev(X, "X")
        _dev(y, "y", (n,))
        _dev(Xs, "Xs", (m, D))
        mean = torch.empty(m, dtype=torch.float64, device=X.device)
        cov = torch.empty((m, m), dtype=torch.float64, device=X.device) if want_cov else None
        inputs.append((X, y, Xs))
        means.append(mean)
        covs.append(cov)
        d = descs[g]
        d.X, d.y, d.Xs, d.n, d.m, d.D, d.tile = X.data_ptr(), y.data_ptr(), Xs.data_ptr(), n, m, D, tile
        d.h = Hyper(*hyper).c
        d.mean_out = mean.data_ptr()
        d.cov_out = cov.data_ptr() if cov is not None else None
    return descs, inputs, means, covs


def batch_predict(ctx: Context, gps, want_cov: bool = True):
    """One-shot gp_batch_predict on entries (X, y, Xs, hyper[, tile]): returns (means, covs), covs
    None per GP without want_cov. Waits for the GPU; device errors raise GPError."""
    descs, inputs, means, covs = _batch_descs(gps, want_cov)
    info = ctypes.c_int64(0)
    s = ctx.lib.gp_batch_predict(ctx.h, len(gps), descs, int(bool(want_cov)), ctypes.byref(info))
    del inputs
    if s != N.GP_OK:
        raise GPError(s, info.value, "gp_batch_predict")
    return means, covs


def _pow2_ceil(x: int) -> int:
    return 1 << max(0, int(x) - 1).bit_length()


def autotune_cache_key(gpu: str, precision: str, gps_shape, want_cov: bool, tiles=(), classes: int = 0) -> str:
    """Key of a batch in the autotuner's JSON cache: the GPU's name, the precision, whether the
    covariance is wanted, the search options, and the batch's shape in coarse buckets -- the GP count
    and, for each of the autotuner's equal-count size classes (GPs sorted by n), its largest n, both
    rounded up to powers of two; the set of input dimensions D; the largest m rounded up to a power
    of two. gps_shape: (n, m, D) per GP."""
    ns = sorted(int(n) for n, _, _ in gps_shape)
    B = len(ns)
    nc = min(classes if classes > 0 else 3, 8, B)
    nmax = [ns[(k + 1) * B // nc - 1] for k in range(nc)]
    ds = sorted({int(d) for _, _, d in gps_shape})
    mmax = max(int(m) for _, m, _ in gps_shape)
    cand = sorted({int(t) for t in tiles if t}) or [32, 64, 128, 256]
    return (f"{gpu}|{precision}|cov{int(bool(want_cov))}|tiles{cand}|B{_pow2_ceil(B)}"
            f"|n{[_pow2_ceil(x) for x in nmax]}|D{ds}|m{_pow2_ceil(mmax)}")


def tiles_from_classes(classes, ns):
    """Tile edge per GP from an autotuner class table [{"n_max", "tile"}, ...] (ascending n_max): a
    GP takes the tile of the first class whose n_max >= n, beyond the last class the last one's."""
    out = []
    for n in ns:
        t = classes[-1]["tile"]
        for c in classes:
            if n <= c["n_max"]:
                t = c["tile"]
                break
        out.append(int(t))
    return out


def batch_autotune(ctx: Context, gps, want_cov: bool = True, tiles=(), classes: int = 0, sample: int = 0,
                   reps: int = 0, cache_path: str | None = None):
    """Runs gp_batch_autotune on entries (X, y, Xs, hyper[, tile]). Returns (entries with the chosen
    tile edge appended, report dict); the chosen schedule stays in the context for later Batch()es.

    cache_path: a JSON file of earlier choices keyed by autotune_cache_key (GPU name, precision,
    batch-shape buckets). On a hit the cached class table and schedule are applied without timing
    anything (report["cached"] is True); on a miss the search runs and its choice is added to the file."""
    import json
    import os
    key = None
    if cache_path:
        shape = [(e[0].shape[0], e[2].shape[0], e[0].shape[1]) for e in gps]
        key = autotune_cache_key(torch.cuda.get_device_name(ctx.device), ctx.precision, shape, want_cov, tiles,
                                 classes)
        try:
            with open(cache_path) as fh:
                cache = json.load(fh)
        except (FileNotFoundError, ValueError):
            cache = {}
        hit = cache.get(key)
        if hit:
            if hit["default"]:  # the library's own rule won: no per-GP tile, default schedule
                tl = [0] * len(gps)
            else:
                tl = tiles_from_classes(hit["classes"], [e[0].shape[0] for e in gps])
            _check(ctx.lib.gp_set_batch_schedule(ctx.h, int(hit["order"]), int(hit["ctas_per_sm"])),
                   "gp_set_batch_schedule")
            return [tuple(e[:4]) + (t,) for e, t in zip(gps, tl)], dict(hit, cached=True)
    descs, inputs, means, covs = _batch_descs(gps, want_cov)
    o = N.gp_autotune_opts()
    for k, t in enumerate(list(tiles)[:6]):
        o.tiles[k] = int(t)
    o.classes, o.sample, o.reps = classes, sample, reps
    r = N.gp_autotune_result()
    _check(ctx.lib.gp_batch_autotune(ctx.h, len(gps), descs, ctypes.byref(o), ctypes.byref(r)), "gp_batch_autotune")
    tuned = [tuple(e[:4]) + (int(descs[g].tile),) for g, e in enumerate(gps)]
    rep = {"classes": [{"n_max": int(r.class_nmax[k]), "tile": int(r.class_tile[k]),
                        "sample_s": float(r.class_seconds[k])} for k in range(r.nclass)],
           "order": int(r.order), "ctas_per_sm": int(r.ctas_per_sm), "trials": int(r.trials),
           "seconds_tuned": float(r.seconds_tuned), "seconds_default": float(r.seconds_default),
           "seconds_spent": float(r.seconds_spent), "default": all(t[4] == 0 for t in tuned)}
    del inputs, means, covs
    if cache_path:
        try:
            with open(cache_path) as fh:
                cache = json.load(fh)
        except (FileNotFoundError, ValueError):
            cache = {}
        cache[key] = rep
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    return tuned, dict(rep, cached=False)


class Batch:
    """A gp_batch: many independent GPs assembled, factored and predicted by one captured CUDA graph
    (batched assembly, one persistent task-DAG launch, outputs). Entries are (X, y, Xs, hyper) or
    (X, y, Xs, hyper, tile); outputs are allocated here and refilled by every run()."""

    def __init__(self, ctx: Context, gps, want_cov: bool = True):
        self.ctx = ctx
        descs, self.inputs, self.means, self.covs = _batch_descs(gps, want_cov)
        self.h = ctypes.c_void_p()
        _check(ctx.lib.gp_batch_create(ctx.h, len(gps), descs, ctypes.byref(self.h)), "gp_batch_create")

    def run(self):
        _check(self.ctx.lib.gp_batch_run(self.ctx.h, self.h), "gp_batch_run")

    def free(self):
        if self.h and self.h.value:
            self.ctx.lib.gp_batch_free(self.ctx.h, self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class GPNLML(torch.autograd.Function):
    """nlml(l, v, s2) for fixed data, with the gradient from the library's blocked Cholesky adjoint.

    forward runs gp_nlml_grad once (value and gradient together); backward scales the stored gradient
    by the incoming gradient. X and y get no gradient."""

    @staticmethod
    def forward(fctx, X, y, l, v, s2, ctx):
        nl, g = gp_nlml_grad(ctx, X, y, Hyper(float(l), float(v), float(s2)))
        fctx.save_for_backward(torch.tensor(g, dtype=torch.float64, device=l.device))
        return torch.tensor(nl, dtype=torch.float64, device=l.device)

    @staticmethod
    def backward(fctx, gout):
        (g,) = fctx.saved_tensors
        g = g * gout
        return None, None, g[0], g[1], g[2], None


def nlml(X, y, l, v, s2, ctx: Context):
    """Differentiable negative log marginal likelihood in (l, v, s2) (0-d float64 tensors)."""
    return GPNLML.apply(X, y, l, v, s2, ctx)


def _adam_log_read(path: str, theta0, steps: int):
    """The complete step records of an Adam log, in order from step 0 (a torn last line, or anything
    after the first unreadable line, is dropped)."""
    import json
    recs = []
    try:
        with open(path) as fh:
            lines = fh.read().split("\n")
    except FileNotFoundError:
        return recs
    for line in lines:
        try:
            r = json.loads(line)
            ok = r["step"] == len(recs) and all(k in r for k in ("theta", "loss", "grad", "next", "adam"))
        except (ValueError, KeyError, TypeError):
            ok = False
        if not ok:
            break
        recs.append(r)
    if recs and [float(t) for t in recs[0]["theta"]] != [float(t) for t in theta0]:
        raise ValueError(f"{path}: the log starts from {recs[0]['theta']}, not from {list(theta0)}")
    return recs[:steps]


def adam_fit(loss_fn, theta0, steps: int = 50, lr: float = 0.05, floor: float = 1e-6, device=None,
             log_path: str | None = None, resume: bool = False):
    """Adam (torch.optim.Adam, beta = (0.9, 0.999), eps = 1e-8) on raw parameters, each clamped to
    >= floor after every step. loss_fn(params) takes the list of 0-d float64 parameter tensors and
    returns a differentiable 0-d loss. Returns [(theta, loss, grad)], one entry per step.

    Checkpoint and resume: with log_path, every step appends one flushed JSON line {step, theta, loss,
    grad, next, adam}, where next holds the parameters after the step and adam the optimizer's
    per-parameter state after it (JSON floats round-trip exactly). resume=True continues from the
    last complete line of an existing log (a run that was cut off, even mid-line): parameters and
    optimizer state are restored from it, so the resumed run repeats the uninterrupted run's
    trajectory bit for bit. A log that starts from other parameters raises ValueError."""
    import json
    import os
    theta0 = [float(t) for t in theta0]
    recs = _adam_log_read(log_path, theta0, steps) if (log_path and resume) else []
    start = [float(t) for t in recs[-1]["next"]] if recs else theta0
    params = [torch.tensor(t, dtype=torch.float64, device=device, requires_grad=True) for t in start]
    opt = torch.optim.Adam(params, lr=lr, betas=(0.9, 0.999), eps=1e-8)
    if recs:
        sd = opt.state_dict()
        sd["state"] = {i: {"step": torch.tensor(float(a["step"]), dtype=torch.float32),
                           "exp_avg": torch.tensor(float(a["exp_avg"]), dtype=torch.float64),
                           "exp_avg_sq": torch.tensor(float(a["exp_avg_sq"]), dtype=torch.float64)}
                       for i, a in enumerate(recs[-1]["adam"])}
        opt.load_state_dict(sd)
    hist = [([float(t) for t in r["theta"]], float(r["loss"]), [float(g) for g in r["grad"]]) for r in recs]
    fh = None
    if log_path:
        tmp = log_path + ".tmp"  # the kept records only: drops a torn tail before appending
        with open(tmp, "w") as out:
            out.writelines(json.dumps(r) + "\n" for r in recs)
        os.replace(tmp, log_path)
        fh = open(log_path, "a")
    try:
        for k in range(len(recs), steps):
            opt.zero_grad()
            loss = loss_fn(params)
            loss.backward()
            theta = [p.item() for p in params]
            grad = [p.grad.item() for p in params]
            opt.step()
            with torch.no_grad():
                for p in params:
                    p.clamp_(min=floor)
            hist.append((theta, loss.item(), grad))
            if fh:
                st = [opt.state[p] for p in params]
                rec = {"step": k, "theta": theta, "loss": loss.item(), "grad": grad, "next": [p.item() for p in params],
                       "adam": [{"step": float(s["step"]), "exp_avg": float(s["exp_avg"]),
                                 "exp_avg_sq": float(s["exp_avg_sq"])} for s in st]}
                fh.write(json.dumps(rec) + "\n")
                fh.flush()
    finally:
        if fh:
            fh.close()
    return hist


def fit_adam(ctx: Context, X, y, theta0=(0.5, 2.0, 0.5), steps: int = 50, lr: float = 0.05, floor: float = 1e-6,
             log_path: str | None = None, resume: bool = False):
    """Hyperparameter fitting of (l, v, s2) by adam_fit on the library's NLML (GPNLML: the gradient
    from the blocked Cholesky adjoint), parameters on X's device. log_path / resume: checkpoint and
    restart, as adam_fit describes. Returns [(theta, nlml, grad)]."""
    return adam_fit(lambda p: nlml(X, y, *p, ctx), theta0, steps, lr, floor, X.device, log_path, resume)


def predict(X, y, Xs, hyper=Hyper(), ctx: Context | None = None, full_cov: bool = True):
    """Convenience: assemble, factor, and predict mean (and full covariance) in one call."""
    ctx = ctx or Context(X.device.index or 0)
    f = gp_assemble(ctx, X, hyper)
    gp_cholesky(ctx, f)
    mean = gp_predict_mean(ctx, f, y, Xs)
    cov = gp_predict_full_cov(ctx, f, Xs) if full_cov else None
    gp_sync(ctx)
    return mean, cov
