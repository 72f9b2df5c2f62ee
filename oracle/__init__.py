"""FP64 CPU oracle for exact GP prediction -- TEST INFRASTRUCTURE ONLY.

This package is the independent reference that the CUDA library is checked against. It is plain
C (``gp_oracle.c``) driven through ctypes, written from the paper's definitions: the SE kernel
(Eq. 1), the predictive mean (Eq. 2) and covariance (Eq. 3) by the paper's solve recipe (Sec. 3.1),
the Cholesky factor by the unblocked definition and by the tiled right-looking algorithm of
Sec. 3.2 (Fig. 1), and the marginal likelihood with its gradient from Rasmussen & Williams (2006),
which the paper cites for the kernel.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import it.
It shares no code with the CUDA path and never calls it.

Every function here is pinned by tests under ``tests/test_oracle_*.py`` (closed forms, invariants,
brute force, LAPACK cross-checks, finite differences); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from typing import NamedTuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gp_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libgp_oracle.so")
_lock = threading.Lock()
_lib = None


class Hyper(NamedTuple):
    """SE hyperparameters: lengthscale l, vertical scale v, noise variance s2 (Sec. 3.1)."""
    l: float = 1.0
    v: float = 1.0
    s2: float = 0.1


def build() -> str:
    """Compiles gp_oracle.c (gcc, OpenMP, no fused multiply-add contraction)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _lib_handle():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
            sig = {
                "oracle_assemble_K": ([P, I64, I32, D, D, D, P], None),
                "oracle_assemble_cross": ([P, I64, P, I64, I32, D, D, P], None),
                "oracle_assemble_prior": ([P, I64, I32, D, D, D, P], None),
                "oracle_kernel_entries": ([P, P, I32, D, D, D, I64, P, P, P, P], None),
                "oracle_kernel_rows_matvec": ([P, I64, I32, D, D, D, I64, P, P, P], None),
                "oracle_cholesky": ([P, I64], ctypes.c_int),
                "oracle_cholesky_tiled": ([P, I64, I64], ctypes.c_int),
                "oracle_forward": ([P, I64, P, I64, P], None),
                "oracle_backward": ([P, I64, P, P], None),
                "oracle_predict_mean": ([P, I64, P, P, I64, P, P], None),
                "oracle_predict_cov": ([P, I64, P, P, I64, P, P], None),
                "oracle_logdet": ([P, I64], D),
                "oracle_nlml": ([P, I64, P, P], D),
                "oracle_kinv": ([P, I64, P], None),
                "oracle_nlml_grad": ([P, I64, I32, D, D, P, P, P], None),
            }
            for name, (args, res) in sig.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


def _c(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a):
    return a.ctypes.data


class NotPositiveDefinite(ArithmeticError):
    """The Cholesky pivot of 1-based column `info` was not positive."""

    def __init__(self, info: int):
        super().__init__(f"matrix not positive definite at column {info}")
        self.info = info


# ---------------------------------------------------------------- Eq. (1)

def assemble_K(X, h: Hyper) -> np.ndarray:
    X = _c(X)
    n, D = X.shape
    K = np.empty((n, n))
    _lib_handle().oracle_assemble_K(_p(X), n, D, h.l, h.v, h.s2, _p(K))
    return K


def assemble_cross(A, B, h: Hyper) -> np.ndarray:
    """K_{A,B}: no noise term (different point sets)."""
    A, B = _c(A), _c(B)
    out = np.empty((A.shape[0], B.shape[0]))
    _lib_handle().oracle_assemble_cross(_p(A), A.shape[0], _p(B), B.shape[0], A.shape[1], h.l, h.v, _p(out))
    return out


def assemble_prior(Xs, h: Hyper, noisy: bool = False) -> np.ndarray:
    """K_{Xs,Xs}; the latent covariance by default, + s2 I when noisy."""
    Xs = _c(Xs)
    out = np.empty((Xs.shape[0], Xs.shape[0]))
    _lib_handle().oracle_assemble_prior(_p(Xs), Xs.shape[0], Xs.shape[1], h.l, h.v, h.s2 if noisy else 0.0, _p(out))
    return out


def kernel_entries(A, B, ia, ib, same, h: Hyper) -> np.ndarray:
    """Entries k(A[ia[t]], B[ib[t]]) (+ s2 where same[t])."""
    A, B = _c(A), _c(B)
    ia, ib = _c(ia, np.int64), _c(ib, np.int64)
    same = _c(same, np.int32)
    out = np.empty(len(ia))
    _lib_handle().oracle_kernel_entries(_p(A), _p(B), A.shape[1], h.l, h.v, h.s2, len(ia), _p(ia), _p(ib),
                                        _p(same), _p(out))
    return out


def kernel_rows_matvec(X, rows, w, h: Hyper) -> np.ndarray:
    """(K w)[rows] with the kernel entries recomputed from X."""
    X, w = _c(X), _c(w)
    rows = _c(rows, np.int64)
    out = np.empty(len(rows))
    _lib_handle().oracle_kernel_rows_matvec(_p(X), X.shape[0], X.shape[1], h.l, h.v, h.s2, len(rows), _p(rows),
                                            _p(w), _p(out))
    return out


# ---------------------------------------------------------------- Cholesky

def cholesky(K) -> np.ndarray:
    """Lower L with L L^T = K, unblocked right-looking definition. Raises NotPositiveDefinite."""
    L = np.array(K, dtype=np.float64, order="C", copy=True)
    info = _lib_handle().oracle_cholesky(_p(L), L.shape[0])
    if info:
        raise NotPositiveDefinite(info)
    return L


def cholesky_tiled(K, T: int) -> np.ndarray:
    """Lower L by the paper's tiled right-looking algorithm (Fig. 1) with tile edge T."""
    L = np.array(K, dtype=np.float64, order="C", copy=True)
    info = _lib_handle().oracle_cholesky_tiled(_p(L), L.shape[0], int(T))
    if info:
        raise NotPositiveDefinite(info)
    return L


def forward(L, b) -> np.ndarray:
    L = _c(L)
    b = _c(b)
    B = b.reshape(b.shape[0], -1)
    x = np.empty_like(B)
    _lib_handle().oracle_forward(_p(L), L.shape[0], _p(B), B.shape[1], _p(x))
    return x.reshape(b.shape)


def backward(L, b) -> np.ndarray:
    L, b = _c(L), _c(b)
    x = np.empty_like(b)
    _lib_handle().oracle_backward(_p(L), L.shape[0], _p(b), _p(x))
    return x


# ---------------------------------------------------------------- Eqs. (2), (3)

def predict_mean(L, y, Kxs):
    """(alpha, mean) with alpha = K^{-1} y by two substitutions and mean = K_{Xs,X} alpha (Eq. 2)."""
    L, y, Kxs = _c(L), _c(y), _c(Kxs)
    n, m = L.shape[0], Kxs.shape[0]
    alpha, mean = np.empty(n), np.empty(m)
    _lib_handle().oracle_predict_mean(_p(L), n, _p(y), _p(Kxs), m, _p(alpha), _p(mean))
    return alpha, mean


def predict_cov(L, Kxs, Kss):
    """(V, cov) with L V = K_{X,Xs} and cov = K_{Xs,Xs} - V^T V (Eq. 3)."""
    L, Kxs, Kss = _c(L), _c(Kxs), _c(Kss)
    n, m = L.shape[0], Kxs.shape[0]
    V, cov = np.empty((n, m)), np.empty((m, m))
    _lib_handle().oracle_predict_cov(_p(L), n, _p(Kxs), _p(Kss), m, _p(V), _p(cov))
    return V, cov


def logdet(L) -> float:
    L = _c(L)
    return _lib_handle().oracle_logdet(_p(L), L.shape[0])


def nlml(L, y, alpha) -> float:
    L, y, alpha = _c(L), _c(y), _c(alpha)
    return _lib_handle().oracle_nlml(_p(L), L.shape[0], _p(y), _p(alpha))


def kinv(L) -> np.ndarray:
    L = _c(L)
    out = np.empty_like(L)
    _lib_handle().oracle_kinv(_p(L), L.shape[0], _p(out))
    return out


def nlml_grad_terms(X, h: Hyper, Kinv, alpha) -> np.ndarray:
    X, Kinv, alpha = _c(X), _c(Kinv), _c(alpha)
    g = np.empty(3)
    _lib_handle().oracle_nlml_grad(_p(X), X.shape[0], X.shape[1], h.l, h.v, _p(Kinv), _p(alpha), _p(g))
    return g


# ---------------------------------------------------------------- end-to-end helpers

def gp_predict(X, y, Xs, h: Hyper, tile: int | None = None, noisy_prior: bool = False):
    """Full pipeline: K, L (tiled if `tile`), alpha, mean, V and covariance. Returns a dict."""
    K = assemble_K(X, h)
    L = cholesky_tiled(K, tile) if tile else cholesky(K)
    Kxs = assemble_cross(Xs, X, h)
    Kss = assemble_prior(Xs, h, noisy_prior)
    alpha, mean = predict_mean(L, y, Kxs)
    V, cov = predict_cov(L, Kxs, Kss)
    return {"K": K, "L": L, "Kxs": Kxs, "Kss": Kss, "alpha": alpha, "mean": mean, "V": V, "cov": cov,
            "logdet": logdet(L)}


def nlml_and_grad(X, y, h: Hyper):
    """(nlml, grad[3]) at h; grad w.r.t. (l, v, s2)."""
    K = assemble_K(X, h)
    L = cholesky(K)
    alpha, _ = predict_mean(L, y, np.zeros((0, X.shape[0])))
    return nlml(L, y, alpha), nlml_grad_terms(X, h, kinv(L), alpha)


def adam(theta0, grad_fn, steps: int, lr: float = 0.05, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8,
         floor: float = 1e-6):
    """Textbook Adam (Kingma & Ba 2015) on the raw parameters, each clamped to >= floor after the
    update. grad_fn(theta) -> (loss, grad). Returns the list of (theta, loss, grad) per step."""
    theta = np.array(theta0, dtype=np.float64)
    m1 = np.zeros_like(theta)
    m2 = np.zeros_like(theta)
    hist = []
    for t in range(1, steps + 1):
        loss, g = grad_fn(theta)
        g = np.asarray(g, dtype=np.float64)
        hist.append((theta.copy(), float(loss), g.copy()))
        m1 = b1 * m1 + (1 - b1) * g
        m2 = b2 * m2 + (1 - b2) * g * g
        mhat = m1 / (1 - b1 ** t)
        vhat = m2 / (1 - b2 ** t)
        theta = np.maximum(theta - lr * mhat / (np.sqrt(vhat) + eps), floor)
    return hist


LOG_2PI = math.log(2.0 * math.pi)
