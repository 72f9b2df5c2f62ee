"""Seeded synthetic NFIR data: a coupled mass-spring-damper chain driven by a random force.

The paper trains and tests its GP on a coupled mass-spring-damper system in which the position of
the last mass depends non-linearly on the force applied to the first, modelled as an NFIR system
whose feature vector holds D lagged input forces (Sec. 1, Sec. 3.1). Its simulator and dataset are
not available here, so this module is a self-contained stand-in with that structure; the
simulation itself is `nfir.c` (parameters and readings documented there).

This is the one module that the oracle and the CUDA path both use. It holds none of the GP
arithmetic: no kernel evaluation, factorisation or solve.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nfir.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libnfir.so")
_lock = threading.Lock()
_lib = None


def build() -> str:
    """Compiles nfir.c into a shared library next to it (no-op when up to date)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.nfir_simulate.argtypes = [ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]
            lib.nfir_simulate.restype = None
            lib.nfir_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p]
            lib.nfir_splitmix64.restype = None
            _lib = lib
    return _lib


def splitmix64(seed: int, count: int) -> np.ndarray:
    """The first `count` SplitMix64 outputs for `seed` (uint64)."""
    out = np.empty(count, dtype=np.uint64)
    _load().nfir_splitmix64(seed & ((1 << 64) - 1), count, out.ctypes.data)
    return out


def simulate(n_samples: int, seed: int):
    """Force sequence u and noisy output y (both float64, length n_samples) of one trajectory."""
    u = np.empty(n_samples, dtype=np.float64)
    y = np.empty(n_samples, dtype=np.float64)
    if n_samples > 0:
        _load().nfir_simulate(n_samples, seed & ((1 << 64) - 1), u.ctypes.data, y.ctypes.data)
    return u, y


def features(u: np.ndarray, y: np.ndarray, D: int):
    """NFIR rows x_i = (u_i, u_{i-1}, ..., u_{i-D+1}) and targets y_i; the first D-1 samples are
    dropped so that every row has D lags."""
    n = len(u) - (D - 1)
    X = np.empty((max(n, 0), D), dtype=np.float64)
    for d in range(D):
        X[:, d] = u[D - 1 - d: D - 1 - d + n]
    return X, y[D - 1:].copy()


def make_dataset(n: int, m: int, D: int = 8, seed: int = 0):
    """(X, y, Xs, ys): n training rows from seed, m test rows from the independent seed+1."""
    X, y = features(*simulate(n + D - 1, seed), D)
    Xs, ys = features(*simulate(m + D - 1, seed + 1), D)
    return X, y, Xs, ys


def batch_sizes(B: int = 512, n_lo: int = 128, n_hi: int = 4096, seed: int = 999):
    """Uneven GP sizes for the batched workload: n_g = n_lo + floor(U * (n_hi - n_lo + 1)) and
    D_g drawn from {4, 8, 16}, from one SplitMix64 stream."""
    z = splitmix64(seed, 2 * B)
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    ns = n_lo + np.floor(u[0::2] * (n_hi - n_lo + 1)).astype(np.int64)
    Ds = np.array([4, 8, 16], dtype=np.int64)[np.minimum((u[1::2] * 3).astype(np.int64), 2)]
    return ns, Ds


def make_batch(B: int = 512, m: int = 256, n_lo: int = 128, n_hi: int = 4096, base_seed: int = 1000):
    """B independent GPs: list of (X, y, Xs, ys); GP g uses seeds base_seed+2g (train) and
    base_seed+2g+1 (test)."""
    ns, Ds = batch_sizes(B, n_lo, n_hi)
    return [make_dataset(int(ns[g]), m, int(Ds[g]), base_seed + 2 * g) for g in range(B)]
