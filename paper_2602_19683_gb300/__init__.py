"""GB300-native exact Gaussian-process prediction (arxiv 2602.19683's hot path).

SE-kernel covariance assembly, tiled right-looking Cholesky driven by a device-side task DAG in one
persistent kernel, and the triangular solves of the predictive mean and full covariance, all as
hand-written sm_103a CUDA behind the C ABI in include/gp.h. `api` is the thin torch binding.
"""
from .build import build as build_library  # noqa: F401
