"""Covariance-entry evaluation (Eq. 1) on the GPU: the table-driven exponential and the exact
fixed-point squared distances of the assembly kernels.

Pins: (1) the exponential within one ulp of CUDA's exp (torch.exp on the device) and of the host's
libm exp over [-745.2, 0], the subnormal range and tiny arguments, and the special values; (2) K, the
predictive mean and the covariance element by element against the FP64 oracle at the FP64 bars, on
inputs that take the fixed-point distances (every coordinate within 64 lengthscales) and on inputs
that take the FP64 fallback (coordinates far from the lengthscale: a large offset, a small
lengthscale; a dimension without an unrolled kernel); (3) test points of a larger range than the
training points (the common scale of both sets).
"""
import numpy as np
import pytest
import torch

import __graft_entry__
import nfir
import oracle
from oracle import Hyper

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    __graft_entry__.build()
    from paper_2602_19683_gb300 import api as A
    return A


def ulp_diff(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Distance in units in the last place between non-negative doubles (their bit patterns)."""
    return np.abs(a.view(np.int64) - b.view(np.int64))


@pytest.mark.parametrize("lo,hi", [(-745.2, 0.0), (-1.0, 0.0), (-40.0, -1.0), (-745.13, -700.0), (-1e-9, 0.0)])
def test_exp_within_one_ulp_of_cuda_and_libm(api, lo, hi):
    ctx = api.Context(0)
    x = torch.linspace(lo, hi, 1 << 21, dtype=torch.float64, device="cuda")
    ours = api.debug_exp_neg(ctx, x)
    ref_cuda = torch.exp(x)
    api.gp_sync(ctx)
    o, rc = ours.cpu().numpy(), ref_cuda.cpu().numpy()
    rl = np.exp(x.cpu().numpy())
    d_cuda, d_libm = int(ulp_diff(o, rc).max()), int(ulp_diff(o, rl).max())
    print(f"[{lo}, {hi}]: max ulp difference vs CUDA exp {d_cuda}, vs libm exp {d_libm}")
    assert d_cuda <= 1 and d_libm <= 1


def test_exp_special_values(api):
    ctx = api.Context(0)
    x = torch.tensor([float("nan"), float("-inf"), -0.0, 0.0, -746.0, -745.25, -1e-300, -708.5],
                     dtype=torch.float64, device="cuda")
    o = api.debug_exp_neg(ctx, x).cpu().numpy()
    api.gp_sync(ctx)
    assert np.isnan(o[0])
    assert o[1] == 0.0 and o[4] == 0.0 and o[5] == 0.0
    assert o[2] == 1.0 and o[3] == 1.0 and o[6] == 1.0
    assert ulp_diff(o[7:8], np.exp(np.array([-708.5]))).max() <= 1  # subnormal result


def to_dev(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).to("cuda") for a in arrs]


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    d = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (d if d > 0 else 1.0))


CASES = [
    # name, D, hyper, transform of X, transform of Xs
    ("fixed-point", 8, Hyper(1.0, 1.0, 0.1), lambda X: X, lambda Xs: Xs),
    ("fixed-point, small l", 8, Hyper(0.05, 1.3, 0.2), lambda X: X, lambda Xs: Xs),
    ("fixed-point, wider test range", 16, Hyper(0.8, 1.0, 0.1), lambda X: X, lambda Xs: 3.0 * Xs),
    ("fixed-point, D = 4", 4, Hyper(1.2, 0.7, 0.05), lambda X: X, lambda Xs: Xs),
    ("FP64: offset 1000", 8, Hyper(1.0, 1.0, 0.1), lambda X: X + 1000.0, lambda Xs: Xs + 1000.0),
    ("FP64: lengthscale below range / 64", 8, Hyper(0.01, 1.0, 0.1), lambda X: X, lambda Xs: Xs),
    ("FP64: D = 5", 5, Hyper(1.0, 1.0, 0.1), lambda X: X, lambda Xs: Xs),
]


@pytest.mark.parametrize("name,D,h,fx,fxs", CASES, ids=[c[0] for c in CASES])
def test_assembly_and_prediction_match_oracle(api, name, D, h, fx, fxs):
    n, m, T = 1000, 300, 128
    X, y, Xs, _ = nfir.make_dataset(n, m, D, 21)
    X, Xs = fx(X), fxs(Xs)
    ref = oracle.gp_predict(X, y, Xs, h)
    ctx = api.Context(0, tile=T)
    Xd, yd, Xsd = to_dev(X, y, Xs)
    f = api.gp_assemble(ctx, Xd, api.Hyper(*h))
    K = api.gp_factor_rows(ctx, f).cpu().numpy()
    api.gp_cholesky(ctx, f)
    mean = api.gp_predict_mean(ctx, f, yd, Xsd).cpu().numpy()
    cov = api.gp_predict_full_cov(ctx, f, Xsd).cpu().numpy()
    api.gp_sync(ctx)
    ek, em, ec = rel(K, np.tril(ref["K"])), rel(mean, ref["mean"]), rel(cov, ref["cov"])
    print(f"{name}: K {ek:.2e} mean {em:.2e} cov {ec:.2e}")
    assert ek <= 1e-14
    assert em <= 1e-10 and ec <= 1e-9
    f.free()
