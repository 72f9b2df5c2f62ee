"""GPU parity of the mixed-precision mode (GP_FP32) against the FP64 oracle.

In this mode the trailing SYRK/GEMM updates, the panel TRSMs after the first block column and the
covariance solve run in FP32 with FP32 accumulation; the diagonal POTRFs, the first block column's
TRSMs and the residual of the mean solve stay FP64, and classic iterative refinement recovers the
FP64 solution of K alpha = y. Stated bounds (max-abs error relative to the oracle's max-abs value),
per form of the trailing update:
                         FP32 FMA     tensor cores (tcgen05, 3xTF32)
  mean (refined)         <= 1e-10     <= 1e-10   (the FP64 bar)
  factor ||LL^T-K||/||K|| <= 1e-5     <= 2e-5
  covariance             <= 2e-5      <= 1e-4
  log-determinant        <= 1e-5      <= 1e-5 relative
The tensor-core form is looser because the tensor cores' FP32 accumulation does not round to
nearest, so its error grows with the 256-long accumulation chains.
"""
import numpy as np
import pytest
import torch

import __graft_entry__
import nfir
import oracle
from oracle import Hyper

pytestmark = pytest.mark.gpu

H0 = Hyper(1.0, 1.0, 0.1)


@pytest.fixture(scope="module")
def api():
    __graft_entry__.build()
    from paper_2602_19683_gb300 import api as A
    return A


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    d = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (d if d > 0 else 1.0))


def to_dev(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).to("cuda") for a in arrs]


BOUNDS = {False: {"factor": 1e-5, "cov": 2e-5, "logdet": 1e-5}, True: {"factor": 2e-5, "cov": 1e-4, "logdet": 1e-5}}


@pytest.mark.parametrize("tc", [False, True])
@pytest.mark.parametrize("n,m,D,T,seed", [(1024, 1024, 8, 256, 0), (1500, 300, 8, 128, 1), (700, 70, 4, 64, 2),
                                          (4096, 512, 8, 256, 3)])
def test_mixed_matches_oracle_within_stated_bounds(api, n, m, D, T, seed, tc):
    X, y, Xs, _ = nfir.make_dataset(n, m, D, seed)
    ref = oracle.gp_predict(X, y, Xs, H0)
    ctx = api.Context(0, tile=T, precision="fp32", tensor_cores=tc)
    Xd, yd, Xsd = to_dev(X, y, Xs)
    f = api.gp_assemble(ctx, Xd, api.Hyper(*H0))
    api.gp_cholesky(ctx, f)
    L = api.gp_factor_rows(ctx, f).cpu().numpy()
    mean, iters = api.gp_predict_mean(ctx, f, yd, Xsd, want_iters=True)
    cov = api.gp_predict_full_cov(ctx, f, Xsd)
    logdet = api.gp_logdet(ctx, f)
    api.gp_sync(ctx)
    fac_err = np.linalg.norm(L @ L.T - ref["K"]) / np.linalg.norm(ref["K"])
    em = rel(mean.cpu().numpy(), ref["mean"])
    ec = rel(cov.cpu().numpy(), ref["cov"])
    el = abs(logdet - ref["logdet"]) / abs(ref["logdet"])
    print(f"n={n} tc={tc}: factor {fac_err:.2e} mean {em:.2e} ({iters} IR iterations) cov {ec:.2e} logdet {el:.2e}")
    b = BOUNDS[tc and T % 128 == 0]
    assert 1 <= iters <= 10
    assert fac_err <= b["factor"]
    assert em <= 1e-10
    assert ec <= b["cov"]
    assert el <= b["logdet"]


def test_mixed_first_column_is_fp64(api):
    """With a single tile row below the diagonal (Mt = 2), every TRSM is the first block column's and
    every input of the one trailing update is FP64-exact, so only the update's FP32 rounding remains:
    the first tile column of L matches the FP64 factor to FP64 rounding."""
    X, y, Xs, _ = nfir.make_dataset(128, 4, 8, 5)
    ref = oracle.cholesky(oracle.assemble_K(X, H0))
    ctx = api.Context(0, tile=64, precision="fp32")
    (Xd,) = to_dev(X)
    f = api.gp_assemble(ctx, Xd, api.Hyper(*H0))
    api.gp_cholesky(ctx, f)
    L = api.gp_factor_rows(ctx, f).cpu().numpy()
    api.gp_sync(ctx)
    assert rel(L[:, :64], ref[:, :64]) <= 1e-13
    assert rel(L, ref) <= 1e-5
