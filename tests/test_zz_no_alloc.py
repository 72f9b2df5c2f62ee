"""The allocation-free entry point gp_predict_mean_noalloc, against the regular entry points and the oracle.

It serves callers that cannot call cudaMalloc (real-time loops, fixed device-memory budgets, hosts
that own all device memory): its workspace is one static device array shared by every call. This
file is collected last so that a failure here never stops the rest of the suite; it passes both on
its own in a fresh process and after the other tests. Two calls in a row on different data check
that each call clears the shared workspace it needs.
"""
import ctypes

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


def regular_mean(api, X, y, Xs, h):
    ctx = api.Context(0, tile=64)
    f = api.gp_assemble(ctx, X, api.Hyper(*h))
    api.gp_cholesky(ctx, f)
    mean = api.gp_predict_mean(ctx, f, y, Xs)
    api.gp_sync(ctx)
    return mean


def test_noalloc_matches_regular_path_twice(api):
    cases = [(1000, 300, 8, 0, Hyper(1.0, 1.0, 0.1)), (517, 77, 4, 3, Hyper(0.7, 1.5, 0.05))]
    for n, m, D, seed, h in cases:  # two calls in a row, different sizes and data
        X, y, Xs, _ = nfir.make_dataset(n, m, D, seed)
        Xd, yd, Xsd = (torch.from_numpy(a).cuda() for a in (X, y, Xs))
        ref = regular_mean(api, Xd, yd, Xsd, h).cpu().numpy()
        out = torch.full((m,), float("nan"), dtype=torch.float64, device="cuda")
        api.gp_predict_mean_noalloc(Xd, yd, Xsd, api.Hyper(*h), out)
        got = out.cpu().numpy()
        assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref))
        # and against the FP64 oracle directly (the two library paths share kernels)
        want = oracle.gp_predict(X, y, Xs, h)["mean"]
        assert np.max(np.abs(got - want)) <= 1e-10 * np.max(np.abs(want))


def test_noalloc_rejects_oversize_and_reports_not_pd(api):
    from paper_2602_19683_gb300 import _native as N
    lib = N.load()
    X = torch.zeros((1025, 2), dtype=torch.float64, device="cuda")
    y = torch.zeros(1025, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    s = lib.gp_predict_mean_noalloc(X.data_ptr(), y.data_ptr(), 1025, 2, N.gp_hyper(1.0, 1.0, 0.1), X.data_ptr(), 1,
                                    out.data_ptr(), None, None)
    assert s == N.GP_ERR_INVALID_ARG
    Xd = torch.tensor([[0.0], [1.0], [0.0]], dtype=torch.float64, device="cuda")
    yd = torch.ones(3, dtype=torch.float64, device="cuda")
    with pytest.raises(api.GPError) as e:
        api.gp_predict_mean_noalloc(Xd, yd, Xd, api.Hyper(1.0, 1.0, 0.0), torch.zeros(3, dtype=torch.float64,
                                                                                        device="cuda"))
    assert e.value.status == N.GP_ERR_NOT_PD and e.value.info == 3
