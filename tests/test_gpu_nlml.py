"""GPU parity of the NLML and its gradient (blocked Cholesky adjoint + recomputed dK) against the
FP64 oracle (R&W 2006 Eqs. 2.30, 5.9 with K^{-1} formed explicitly), central differences, and the
oracle's Adam trajectory. Bars: FP64 nlml 1e-12 relative, gradient 1e-8 relative to its largest
component; mixed precision gradient 1e-4."""
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


def dev(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


@pytest.mark.parametrize("n,D,T,h,seed", [(1, 3, 32, Hyper(0.8, 1.7, 0.3), 0), (2, 1, 32, Hyper(0.8, 1.0, 0.1), 1),
                                          (300, 8, 64, Hyper(0.7, 1.4, 0.2), 2), (1024, 8, 256, Hyper(1.0, 1.0, 0.1), 3),
                                          (777, 4, 96, Hyper(1.3, 0.6, 0.05), 4)])
def test_nlml_grad_matches_oracle(api, n, D, T, h, seed):
    X, y, _, _ = nfir.make_dataset(n, 1, D, seed)
    nl_ref, g_ref = oracle.nlml_and_grad(X, y, h)
    ctx = api.Context(0, tile=T)
    Xd, yd = dev(X, y)
    nl, g = api.gp_nlml_grad(ctx, Xd, yd, api.Hyper(*h))
    assert abs(nl - nl_ref) <= 1e-12 * max(1.0, abs(nl_ref))
    scale = max(np.max(np.abs(g_ref)), 1e-300)
    assert np.max(np.abs(np.array(g) - g_ref)) <= 1e-8 * scale, (g, g_ref)


def test_nlml_grad_central_differences(api):
    X, y, _, _ = nfir.make_dataset(400, 1, 8, 7)
    h = Hyper(0.9, 1.2, 0.15)
    ctx = api.Context(0, tile=64)
    Xd, yd = dev(X, y)
    _, g = api.gp_nlml_grad(ctx, Xd, yd, api.Hyper(*h))
    step = 1e-5
    for k in range(3):
        hp, hm = list(h), list(h)
        hp[k] += step
        hm[k] -= step
        fd = (api.gp_nlml_grad(ctx, Xd, yd, api.Hyper(*hp))[0] - api.gp_nlml_grad(ctx, Xd, yd, api.Hyper(*hm))[0]) / (2 * step)
        assert g[k] == pytest.approx(fd, rel=1e-6, abs=1e-6)


def test_nlml_grad_mixed_precision(api):
    X, y, _, _ = nfir.make_dataset(1024, 1, 8, 8)
    h = Hyper(1.0, 1.0, 0.1)
    nl_ref, g_ref = oracle.nlml_and_grad(X, y, h)
    ctx = api.Context(0, tile=128, precision="fp32")
    Xd, yd = dev(X, y)
    nl, g = api.gp_nlml_grad(ctx, Xd, yd, api.Hyper(*h))
    assert abs(nl - nl_ref) <= 1e-5 * abs(nl_ref)
    assert np.max(np.abs(np.array(g) - g_ref)) <= 1e-4 * np.max(np.abs(g_ref))


def test_autograd_function_and_adam_trajectory(api):
    """torch.autograd through GPNLML gives the library's gradient, and five Adam steps from
    (0.5, 2.0, 0.5) follow the oracle's Adam trajectory."""
    X, y, _, _ = nfir.make_dataset(256, 1, 8, 9)
    ctx = api.Context(0, tile=64)
    Xd, yd = dev(X, y)
    l, v, s2 = (torch.tensor(t, dtype=torch.float64, device="cuda", requires_grad=True) for t in (0.5, 2.0, 0.5))
    loss = api.nlml(Xd, yd, l, v, s2, ctx)
    loss.backward()
    _, g = api.gp_nlml_grad(ctx, Xd, yd, api.Hyper(0.5, 2.0, 0.5))
    assert [float(l.grad), float(v.grad), float(s2.grad)] == pytest.approx(g, rel=1e-14)
    hist = api.fit_adam(ctx, Xd, yd, (0.5, 2.0, 0.5), steps=5)
    ref = oracle.adam([0.5, 2.0, 0.5], lambda t: oracle.nlml_and_grad(X, y, Hyper(*t)), steps=5)
    for (th, loss_, _), (th_r, loss_r, _) in zip(hist, ref):
        assert np.allclose(th, th_r, rtol=1e-9, atol=0)
        assert loss_ == pytest.approx(loss_r, rel=1e-11)


def test_adam_checkpoint_resume_on_the_library_gradient(api, tmp_path):
    """fit_adam with a JSONL checkpoint: a run stopped after 3 of 6 steps and resumed from its log
    repeats the uninterrupted run bit for bit (the FP64 gradient is run-to-run bit-identical)."""
    X, y, _, _ = nfir.make_dataset(256, 1, 8, 9)
    ctx = api.Context(0, tile=64)
    Xd, yd = dev(X, y)
    full = api.fit_adam(ctx, Xd, yd, (0.5, 2.0, 0.5), steps=6, log_path=str(tmp_path / "full.jsonl"))
    log = str(tmp_path / "run.jsonl")
    api.fit_adam(ctx, Xd, yd, (0.5, 2.0, 0.5), steps=3, log_path=log)
    resumed = api.fit_adam(ctx, Xd, yd, (0.5, 2.0, 0.5), steps=6, log_path=log, resume=True)
    assert resumed == full
