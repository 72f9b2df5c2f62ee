"""Hyperparameter fitting loop (host side, CPU): the Adam driver of api.fit_adam against the oracle's
textbook Adam, and its checkpoint / resume. Failures are made on the host: a loss function that
raises part-way (a crashed run) and a log whose last line was torn mid-write."""
import json

import numpy as np
import pytest
import torch

import nfir
import oracle
from oracle import Hyper


@pytest.fixture(scope="module")
def api():
    from paper_2602_19683_gb300 import api as A
    return A


class _OracleNLML(torch.autograd.Function):
    """The oracle's NLML and gradient as a differentiable function of (l, v, s2) (CPU)."""

    @staticmethod
    def forward(fctx, X, y, l, v, s2):
        nl, g = oracle.nlml_and_grad(X, y, Hyper(float(l), float(v), float(s2)))
        fctx.save_for_backward(torch.tensor(np.asarray(g), dtype=torch.float64))
        return torch.tensor(nl, dtype=torch.float64)

    @staticmethod
    def backward(fctx, gout):
        (g,) = fctx.saved_tensors
        g = g * gout
        return None, None, g[0], g[1], g[2]


def _data():
    X, y, _, _ = nfir.make_dataset(40, 1, 3, 7)
    return X, y


def test_adam_driver_follows_textbook_adam(api):
    """torch.optim.Adam in the driver against the oracle's Kingma-Ba update on the same loss."""
    X, y = _data()
    theta0 = (0.5, 2.0, 0.5)
    hist = api.adam_fit(lambda p: _OracleNLML.apply(X, y, *p), theta0, steps=12)
    ref = oracle.adam(list(theta0), lambda t: oracle.nlml_and_grad(X, y, Hyper(*t)), steps=12)
    for (th, loss, g), (th_r, loss_r, g_r) in zip(hist, ref):
        assert np.allclose(th, th_r, rtol=1e-11, atol=0)
        assert abs(loss - loss_r) <= 1e-11 * abs(loss_r)


def test_adam_floor_clamps(api):
    """A parameter pushed below the floor stays at it."""
    hist = api.adam_fit(lambda p: p[0] * 100.0 + p[1] ** 2 + p[2] ** 2, (1e-6, 1.0, 1.0), steps=3)
    assert all(th[0] == 1e-6 for th, _, _ in hist)


def _smooth(p):
    """A deterministic smooth loss in three parameters (plain torch CPU ops: bitwise repeatable, which
    the oracle's thread-parallel sums are not)."""
    return 3.0 * (p[0] - 1.3) ** 2 + torch.log1p(p[1] ** 2) * (p[2] + 0.1) + torch.exp(-p[2]) + p[0] * p[1]


def test_adam_resume_after_crash_and_torn_line(api, tmp_path):
    """A run cut off by an exception at step 7, whose log then loses half of its last line, resumes to
    the uninterrupted run's trajectory and log, bit for bit."""
    theta0 = (0.5, 2.0, 0.5)
    steps = 15
    full_log = tmp_path / "full.jsonl"
    full = api.adam_fit(_smooth, theta0, steps, log_path=str(full_log))

    calls = {"n": 0}

    def crashing(p):
        calls["n"] += 1
        if calls["n"] == 8:
            raise RuntimeError("rank died")
        return _smooth(p)

    log = tmp_path / "run.jsonl"
    with pytest.raises(RuntimeError):
        api.adam_fit(crashing, theta0, steps, log_path=str(log))
    lines = log.read_text().splitlines()
    assert len(lines) == 7
    log.write_text("\n".join(lines[:6]) + "\n" + lines[6][: len(lines[6]) // 2])  # torn mid-write
    resumed = api.adam_fit(_smooth, theta0, steps, log_path=str(log), resume=True)
    assert resumed == full
    assert log.read_text() == full_log.read_text()
    # resuming a finished log computes nothing
    done = api.adam_fit(lambda p: (_ for _ in ()).throw(AssertionError("no step expected")), theta0, steps,
                        log_path=str(log), resume=True)
    assert done == full


def test_adam_resume_rejects_a_foreign_log(api, tmp_path):
    log = tmp_path / "other.jsonl"
    api.adam_fit(lambda p: p[0] ** 2 + p[1] ** 2 + p[2] ** 2, (1.0, 1.0, 1.0), 2, log_path=str(log))
    with pytest.raises(ValueError):
        api.adam_fit(lambda p: p[0] ** 2 + p[1] ** 2 + p[2] ** 2, (2.0, 1.0, 1.0), 4, log_path=str(log), resume=True)
    rec = json.loads(log.read_text().splitlines()[0])
    assert rec["step"] == 0 and rec["theta"] == [1.0, 1.0, 1.0]
