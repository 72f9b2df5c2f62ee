"""The FP32 blocked triangular solves (Eq. 2's two substitutions with the factor's FP32 copy): the
correction solves of the refined precision forms, run by the solve kernel (G persistent CTAs, one per SM
unless the context fixes fewer, CTA c owning tile rows c, c + G, ...; tiles streamed by bulk copies).

Pins: (1) the solve's normwise backward error on the GPU's own factor L~ (read back, rounded to FP32 as
the kernel reads it), ||b - L~ L~^T x|| <= 2 n u32 (|L~| |L~^T| |x| + |b|), the worst-case bound of two
FP32 substitutions (gamma_n per sweep), independent of the conditioning of K: a wrong tile, index, mask
or sign gives O(1); (2) the refined mean and alpha of the same factorisations against the FP64 oracle at
the FP64 bars. Shapes reach every branch of the kernel: more tile rows than CTAs (each owning several),
fewer tile rows than SMs, a single tile, ragged tails, both tile edges (128, 256). The FP64 forms'
solve (the DAG kernel's chunked FP64 tasks) is checked at the FP64 bars. A withheld block makes the
kernel's bounded waits expire: the call ends with GP_ERR_TIMEOUT and the GPU stays usable.
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
U32 = 2.0 ** -24


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


CASES = [
    # n, T, CTAs (0: one per SM), precision form, seed; tile rows Mt = ceil(n / T)
    (3000, 128, 5, "fp32", 0),     # Mt = 24 on 5 CTAs: four or five rows each; ragged tail of 56
    (2100, 128, 0, "bf16x6", 1),   # Mt = 17, fewer rows than SMs; ragged
    (2560, 256, 3, "fp32", 2),     # Mt = 10 on 3 CTAs, no tail
    (700, 256, 2, "tf32", 3),      # Mt = 3 on 2 CTAs, ragged; shifted factor, GMRES refinement
    (1500, 128, 4, "bf16x3", 4),   # Mt = 12 on 4 CTAs, ragged
    (100, 128, 0, "fp32", 5),      # a single tile
]


def factor_f32(api, ctx, f):
    return api.gp_factor_rows(ctx, f).cpu().numpy().astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("n,T,grid,prec,seed", CASES)
def test_fp32_solve_backward_error_and_refined_mean(api, n, T, grid, prec, seed):
    m, D = 16, 8
    X, y, Xs, _ = nfir.make_dataset(n, m, D, seed)
    ctx = api.Context(0, tile=T, grid=grid, precision=prec)
    Xd, yd, Xsd = to_dev(X, y, Xs)
    f = api.gp_assemble(ctx, Xd, api.Hyper(*H0))
    api.gp_cholesky(ctx, f)
    Lf = factor_f32(api, ctx, f)
    rng = np.random.default_rng(seed)
    b = rng.standard_normal(n)
    (bd,) = to_dev(b)
    x = api.gp_solve(ctx, f, bd).cpu().numpy()
    mean = api.gp_predict_mean(ctx, f, yd, Xsd).cpu().numpy()
    alpha = api.gp_alpha(ctx, f).cpu().numpy()
    api.gp_sync(ctx)
    r = b - Lf @ (Lf.T @ x)
    scale = np.abs(Lf) @ (np.abs(Lf.T) @ np.abs(x)) + np.abs(b)
    eta = float(np.max(np.abs(r) / scale))
    K = oracle.assemble_K(X, H0)
    alpha_ref, mean_ref = oracle.predict_mean(oracle.cholesky(K), y, oracle.assemble_cross(Xs, X, H0))
    ea, em = rel(alpha, alpha_ref), rel(mean, mean_ref)
    print(f"{prec} n={n} T={T} grid={grid}: FP32 solve backward error {eta:.2e} (bar {2 * n * U32:.1e}); "
          f"refined alpha {ea:.2e} mean {em:.2e}")
    assert eta <= 2 * n * U32
    assert ea <= 1e-10 and em <= 1e-10
    f.free()


@pytest.mark.parametrize("prec,T", [("fp64", 128), ("fp64", 96), ("fp64_ozaki", 128)])
def test_fp64_solve_matches_oracle(api, prec, T):
    n = 1500
    X, _, _, _ = nfir.make_dataset(n, 1, 8, 7)
    b = np.random.default_rng(7).standard_normal(n)
    ctx = api.Context(0, tile=T, precision=prec)
    (Xd, bd) = to_dev(X, b)
    f = api.gp_assemble(ctx, Xd, api.Hyper(*H0))
    api.gp_cholesky(ctx, f)
    x = api.gp_solve(ctx, f, bd).cpu().numpy()
    api.gp_sync(ctx)
    L = oracle.cholesky(oracle.assemble_K(X, H0))
    x_ref = oracle.backward(L, oracle.forward(L, b))
    assert rel(x, x_ref) <= 1e-10


def test_fp32_solve_repeated_calls_agree(api):
    """Same factor, same right-hand side: the solve is deterministic (fixed summation order per block)."""
    X, y, _, _ = nfir.make_dataset(2000, 1, 8, 9)
    ctx = api.Context(0, tile=128, grid=3, precision="fp32")
    Xd, yd = to_dev(X, y)
    f = api.gp_assemble(ctx, Xd, api.Hyper(*H0))
    api.gp_cholesky(ctx, f)
    outs = [api.gp_solve(ctx, f, yd).cpu().numpy() for _ in range(3)]
    api.gp_sync(ctx)
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def test_withheld_solve_block_times_out_and_context_survives(api):
    X, y, Xs, _ = nfir.make_dataset(1024, 8, 8, 12)
    Xd, yd, Xsd = to_dev(X, y, Xs)
    ctx = api.Context(0, tile=128, precision="fp32", timeout_s=0.2, withhold_solve_block=2)
    f = api.gp_assemble(ctx, Xd, api.Hyper(*H0))
    api.gp_cholesky(ctx, f)
    api.gp_solve(ctx, f, yd)
    with pytest.raises(api.GPError) as e:
        api.gp_sync(ctx)
    assert e.value.status == 6
    ctx2 = api.Context(0, tile=128, precision="fp32")
    f2 = api.gp_assemble(ctx2, Xd, api.Hyper(*H0))
    api.gp_cholesky(ctx2, f2)
    mean = api.gp_predict_mean(ctx2, f2, yd, Xsd).cpu().numpy()
    api.gp_sync(ctx2)
    K = oracle.assemble_K(X, H0)
    _, mean_ref = oracle.predict_mean(oracle.cholesky(K), y, oracle.assemble_cross(Xs, X, H0))
    assert rel(mean, mean_ref) <= 1e-10
