"""One tensor-core tile product C -= A B^T (the trailing SYRK/GEMM update of Sec. 3.2) in every operand
form, through the library's own packing and tcgen05 routines (test hook gp_debug_tile_product),
against the exact product.

The reference is exact: each FP64 product a b is split (Veltkamp/Dekker) into four exact partial
products and every entry is summed with math.fsum, so the only error left is the form's own.
Bars, as max |C - C_exact| over max_ij sum_k |a_ik b_jk| (plus, where C is updated, half an FP64 unit
in the last place of the stored result, the rounding of the subtraction itself):
  GP_FP64_OZAKI: no worse than the FP64 product of the same operands (numpy's BLAS DGEMM, measured
  against the same exact result) or 2^-53, whichever is larger: it is an FP64 product;
  GP_FP32 (3xTF32) <= 2e-6, GP_BF16X6 <= 2e-6 (FP32-class), GP_BF16X3 <= 1e-4, GP_TF32 <= 2e-3,
  GP_BF16 <= 2e-2 (one product of 11 / 8 significant bits).
"""
import math

import numpy as np
import pytest
import torch

import __graft_entry__

pytestmark = pytest.mark.gpu

BARS = {"fp64_ozaki": 2.0 ** -53, "fp32": 2e-6, "bf16x6": 2e-6, "bf16x3": 1e-4, "tf32": 2e-3, "bf16": 2e-2}


def bar(prec, scale, fp64_err):
    """Allowed absolute error of a form (fp64_err: the FP64 BLAS product's error on the same inputs)."""
    b = BARS[prec] * scale
    return max(b, fp64_err) if prec == "fp64_ozaki" else b


@pytest.fixture(scope="module")
def api():
    __graft_entry__.build()
    from paper_2602_19683_gb300 import api as A
    return A


def exact_product(A, B):
    """A B^T with every entry rounded once from the exact sum (Dekker split + fsum)."""
    def split(x):
        c = 134217729.0 * x
        hi = c - (c - x)
        return hi, x - hi
    ah, al = split(A)
    bh, bl = split(B)
    out = np.empty((A.shape[0], B.shape[0]))
    for i in range(A.shape[0]):
        terms = np.concatenate([ah[i] * bh, ah[i] * bl, al[i] * bh, al[i] * bl], axis=1)  # (n, 4K), all exact
        for j in range(B.shape[0]):
            out[i, j] = math.fsum(terms[j])
    return out


def operands(K, seed, kind="normal"):
    rng = np.random.default_rng(seed)
    if kind == "normal":
        A, B = rng.standard_normal((128, K)), rng.standard_normal((128, K))
    else:  # rows of a Cholesky-like factor: norms <= 1, entries of very different size
        A = rng.standard_normal((128, K)) * np.exp(rng.uniform(-12, 0, (128, K)))
        B = rng.standard_normal((128, K)) * np.exp(rng.uniform(-12, 0, (128, K)))
        A /= np.linalg.norm(A, axis=1, keepdims=True) * 1.01
        B /= np.linalg.norm(B, axis=1, keepdims=True) * 1.01
    return A, B


@pytest.mark.parametrize("prec", list(BARS))
@pytest.mark.parametrize("K,kind", [(128, "normal"), (512, "normal"), (256, "factor")])
def test_tile_product_matches_exact(api, prec, K, kind):
    A, B = operands(K, 17 + K, kind)
    C0 = np.random.default_rng(5).standard_normal((128, 128))
    ctx = api.Context(0)
    Ad, Bd = (torch.from_numpy(x).cuda() for x in (A, B))
    C = torch.from_numpy(C0.copy()).cuda()
    api.debug_tile_product(ctx, prec, Ad, Bd, C)
    exact = exact_product(A, B)
    scale = float(np.max(np.abs(A) @ np.abs(B).T))
    got = C.cpu().numpy()
    rounding = 2.0 ** -53 * float(np.max(np.abs(got)))
    err = float(np.max(np.abs((C0 - got) - exact)))
    c64 = C0 - A @ B.T
    err64 = float(np.max(np.abs((C0 - c64) - exact)))
    print(f"{prec} K={K} {kind}: max error {err / scale:.3e} of sum|ab| (FP64 BLAS {err64 / scale:.3e}; bar "
          f"{bar(prec, scale, err64) / scale:.1e}; output rounding {rounding / scale:.1e})")
    assert err <= bar(prec, scale, err64) + rounding


@pytest.mark.parametrize("prec", list(BARS))
def test_tile_product_store_and_lower(api, prec):
    A, B = operands(128, 3)
    ctx = api.Context(0)
    Ad, Bd = (torch.from_numpy(x).cuda() for x in (A, B))
    exact = exact_product(A, B)
    scale = float(np.max(np.abs(A) @ np.abs(B).T))
    err64 = float(np.max(np.abs(A @ B.T - exact)))
    C = torch.full((128, 128), 7.0, dtype=torch.float64, device="cuda")
    api.debug_tile_product(ctx, prec, Ad, Bd, C, store=True)
    assert float(np.max(np.abs(C.cpu().numpy() - exact))) <= bar(prec, scale, err64) + 2.0 ** -53 * scale
    C0 = np.random.default_rng(9).standard_normal((128, 128))
    C = torch.from_numpy(C0.copy()).cuda()
    api.debug_tile_product(ctx, prec, Ad, Bd, C, lower=True)
    got = C.cpu().numpy()
    iu = np.triu_indices(128, 1)
    assert np.array_equal(got[iu], C0[iu])  # above the diagonal: untouched
    il = np.tril_indices(128)
    rounding = 2.0 ** -53 * float(np.max(np.abs(got)))
    assert float(np.max(np.abs((C0 - got)[il] - exact[il]))) <= bar(prec, scale, err64) + rounding


def test_tile_product_rates(api):
    """Throughput of one CTA (one SM) per form, for the record (no bar)."""
    K, reps = 512, 40
    A, B = operands(K, 1)
    ctx = api.Context(0)
    Ad, Bd = (torch.from_numpy(x).cuda() for x in (A, B))
    C = torch.zeros((128, 128), dtype=torch.float64, device="cuda")
    prods = {"fp32": 3, "tf32": 1, "bf16": 1, "bf16x3": 3, "bf16x6": 6, "fp64_ozaki": 28}
    for prec in BARS:
        api.debug_tile_product(ctx, prec, Ad, Bd, C, reps=2)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        api.debug_tile_product(ctx, prec, Ad, Bd, C, reps=reps)
        e1.record(ctx.stream)
        e1.synchronize()
        s = e0.elapsed_time(e1) / 1e3
        alg = 2.0 * 128 * 128 * K * reps
        print(f"{prec}: {s / reps * 1e6:.1f} us per 128x128x{K} product; algorithmic {alg / s / 1e12:.3f} TFLOP/s "
              f"per SM, tensor pipe {prods[prec] * alg / s / 1e12:.2f} TFLOP/s per SM")
