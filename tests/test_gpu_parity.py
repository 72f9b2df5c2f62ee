"""GPU parity of the FP64 path against the FP64 oracle, through the C ABI.

Bars (from the method's stated accuracy): the factor reconstructs K to ||LL^T - K||_F/||K||_F <= 1e-13;
the predictive mean (Eq. 2) agrees to <= 1e-10 and the covariance (Eq. 3) to <= 1e-9, both as
max-abs error relative to the oracle's max-abs value. Assembly (Eq. 1) agrees to 1e-14 relative:
both sides evaluate the same expression, the only freedom being fused multiply-adds in |x_i-x_j|^2.
"""
import warnings

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


CASES = [
    # n, m, D, T, h, seed
    (1024, 1024, 8, 256, H0, 0),          # 4 x 4 tiles: the small workload
    (1000, 333, 8, 64, H0, 1),            # ragged n and m
    (777, 100, 4, 96, Hyper(0.8, 1.3, 0.05), 2),
    (33, 65, 3, 32, Hyper(1.5, 0.7, 0.2), 3),  # D with no specialised kernel
    (1, 1, 16, 32, H0, 4),                # n = 1, m = 1
    (2048, 512, 16, 128, Hyper(2.0, 1.0, 0.1), 5),
]


@pytest.mark.parametrize("n,m,D,T,h,seed", CASES)
def test_fp64_pipeline_matches_oracle(api, n, m, D, T, h, seed):
    X, y, Xs, _ = nfir.make_dataset(n, m, D, seed)
    ref = oracle.gp_predict(X, y, Xs, h)
    ctx = api.Context(0, tile=T)
    Xd, yd, Xsd = to_dev(X, y, Xs)
    f = api.gp_assemble(ctx, Xd, api.Hyper(*h))
    K = api.gp_factor_rows(ctx, f).cpu().numpy()
    api.gp_cholesky(ctx, f)
    L = api.gp_factor_rows(ctx, f).cpu().numpy()
    mean = api.gp_predict_mean(ctx, f, yd, Xsd)
    alpha = api.gp_alpha(ctx, f)
    cov = api.gp_predict_full_cov(ctx, f, Xsd)
    logdet = api.gp_logdet(ctx, f)
    api.gp_sync(ctx)
    assert ctx.launch_count() > 0
    Kref = np.tril(ref["K"])
    assert rel(K, Kref) <= 1e-14
    assert np.linalg.norm(L @ L.T - ref["K"]) / np.linalg.norm(ref["K"]) <= 1e-13
    assert np.all(np.triu(L, 1) == 0)
    assert rel(L, ref["L"]) <= 1e-12
    assert rel(alpha.cpu().numpy(), ref["alpha"]) <= 1e-10
    assert rel(mean.cpu().numpy(), ref["mean"]) <= 1e-10
    c = cov.cpu().numpy()
    assert rel(c, ref["cov"]) <= 1e-9
    assert np.array_equal(c, c.T)
    assert abs(logdet - ref["logdet"]) <= 1e-12 * max(1.0, abs(ref["logdet"]))
    f.free()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp64_ozaki", "bf16x6"])
def test_variance_only_matches_covariance_diagonal(api, precision):
    """gp_predict_var = diag of Eq. (3) (oracle), without forming V^T V."""
    X, y, Xs, _ = nfir.make_dataset(900, 150, 8, 13)
    ref = oracle.gp_predict(X, y, Xs, H0)
    ctx = api.Context(0, tile=128, precision=precision)
    Xd, Xsd = to_dev(X, Xs)
    f = api.gp_assemble(ctx, Xd, api.Hyper(*H0))
    api.gp_cholesky(ctx, f)
    var = api.gp_predict_var(ctx, f, Xsd).cpu().numpy()
    api.gp_sync(ctx)
    assert rel(var, np.diag(ref["cov"])) <= (1e-9 if precision in ("fp64", "fp64_ozaki") else 1e-4)


def test_noisy_prior_adds_s2(api):
    X, y, Xs, _ = nfir.make_dataset(200, 50, 8, 7)
    ref = oracle.gp_predict(X, y, Xs, H0, noisy_prior=True)
    ctx = api.Context(0, tile=64, noisy_prior=True)
    Xd, yd, Xsd = to_dev(X, y, Xs)
    mean, cov = api.predict(Xd, yd, Xsd, api.Hyper(*H0), ctx=ctx)
    assert rel(cov.cpu().numpy(), ref["cov"]) <= 1e-9


def test_tile_size_invariance(api):
    """Same factor and predictions for every tile edge, up to rounding (Sec. 3.2's tiling is exact)."""
    X, y, Xs, _ = nfir.make_dataset(600, 90, 8, 9)
    Xd, yd, Xsd = to_dev(X, y, Xs)
    outs = []
    for T in (32, 64, 160, 256, 640):
        ctx = api.Context(0, tile=T)
        outs.append([t.cpu().numpy() for t in api.predict(Xd, yd, Xsd, api.Hyper(*H0), ctx=ctx)])
    for mean, cov in outs[1:]:
        assert rel(mean, outs[0][0]) <= 1e-11
        assert rel(cov, outs[0][1]) <= 1e-11


def test_repeatable_bitwise(api):
    """Updates into each tile are applied in increasing J order whatever the schedule, so two runs
    (and two CTA counts) give bit-identical factors."""
    X, y, Xs, _ = nfir.make_dataset(900, 10, 8, 11)
    (Xd,) = to_dev(X)
    Ls = []
    for grid in (0, 37, 0):
        ctx = api.Context(0, tile=64, grid=grid)
        f = api.gp_assemble(ctx, Xd, api.Hyper(*H0))
        api.gp_cholesky(ctx, f)
        Ls.append(api.gp_factor_rows(ctx, f).cpu().numpy())
        api.gp_sync(ctx)
    assert np.array_equal(Ls[0], Ls[1]) and np.array_equal(Ls[0], Ls[2])


def test_not_positive_definite_reports_column(api):
    """Duplicate points with s2 = 0: the second copy's pivot is exactly 0 (Q3 reading)."""
    X = np.array([[0.0], [1.0], [0.0]])
    ctx = api.Context(0, tile=32)
    (Xd,) = to_dev(X)
    f = api.gp_assemble(ctx, Xd, api.Hyper(1.0, 1.0, 0.0))
    api.gp_cholesky(ctx, f)
    with pytest.raises(api.GPError) as e:
        api.gp_sync(ctx)
    assert e.value.status == 2 and e.value.info == 3
    # the context stays usable after the error is collected
    f2 = api.gp_assemble(ctx, Xd, api.Hyper(1.0, 1.0, 0.1))
    api.gp_cholesky(ctx, f2)
    api.gp_sync(ctx)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_nonfinite_inputs_reported_and_context_recovers(api, precision):
    """NaN/Inf in X, y or Xs: GP_ERR_NONFINITE with the 1-based flat index of the first bad entry (for
    the mean: y's n entries, then Xs's m*D), the context's later persistent launches skip their tasks
    until gp_sync collects the error, and the same context then reproduces the oracle."""
    n, m, D = 600, 70, 4
    X, y, Xs, _ = nfir.make_dataset(n, m, D, 21)
    ref = oracle.gp_predict(X, y, Xs, H0)
    ctx = api.Context(0, tile=128, precision=precision)
    Xd, yd, Xsd = to_dev(X, y, Xs)

    def expect_nonfinite(info, fn):
        with pytest.raises(api.GPError) as e:
            with warnings.catch_warnings():
                warnings.simplefilter("ignore", RuntimeWarning)  # mixed mode: refinement cut short
                fn()
            api.gp_sync(ctx)
        assert e.value.status == 3 and e.value.info == info

    Xb = Xd.clone()
    Xb[300, 1] = float("inf")
    Xb[17, 2] = float("nan")
    f = None

    def factor_bad():
        nonlocal f
        f = api.gp_assemble(ctx, Xb, api.Hyper(*H0))
        api.gp_cholesky(ctx, f)

    expect_nonfinite(17 * D + 2 + 1, factor_bad)
    f = api.gp_assemble(ctx, Xd, api.Hyper(*H0), f)
    api.gp_cholesky(ctx, f)
    yb = yd.clone()
    yb[5] = float("-inf")
    expect_nonfinite(5 + 1, lambda: api.gp_predict_mean(ctx, f, yb, Xsd))
    Xsb = Xsd.clone()
    Xsb[3, 0] = float("nan")
    expect_nonfinite(n + 3 * D + 1, lambda: api.gp_predict_mean(ctx, f, yd, Xsb))
    expect_nonfinite(3 * D + 1, lambda: api.gp_predict_full_cov(ctx, f, Xsb))
    expect_nonfinite(3 * D + 1, lambda: api.gp_predict_var(ctx, f, Xsb))
    mean = api.gp_predict_mean(ctx, f, yd, Xsd)
    cov = api.gp_predict_full_cov(ctx, f, Xsd)
    api.gp_sync(ctx)
    tol_mean, tol_cov = (1e-10, 1e-9) if precision == "fp64" else (1e-10, 1e-4)
    assert rel(mean.cpu().numpy(), ref["mean"]) <= tol_mean
    assert rel(cov.cpu().numpy(), ref["cov"]) <= tol_cov


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_allocation_failures_leave_objects_usable(api, precision):
    """Host-side fault injection: the k-th device allocation of the pipeline fails, for every k in
    turn. The entry point that needed it returns GP_ERR_OOM, nothing faults, and with the hook off the
    same context, reusing the factor object when there is one, reproduces the oracle."""
    n, m, D = 500, 60, 4
    X, y, Xs, _ = nfir.make_dataset(n, m, D, 22)
    ref = oracle.gp_predict(X, y, Xs, H0)
    Xd, yd, Xsd = to_dev(X, y, Xs)
    tol_cov = 1e-9 if precision == "fp64" else 1e-4
    failures = 0
    for k in range(1, 60):
        ctx = api.Context(0, tile=128, precision=precision)  # its own allocations come before the hook
        f, failed = None, None
        api.debug_fail_alloc(k)
        try:
            f = api.gp_assemble(ctx, Xd, api.Hyper(*H0))
            api.gp_cholesky(ctx, f)
            api.gp_predict_mean(ctx, f, yd, Xsd)
            api.gp_predict_full_cov(ctx, f, Xsd)
            api.gp_sync(ctx)
        except api.GPError as e:
            failed = e
        finally:
            api.debug_fail_alloc(0)
        if failed is None:
            break  # k is past the pipeline's last allocation
        assert failed.status == 4, str(failed)
        failures += 1
        f = api.gp_assemble(ctx, Xd, api.Hyper(*H0), f)
        api.gp_cholesky(ctx, f)
        mean = api.gp_predict_mean(ctx, f, yd, Xsd)
        cov = api.gp_predict_full_cov(ctx, f, Xsd)
        api.gp_sync(ctx)
        assert rel(mean.cpu().numpy(), ref["mean"]) <= 1e-10
        assert rel(cov.cpu().numpy(), ref["cov"]) <= tol_cov
    assert 8 <= failures < 59


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["two_point", "three_point"])
def test_golden_closed_forms_gpu(api, case, precision):
    """The library on the 2- and 3-point problems against their 40-digit evaluation from the
    definitions (tests/golden/closed_forms.txt): factor, mean, variance (Eqs. 1-3), log-determinant
    and nlml. FP64 to 1e-13; the mixed mode's refined mean to 1e-10 and its unrefined quantities to
    its stated bounds."""
    from test_oracle_pins import GOLDEN_CASES, load_golden
    g = load_golden()[case]
    xs, ys = GOLDEN_CASES[case]
    X, y = np.array(xs)[:, None], np.array(ys)
    Xd, yd, Xsd = to_dev(X, y, np.array([[0.5]]))
    ctx = api.Context(0, tile=32, precision=precision)
    f = api.gp_assemble(ctx, Xd, api.Hyper(*H0))
    api.gp_cholesky(ctx, f)
    L = api.gp_factor_rows(ctx, f).cpu().numpy()
    mean = api.gp_predict_mean(ctx, f, yd, Xsd).cpu().numpy()
    var = api.gp_predict_full_cov(ctx, f, Xsd).cpu().numpy()
    logdet = api.gp_logdet(ctx, f)
    nl, _ = api.gp_nlml_grad(ctx, Xd, yd, api.Hyper(*H0))
    api.gp_sync(ctx)
    tol = 1e-13 if precision == "fp64" else 1e-5
    for i in range(len(xs)):
        for j in range(i + 1):
            assert L[i, j] == pytest.approx(g[f"L{i}{j}"], rel=tol, abs=tol)
    assert mean[0] == pytest.approx(g["mean"], rel=1e-13 if precision == "fp64" else 1e-10)
    assert var[0, 0] == pytest.approx(g["var"], rel=tol * 10)
    assert logdet == pytest.approx(g["logdet"], rel=tol)
    assert nl == pytest.approx(g["nlml"], rel=tol)


def test_withheld_task_times_out_and_context_survives(api):
    """A task whose completion is never published makes its dependants' bounded waits expire: the
    persistent kernel returns GP_ERR_TIMEOUT instead of hanging, and the GPU stays usable."""
    X, y, Xs, _ = nfir.make_dataset(512, 8, 8, 12)
    (Xd,) = to_dev(X)
    ctx = api.Context(0, tile=64, timeout_s=0.2, withhold_task=0)
    f = api.gp_assemble(ctx, Xd, api.Hyper(*H0))
    api.gp_cholesky(ctx, f)
    with pytest.raises(api.GPError) as e:
        api.gp_sync(ctx)
    assert e.value.status == 6
    ctx2 = api.Context(0, tile=64)
    f2 = api.gp_assemble(ctx2, Xd, api.Hyper(*H0))
    api.gp_cholesky(ctx2, f2)
    L = api.gp_factor_rows(ctx2, f2).cpu().numpy()
    api.gp_sync(ctx2)
    assert rel(L, oracle.cholesky(oracle.assemble_K(X, H0))) <= 1e-12


def test_invalid_arguments(api):
    ctx = api.Context(0)
    X = torch.zeros((4, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(api.GPError):
        api.gp_assemble(ctx, X, api.Hyper(-1.0, 1.0, 0.1))
    with pytest.raises(TypeError):
        api.gp_assemble(ctx, X.float(), api.Hyper())
    with pytest.raises(api.GPError):
        api.Context(0, tile=48)


def test_full_size_sampled(api):
    """The large workload (n = 32768 training, m = 4096 test, D = 8) with the benchmark's launch
    configuration. Checked at sampled entries against the oracle: LL^T = K on sampled entries of K
    (recomputed by the oracle), the residual y - K alpha on sampled rows, the mean from alpha, and
    sampled covariance entries k(a,b) - v_a^T v_b with v_a = L^{-1} k_a by the oracle's forward
    substitution on the GPU's factor."""
    n, m, D = 32768, 4096, 8
    X, y, Xs, _ = nfir.make_dataset(n, m, D, 0)
    ctx = api.Context(0)
    Xd, yd, Xsd = to_dev(X, y, Xs)
    f = api.gp_assemble(ctx, Xd, api.Hyper(*H0))
    api.gp_cholesky(ctx, f)
    mean = api.gp_predict_mean(ctx, f, yd, Xsd)
    alpha = api.gp_alpha(ctx, f).cpu().numpy()
    cov = api.gp_predict_full_cov(ctx, f, Xsd)
    api.gp_sync(ctx)
    rng = np.random.default_rng(0)
    rows = np.sort(rng.choice(n, 24, replace=False))
    Lrows = np.concatenate([api.gp_factor_rows(ctx, f, int(r), 1).cpu().numpy() for r in rows])
    # (L L^T)_ij = L_i . L_j for sampled i, j against K_ij from the oracle's kernel
    ii, jj = np.meshgrid(np.arange(len(rows)), np.arange(len(rows)), indexing="ij")
    LLt = Lrows @ Lrows.T
    Kij = oracle.kernel_entries(X, X, rows[ii.ravel()], rows[jj.ravel()], rows[ii.ravel()] == rows[jj.ravel()], H0)
    assert rel(LLt.ravel(), Kij) <= 1e-13
    # residual of K alpha = y on sampled rows (backward-stable solve: ~ n eps ||K|| ||alpha||)
    r = y[rows] - oracle.kernel_rows_matvec(X, rows, alpha, H0)
    assert np.max(np.abs(r)) <= 1e-9 * np.max(np.abs(y))
    cols = np.sort(rng.choice(m, 16, replace=False))
    mref = oracle.assemble_cross(Xs[cols], X, H0) @ alpha
    assert rel(mean.cpu().numpy()[cols], mref) <= 1e-10
    L = api.gp_factor_rows(ctx, f).cpu().numpy()
    ks = oracle.assemble_cross(Xs[cols], X, H0)  # 16 x n
    V = oracle.forward(L, np.ascontiguousarray(ks.T))
    cref = oracle.assemble_prior(Xs[cols], H0) - V.T @ V
    c = cov.cpu().numpy()[np.ix_(cols, cols)]
    assert rel(c, cref) <= 1e-9


def test_full_size_sampled_mixed(api):
    """The mixed-precision form of the large workload (n = 32768, m = 4096, D = 8) in the benchmark's
    launch configuration (tile 128, tensor cores, packed operands, FP64 refinement), checked at sampled
    entries against the oracle: LL^T = K to the FP32-class bound, the refined solution's residual
    y - K alpha to the FP64 bar and the mean from alpha to 1e-10, and sampled covariance entries against
    k(a,b) - v_a^T v_b with v_a = L^{-1} k_a by the oracle's FP64 forward substitution on the GPU's own
    factor (what remains is the FP32-class error of the V solve and of V^T V). That error is bounded in
    absolute terms against the prior scale v: Sigma = K** - V^T V cancels at that scale, and test
    points near the data have posterior entries far below it."""
    n, m, D = 32768, 4096, 8
    X, y, Xs, _ = nfir.make_dataset(n, m, D, 0)
    ctx = api.Context(0, precision="fp32")
    Xd, yd, Xsd = to_dev(X, y, Xs)
    f = api.gp_assemble(ctx, Xd, api.Hyper(*H0))
    api.gp_cholesky(ctx, f)
    mean, iters = api.gp_predict_mean(ctx, f, yd, Xsd, want_iters=True)
    alpha = api.gp_alpha(ctx, f).cpu().numpy()
    cov = api.gp_predict_full_cov(ctx, f, Xsd)
    api.gp_sync(ctx)
    assert 1 <= iters <= 10
    rng = np.random.default_rng(1)
    rows = np.sort(rng.choice(n, 24, replace=False))
    Lrows = np.concatenate([api.gp_factor_rows(ctx, f, int(r), 1).cpu().numpy() for r in rows])
    ii, jj = np.meshgrid(np.arange(len(rows)), np.arange(len(rows)), indexing="ij")
    Kij = oracle.kernel_entries(X, X, rows[ii.ravel()], rows[jj.ravel()], rows[ii.ravel()] == rows[jj.ravel()], H0)
    assert rel((Lrows @ Lrows.T).ravel(), Kij) <= 2e-5
    r = y[rows] - oracle.kernel_rows_matvec(X, rows, alpha, H0)
    assert np.max(np.abs(r)) <= 1e-9 * np.max(np.abs(y))
    cols = np.sort(rng.choice(m, 16, replace=False))
    mref = oracle.assemble_cross(Xs[cols], X, H0) @ alpha
    assert rel(mean.cpu().numpy()[cols], mref) <= 1e-10
    L = api.gp_factor_rows(ctx, f).cpu().numpy()
    ks = oracle.assemble_cross(Xs[cols], X, H0)
    V = oracle.forward(L, np.ascontiguousarray(ks.T))
    cref = oracle.assemble_prior(Xs[cols], H0) - V.T @ V
    c = cov.cpu().numpy()[np.ix_(cols, cols)]
    assert np.max(np.abs(c - cref)) <= 1e-4 * H0[1]


@pytest.mark.parametrize("variant", ["left", "top"])
@pytest.mark.parametrize("n,m,T", [(1000, 200, 64), (2048, 256, 128)])
def test_left_and_top_looking_match_oracle(api, variant, n, m, T):
    """The left- and top-looking tile variants of Sec. 3.2 (every tile's updates fused into one task,
    dispatched column by column / row by row) give the FP64 results at the FP64 bars."""
    X, y, Xs, _ = nfir.make_dataset(n, m, 8, 21)
    ref = oracle.gp_predict(X, y, Xs, H0)
    ctx = api.Context(0, tile=T, tile_variant=variant)
    Xd, yd, Xsd = to_dev(X, y, Xs)
    f = api.gp_assemble(ctx, Xd, api.Hyper(*H0))
    api.gp_cholesky(ctx, f)
    L = api.gp_factor_rows(ctx, f).cpu().numpy()
    mean = api.gp_predict_mean(ctx, f, yd, Xsd)
    cov = api.gp_predict_full_cov(ctx, f, Xsd)
    api.gp_sync(ctx)
    assert np.linalg.norm(L @ L.T - ref["K"]) / np.linalg.norm(ref["K"]) <= 1e-13
    assert rel(mean.cpu().numpy(), ref["mean"]) <= 1e-10
    assert rel(cov.cpu().numpy(), ref["cov"]) <= 1e-9
    f.free()
