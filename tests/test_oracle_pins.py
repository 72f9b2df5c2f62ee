"""Pins of the FP64 oracle to facts outside itself (closed forms, invariants, brute force, LAPACK).

Each test names the passage it follows. The hand-derived closed forms use the explicit 2x2 inverse
or scalar algebra, not the oracle's substitution steps, so a dropped term, a wrong sign or index
or a transposed operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

import nfir
import oracle
from oracle import Hyper

H0 = Hyper(1.0, 1.0, 0.1)  # the paper's fixed defaults (Sec. 3.1)


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    den = np.max(np.abs(b)) if b.size else 1.0
    return float(np.max(np.abs(a - b)) / (den if den > 0 else 1.0)) if a.size else 0.0


# ---------------------------------------------------------------- Eq. (1)

def test_kernel_matches_independent_rbf():
    """Eq. (1), textbook form v*exp(-r^2/(2 l^2)): against scipy's squared Euclidean distances,
    with the noise only on the diagonal of K_{X,X} and never on the cross-covariance."""
    from scipy.spatial.distance import cdist
    rng = np.random.default_rng(1)
    A, B = rng.normal(size=(37, 5)), rng.normal(size=(23, 5))
    for h in (Hyper(1.0, 1.0, 0.1), Hyper(0.7, 2.5, 0.3)):
        ref = h.v * np.exp(-cdist(A, B, "sqeuclidean") / (2 * h.l ** 2))
        assert rel(oracle.assemble_cross(A, B, h), ref) < 1e-14
        KA = oracle.assemble_K(A, h)
        refA = h.v * np.exp(-cdist(A, A, "sqeuclidean") / (2 * h.l ** 2)) + h.s2 * np.eye(len(A))
        assert rel(KA, refA) < 1e-14
        assert rel(oracle.assemble_prior(A, h), refA - h.s2 * np.eye(len(A))) < 1e-14
        assert rel(oracle.assemble_prior(A, h, noisy=True), refA) < 1e-14


def test_kernel_scalar_values():
    """k(0, 1) = v e^{-1/(2l^2)} for 1-D points; l enters squared (reading of Eq. 1)."""
    h = Hyper(0.5, 2.0, 0.1)
    k = oracle.assemble_cross(np.array([[0.0]]), np.array([[1.0]]), h)[0, 0]
    assert k == pytest.approx(2.0 * math.exp(-2.0), rel=1e-15)


def test_kernel_entries_and_rows_matvec():
    X, y, _, _ = nfir.make_dataset(300, 1, 8, 3)
    K = oracle.assemble_K(X, H0)
    rng = np.random.default_rng(2)
    ia, ib = rng.integers(0, 300, 50), rng.integers(0, 300, 50)
    e = oracle.kernel_entries(X, X, ia, ib, ia == ib, H0)
    assert np.array_equal(e, K[ia, ib])
    rows = rng.integers(0, 300, 20)
    w = rng.normal(size=300)
    assert rel(oracle.kernel_rows_matvec(X, rows, w, H0), (K @ w)[rows]) < 1e-13


# ---------------------------------------------------------------- closed forms (Eqs. 2, 3)

def two_point_closed_form():
    """x = (0, 1), y = (1, 2), test point 0.5, l = v = 1, s2 = 0.1. With a = v + s2, b = e^{-1/2}:
    K^{-1} = [[a, -b], [-b, a]] / (a^2 - b^2); k* = (e^{-1/8}, e^{-1/8})."""
    a, b, ks = 1.1, math.exp(-0.5), math.exp(-0.125)
    det = a * a - b * b
    alpha = np.array([a * 1 - b * 2, -b * 1 + a * 2]) / det
    mean = ks * (alpha[0] + alpha[1])
    var = 1.0 - (ks * ks * (a - b) * 2) / det
    logdet = math.log(det)
    nlml = 0.5 * (1 * alpha[0] + 2 * alpha[1]) + 0.5 * logdet + math.log(2 * math.pi)
    return alpha, mean, var, logdet, nlml


def test_two_point_closed_form():
    X = np.array([[0.0], [1.0]])
    y = np.array([1.0, 2.0])
    Xs = np.array([[0.5]])
    r = oracle.gp_predict(X, y, Xs, H0)
    alpha, mean, var, ld, nl = two_point_closed_form()
    assert rel(r["alpha"], alpha) < 1e-14
    assert r["mean"][0] == pytest.approx(mean, rel=1e-14)
    assert r["cov"][0, 0] == pytest.approx(var, rel=1e-13)
    assert r["logdet"] == pytest.approx(ld, rel=1e-14)
    assert oracle.nlml(r["L"], y, r["alpha"]) == pytest.approx(nl, rel=1e-14)
    # Symmetric case printed in hand-derived form: mean = k*(y1+y2)/(a+b).
    assert mean == pytest.approx(math.exp(-0.125) * 3 / (1.1 + math.exp(-0.5)), rel=1e-14)


def test_single_point_closed_form():
    """n = 1: mean = k* y/(v+s2), var = v - k*^2/(v+s2), nlml = y^2/(2(v+s2)) + log(v+s2)/2 + log(2pi)/2."""
    h = Hyper(0.8, 1.7, 0.3)
    X, y, Xs = np.array([[0.2, -0.1]]), np.array([0.9]), np.array([[0.5, 0.4], [3.0, 3.0]])
    r = oracle.gp_predict(X, y, Xs, h)
    s = h.v + h.s2
    ks = h.v * np.exp(-np.sum((Xs - X[0]) ** 2, axis=1) / (2 * h.l ** 2))
    assert rel(r["mean"], ks * y[0] / s) < 1e-14
    assert rel(np.diag(r["cov"]), h.v - ks ** 2 / s) < 1e-14
    assert r["cov"][0, 1] == pytest.approx(
        h.v * math.exp(-np.sum((Xs[0] - Xs[1]) ** 2) / (2 * h.l ** 2)) - ks[0] * ks[1] / s, rel=1e-13)
    nl, g = oracle.nlml_and_grad(X, y, h)
    assert nl == pytest.approx(0.5 * y[0] ** 2 / s + 0.5 * math.log(s) + 0.5 * math.log(2 * math.pi), rel=1e-15)
    dv = 0.5 * (1 / s - y[0] ** 2 / s ** 2)
    assert g[0] == 0.0 and g[1] == pytest.approx(dv, rel=1e-14) and g[2] == pytest.approx(dv, rel=1e-14)


def test_three_point_against_explicit_inverse():
    """x = (0, 1, 2), y = (1, -1, 0.5): alpha = adj(K) y / det(K) by cofactors."""
    X = np.array([[0.0], [1.0], [2.0]])
    y = np.array([1.0, -1.0, 0.5])
    a, b, c = 1.1, math.exp(-0.5), math.exp(-2.0)
    K = np.array([[a, b, c], [b, a, b], [c, b, a]])
    det = a * (a * a - b * b) - b * (b * a - b * c) + c * (b * b - a * c)
    adj = np.array([[a * a - b * b, -(b * a - c * b), b * b - a * c],
                    [-(b * a - b * c), a * a - c * c, -(a * b - c * b)],
                    [b * b - a * c, -(a * b - b * c), a * a - b * b]])
    alpha = adj @ y / det
    r = oracle.gp_predict(X, y, np.array([[0.5]]), H0)
    assert rel(r["alpha"], alpha) < 1e-13
    assert r["logdet"] == pytest.approx(math.log(det), rel=1e-13)
    assert rel(r["L"] @ r["L"].T, K) < 1e-15
    ks = np.exp(-np.array([0.25, 0.25, 2.25]) / 2)
    assert r["mean"][0] == pytest.approx(ks @ alpha, rel=1e-13)
    assert r["cov"][0, 0] == pytest.approx(1.0 - ks @ (adj @ ks) / det, rel=1e-12)


def test_far_field_reverts_to_prior():
    """A test point 40 lengthscales from all data: mean 0 and variance v (Eqs. 2, 3 with k* = 0)."""
    X, y, _, _ = nfir.make_dataset(64, 1, 4, 5)
    Xs = np.full((2, 4), 100.0)
    Xs[1] += 1.0
    h = Hyper(1.0, 1.3, 0.1)
    r = oracle.gp_predict(X, y, Xs, h)
    assert np.all(r["mean"] == 0.0)
    assert rel(r["cov"], oracle.assemble_prior(Xs, h)) == 0.0


def test_interpolation_as_noise_vanishes():
    """Well-separated training points, s2 -> 1e-10, test = train: the mean reproduces y and the
    variance vanishes (Eqs. 2, 3 with K_{Xs,X} = K - s2 I)."""
    rng = np.random.default_rng(4)
    X = np.arange(12, dtype=np.float64)[:, None] * 2.5 + rng.uniform(0, 0.2, (12, 1))
    y = rng.normal(size=12)
    h = Hyper(1.0, 1.0, 1e-10)
    r = oracle.gp_predict(X, y, X, h)
    assert np.max(np.abs(r["mean"] - y)) < 1e-8
    assert np.max(np.abs(np.diag(r["cov"]))) < 1e-8


# ---------------------------------------------------------------- invariants and library cross-checks

@pytest.fixture(scope="module")
def nfir_case():
    X, y, Xs, ys = nfir.make_dataset(700, 300, 8, 0)
    return X, y, Xs, oracle.gp_predict(X, y, Xs, H0)


def test_factor_reconstructs_K(nfir_case):
    """||L L^T - K||_F / ||K||_F <= 1e-13, L lower with a positive diagonal (Sec. 3.1)."""
    X, y, Xs, r = nfir_case
    L, K = r["L"], r["K"]
    assert np.linalg.norm(L @ L.T - K) / np.linalg.norm(K) < 1e-13
    assert np.all(np.triu(L, 1) == 0) and np.all(np.diag(L) > 0)


def test_against_lapack(nfir_case):
    """Cross-check with LAPACK (numpy/scipy): factor, alpha, mean, covariance, logdet."""
    import scipy.linalg as sl
    X, y, Xs, r = nfir_case
    Lr = np.linalg.cholesky(r["K"])
    assert rel(r["L"], Lr) < 1e-12
    alpha = sl.cho_solve((Lr, True), y)
    assert rel(r["alpha"], alpha) < 1e-10
    assert rel(r["mean"], r["Kxs"] @ alpha) < 1e-10
    V = sl.solve_triangular(Lr, r["Kxs"].T, lower=True)
    assert rel(r["V"], V) < 1e-11
    assert rel(r["cov"], r["Kss"] - V.T @ V) < 1e-12
    assert r["logdet"] == pytest.approx(np.linalg.slogdet(r["K"])[1], rel=1e-12)


def test_covariance_symmetric_psd_bounded(nfir_case):
    """Eq. (3): the posterior covariance is symmetric, PSD and 0 <= diag <= v."""
    *_, r = nfir_case
    C = r["cov"]
    assert np.max(np.abs(C - C.T)) <= 1e-15 * np.max(np.abs(C))
    assert np.min(np.linalg.eigvalsh(C)) >= -1e-12 * H0.v
    d = np.diag(C)
    assert np.all(d >= -1e-14) and np.all(d <= H0.v + 1e-14)


@pytest.mark.parametrize("T", [1, 7, 64, 100, 256, 700, 1000])
def test_tiled_matches_unblocked(nfir_case, T):
    """The tiled right-looking algorithm (Fig. 1) gives the unblocked factor for any tile edge,
    including ragged last tiles and T > n."""
    *_, r = nfir_case
    assert rel(oracle.cholesky_tiled(r["K"], T), r["L"]) < 1e-13


def test_permutation_equivariance(nfir_case):
    """Permuting the training rows leaves mean and covariance unchanged (to rounding)."""
    X, y, Xs, r = nfir_case
    p = np.random.default_rng(7).permutation(len(X))
    r2 = oracle.gp_predict(X[p], y[p], Xs, H0)
    assert rel(r2["mean"], r["mean"]) < 1e-10
    assert rel(r2["cov"], r["cov"]) < 1e-10
    assert r2["logdet"] == pytest.approx(r["logdet"], rel=1e-12)


def test_not_positive_definite_reports_column():
    """Duplicate rows with s2 = 0 make K singular: the pivot of the second copy fails (Q3 reading)."""
    X = np.array([[0.0], [1.0], [0.0]])
    K = oracle.assemble_K(X, Hyper(1.0, 1.0, 0.0))
    with pytest.raises(oracle.NotPositiveDefinite) as e:
        oracle.cholesky(K)
    assert e.value.info == 3
    with pytest.raises(oracle.NotPositiveDefinite) as e:
        oracle.cholesky_tiled(K, 2)
    assert e.value.info == 3


def test_brute_force_extended_precision():
    """n = 9 with mpmath at 40 digits: inverse and determinant directly, no factorisation."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    X, y, Xs, _ = nfir.make_dataset(9, 3, 3, 11)
    X = X + np.arange(9)[:, None] * 0.01  # break exact duplicates
    h = Hyper(0.9, 1.2, 0.05)
    r = oracle.gp_predict(X, y, Xs, h)

    def k(a, b):
        return mp.mpf(h.v) * mp.e ** (-sum((mp.mpf(a[d]) - mp.mpf(b[d])) ** 2 for d in range(len(a))) / (2 * mp.mpf(h.l) ** 2))
    K = mp.matrix(9, 9)
    for i in range(9):
        for j in range(9):
            K[i, j] = k(X[i], X[j]) + (mp.mpf(h.s2) if i == j else 0)
    Ki = K ** -1
    ym = mp.matrix([mp.mpf(v) for v in y])
    alpha = Ki * ym
    assert rel(r["alpha"], [float(alpha[i]) for i in range(9)]) < 1e-10
    assert r["logdet"] == pytest.approx(float(mp.log(mp.det(K))), rel=1e-12)
    for a in range(3):
        ka = mp.matrix([k(Xs[a], X[i]) for i in range(9)])
        assert r["mean"][a] == pytest.approx(float((ka.T * alpha)[0]), rel=1e-10, abs=1e-14)
        for b in range(3):
            kb = mp.matrix([k(Xs[b], X[i]) for i in range(9)])
            cab = k(Xs[a], Xs[b]) - (ka.T * Ki * kb)[0]
            assert r["cov"][a, b] == pytest.approx(float(cab), rel=1e-9, abs=1e-13)


# ---------------------------------------------------------------- NLML gradient and Adam

def test_gradient_central_differences():
    """grad nlml w.r.t. (l, v, s2) against central differences with h = 1e-5 (R&W Sec. 5.4)."""
    X, y, _, _ = nfir.make_dataset(200, 1, 8, 21)
    h = Hyper(0.7, 1.4, 0.2)
    _, g = oracle.nlml_and_grad(X, y, h)
    step = 1e-5
    for k in range(3):
        hp, hm = list(h), list(h)
        hp[k] += step
        hm[k] -= step
        fd = (oracle.nlml_and_grad(X, y, Hyper(*hp))[0] - oracle.nlml_and_grad(X, y, Hyper(*hm))[0]) / (2 * step)
        assert g[k] == pytest.approx(fd, rel=1e-6, abs=1e-6)


def test_gradient_lengthscale_sign():
    """Pin the sign and r^2/l^3 factor of dK/dl on n = 2: nlml(l) closed form differentiated."""
    X, y = np.array([[0.0], [1.0]]), np.array([1.0, 2.0])
    l, v, s2 = 0.8, 1.0, 0.1

    def f(l_):
        a, b = v + s2, v * math.exp(-1 / (2 * l_ * l_))
        det = a * a - b * b
        q = (a * 1 - 2 * b * 2 + a * 4) / det
        return 0.5 * q + 0.5 * math.log(det) + math.log(2 * math.pi)
    a, b = v + s2, v * math.exp(-1 / (2 * l * l))
    db = b / l ** 3  # d b / d l
    det = a * a - b * b
    q = (a * 1 - 4 * b + a * 4)
    dq = (-4 * db * det - q * (-2 * b * db)) / det ** 2
    dlogdet = -2 * b * db / det
    _, g = oracle.nlml_and_grad(X, y, Hyper(l, v, s2))
    assert g[0] == pytest.approx(0.5 * dq + 0.5 * dlogdet, rel=1e-13)
    assert g[0] == pytest.approx((f(l + 1e-6) - f(l - 1e-6)) / 2e-6, rel=1e-7)


def test_adam_first_step_and_floor():
    """Adam's first bias-corrected step has size lr in every coordinate (m_hat/sqrt(v_hat) = sign g);
    the clamp keeps parameters >= 1e-6."""
    hist = oracle.adam([1.0, -2.0, 1e-6], lambda t: (float(t @ t), 2 * t), steps=2, lr=0.05)
    t0, t1 = hist[0][0], hist[1][0]
    assert t1[0] == pytest.approx(0.95, abs=1e-9)
    assert t1[1] == pytest.approx(1e-6)  # -1.95 clamped to the floor
    assert t1[2] == pytest.approx(1e-6)
    assert t0[0] == 1.0


def load_golden(name="closed_forms.txt"):
    """Values of tests/golden/<name> as {case: {key: float}}."""
    import os
    out = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as fh:
        for line in fh:
            if line.startswith("#") or "=" not in line:
                continue
            k, v = (s.strip() for s in line.split("=", 1))
            case, key = k.split(".", 1)
            out.setdefault(case, {})[key] = float(v)
    return out


GOLDEN_CASES = {"two_point": ([0.0, 1.0], [1.0, 2.0]), "three_point": ([0.0, 1.0, 2.0], [1.0, -1.0, 0.5])}


@pytest.mark.parametrize("case", sorted(GOLDEN_CASES))
def test_golden_closed_forms(case):
    """The oracle against the 40-digit evaluation of the definitions (tests/golden/closed_forms.txt):
    factor, alpha, mean, variance (Eqs. 1-3), log-determinant and nlml."""
    g = load_golden()[case]
    xs, ys = GOLDEN_CASES[case]
    X, y = np.array(xs)[:, None], np.array(ys)
    r = oracle.gp_predict(X, y, np.array([[0.5]]), H0)
    n = len(xs)
    for i in range(n):
        for j in range(i + 1):
            assert r["L"][i, j] == pytest.approx(g[f"L{i}{j}"], rel=1e-15, abs=1e-16)
        assert r["alpha"][i] == pytest.approx(g[f"alpha{i}"], rel=1e-14)
    assert r["mean"][0] == pytest.approx(g["mean"], rel=1e-14)
    assert r["cov"][0, 0] == pytest.approx(g["var"], rel=1e-13)
    assert r["logdet"] == pytest.approx(g["logdet"], rel=1e-14)
    assert oracle.nlml(r["L"], y, r["alpha"]) == pytest.approx(g["nlml"], rel=1e-14)
