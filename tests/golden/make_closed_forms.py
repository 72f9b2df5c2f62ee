"""Writes closed_forms.txt: the 2- and 3-point GP problems of the oracle's closed-form pins evaluated
in 40-digit arithmetic (mpmath), from the definitions alone -- Eq. 1 (squared-exponential kernel with
the noise variance on the diagonal of K only), Eq. 2 (mean = K_{Xs,X} K^{-1} y), Eq. 3 (covariance
= K_{Xs,Xs} - K_{Xs,X} K^{-1} K_{X,Xs}), log det K, and the negative log marginal likelihood
1/2 y^T K^{-1} y + 1/2 log det K + n/2 log(2 pi) (Rasmussen & Williams 2006, Eq. 2.30). Nothing here
runs the library or the oracle.

    python tests/golden/make_closed_forms.py
"""
import os

import mpmath as mp

mp.mp.dps = 40


def case(xs, ys, xstar, l=1, v=1, s2=mp.mpf("0.1")):
    n = len(xs)
    k = lambda a, b: v * mp.e ** (-((a - b) ** 2) / (2 * l * l))
    K = mp.matrix(n, n)
    for i in range(n):
        for j in range(n):
            K[i, j] = k(xs[i], xs[j]) + (s2 if i == j else 0)
    L = mp.cholesky(K)
    y = mp.matrix(ys)
    alpha = mp.lu_solve(K, y)
    ks = mp.matrix([k(xstar, x) for x in xs])
    kinv_ks = mp.lu_solve(K, ks)
    mean = sum(ks[i] * alpha[i] for i in range(n))
    var = v - sum(ks[i] * kinv_ks[i] for i in range(n))
    logdet = mp.log(mp.det(K))
    nlml = sum(y[i] * alpha[i] for i in range(n)) / 2 + logdet / 2 + n * mp.log(2 * mp.pi) / 2
    out = {}
    for i in range(n):
        for j in range(i + 1):
            out[f"L{i}{j}"] = L[i, j]
    for i in range(n):
        out[f"alpha{i}"] = alpha[i]
    out.update(mean=mean, var=var, logdet=logdet, nlml=nlml)
    return out


def main():
    here = os.path.dirname(os.path.abspath(__file__))
    cases = {
        "two_point": case([0, 1], [1, 2], mp.mpf("0.5")),
        "three_point": case([0, 1, 2], [1, -1, mp.mpf("0.5")], mp.mpf("0.5")),
    }
    with open(os.path.join(here, "closed_forms.txt"), "w") as fh:
        fh.write("# GP prediction on 1-D inputs, l = v = 1, s2 = 0.1, test input 0.5 (the paper's default\n"
                 "# hyperparameters, Sec. 3.1). two_point: X = (0, 1), y = (1, 2); three_point: X = (0, 1, 2),\n"
                 "# y = (1, -1, 0.5). Definitions: Eq. 1 (kernel), Eq. 2 (mean), Eq. 3 (variance = covariance at\n"
                 "# the one test input), log det K, nlml (Rasmussen & Williams 2006, Eq. 2.30); L is the lower\n"
                 "# Cholesky factor of K, alpha = K^{-1} y. 40-digit mpmath, written by make_closed_forms.py.\n")
        for name, vals in cases.items():
            for key, val in vals.items():
                fh.write(f"{name}.{key} = {mp.nstr(val, 30)}\n")


if __name__ == "__main__":
    main()
