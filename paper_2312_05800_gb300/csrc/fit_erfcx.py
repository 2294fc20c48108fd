"""Coefficients of the GELU used by the tensor-core epilogues (gemm.cuh).

GELU(z) = z Phi(z) = h + |h| erf(sqrt(2) |h|) with h = z / 2, and for a >= 0
erf(a) = 1 - erfcx(a) exp(-a^2), erfcx(a) = exp(a^2) erfc(a) (the scaled
complementary error function: smooth, from 1 at 0 down to about 1 / (sqrt(pi) a)).
The device evaluates exp by the hardware exp2 approximation and erfcx(sqrt(2) x),
x = min(|h|, X), by a polynomial of degree DEG in x. This script fits that
polynomial on [0, X] by iteratively reweighted least squares, minimising the
error of erf itself, |p(x) - erfcx(sqrt 2 x)| exp(-2 x^2) (beyond X = 4.5 / sqrt 2,
erfc(sqrt 2 x) < 4e-10), rounds the coefficients to FP32 and reports the error
of their FP32 Horner evaluation. Run: python fit_erfcx.py
"""
import numpy as np
from scipy.special import erfcx

DEG = 7
X = 4.5 / np.sqrt(2.0)


def fit(deg=DEG, xmax=X, n=40001, iters=200):
    x = np.linspace(0.0, xmax, n)
    g = erfcx(np.sqrt(2.0) * x)
    w = np.exp(-2.0 * x * x)
    V = np.vander(x, deg + 1, increasing=True)
    ww = w.copy()
    for _ in range(iters):
        c, *_ = np.linalg.lstsq(V * ww[:, None], g * ww, rcond=None)
        err = np.abs(V @ c - g) * w
        ww = ww * (1.0 + 2.0 * err / err.max())
    c32 = c.astype(np.float32)
    x32 = x.astype(np.float32)
    y = np.full_like(x32, c32[-1])
    for k in range(deg - 1, -1, -1):
        y = (y * x32 + c32[k]).astype(np.float32)
    return c32, float((np.abs(y.astype(np.float64) - g) * w).max())


if __name__ == "__main__":
    c, e = fit()
    print("max |erf error| of the FP32 Horner evaluation: %.3g" % e)
    print(", ".join("%.9gf" % v for v in c))
