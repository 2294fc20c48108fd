"""The epilogue GELU's erfcx polynomial (CPU): the coefficients compiled into gemm.cuh are
those fit_erfcx.py produces, and the GELU evaluated with them, step by step as the kernel
does in FP32 (exact exp2 in place of the hardware approximation, whose relative error is
about 2^-22), stays within 4e-6 (1 + |z|) of the exact GELU z Phi(z) over [-12, 12]."""
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2312_05800_gb300", "csrc")


def _header_coeffs():
    src = open(os.path.join(CSRC, "gemm.cuh")).read()
    body = src[src.index("float neg_erfcx(float x)"):]
    body = body[:body.index("return y;")]
    lits = [float(v) for v in re.findall(r"(-?\d+\.\d+(?:e-?\d+)?)f", body)]
    # Horner from the top: fmaf(c_d, x, c_{d-1}), then c_{d-2} .. c0
    return np.array(lits[::-1], np.float32)


def test_coefficients_are_the_fit():
    pytest.importorskip("scipy")
    import importlib.util
    spec = importlib.util.spec_from_file_location("fit_erfcx", os.path.join(CSRC, "fit_erfcx.py"))
    fit = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(fit)
    c, err = fit.fit()
    assert err < 8.5e-6
    assert np.array_equal(_header_coeffs(), -c)


def test_gelu_within_its_bound():
    from scipy.special import erf
    nc = _header_coeffs()                        # negated erfcx coefficients, c0 first
    f = np.float32
    z = np.concatenate([np.linspace(-12, 12, 400001), np.random.default_rng(1).normal(size=100000) * 3]).astype(f)
    h = (z * f(0.5)).astype(f)
    x = np.minimum(np.abs(h), f(3.18198052))
    d = nc.size - 1
    y = np.full_like(x, nc[d])
    for k in range(d - 1, -1, -1):
        y = (y.astype(np.float64) * x + nc[k]).astype(f)         # fma: one rounding
    m = ((h * f(-2.88539008)).astype(f) * h).astype(f)
    e = np.exp2(m.astype(np.float64)).astype(f)
    s = (y.astype(np.float64) * e + 1.0).astype(f)
    g = (np.abs(h).astype(np.float64) * s + h).astype(f)
    z64 = z.astype(np.float64)
    exact = 0.5 * z64 * (1.0 + erf(z64 / math.sqrt(2.0)))
    assert np.all(np.abs(g - exact) <= 4e-6 * (1.0 + np.abs(z64)))
