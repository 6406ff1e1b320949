"""The tensor-core epilogues' GELU, its FP32 operations emulated on the CPU, against the exact GELU.

The kernels evaluate x Phi(x) with Abramowitz and Stegun's Eq. 7.1.26 for erf (absolute error
<= 1.5e-7): t = 1 / (1 + p |y|), the Horner polynomial in t, 2^(-w^2) for exp(-y^2) with
w = x sqrt(log2(e) / 2), erf(|y|) = 1 - t P(t) 2^(-w^2), and x Phi(x) = h + h sign(x) erf(|y|),
h = x / 2 (gelu, and gelu2 for two values at once, in the tensor-core header). Here every FP32
operation is reproduced in numpy (a fused multiply-add as the exact FP64 product plus the addend,
rounded to FP32: it can differ from one rounding only where the FP64 sum was itself inexact, by at
most an FP32 ulp), with the reciprocal and the power of two correctly rounded, and pinned to what
mathematics fixes: x Phi(x) from the library erfc, and the special values. The hardware's
reciprocal and power of two (within 1 and 2 ulp) add at most 0.3e-7 |x| and 1.2e-7 |x| to the
bound below, inside the 5e-7 |x| + 2^-23 |GELU| that the elementwise network tests take.
"""
import math

import numpy as np
from scipy.special import erfc

F32 = np.float32
KW = F32(0.84932180028801904)   # sqrt(log2(e) / 2)
KP = F32(0.27273748087922250)   # 0.3275911 / sqrt(log2(e))
A = [F32(v) for v in (0.254829592, -0.284496736, 1.421413741, -1.453152027, 1.061405429)]


def fma(a, b, c):
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(F32)


def mul(a, b):
    with np.errstate(over="ignore"):  # w^2 beyond FP32 for |x| > 1e19: inf, as on the GPU
        return (np.asarray(a, np.float64) * np.asarray(b, np.float64)).astype(F32)


def gelu(x):
    x = np.asarray(x, F32)
    w = mul(x, KW)
    aw = np.abs(w)
    with np.errstate(divide="ignore"):
        t = (1.0 / fma(KP, aw, F32(1)).astype(np.float64)).astype(F32)
    p = np.full_like(t, A[4])
    for a in A[3::-1]:
        p = fma(t, p, a)
    poly = mul(t, p)
    e = np.exp2(-mul(w, w).astype(np.float64)).astype(F32)
    erf_abs = fma(-poly, e, F32(1))
    h = mul(F32(0.5), x)
    return fma(h, np.copysign(erf_abs, x), h)


def test_gelu_within_its_error_bound():
    """|GELU_fp32(x) - x Phi(x)| <= 3e-7 |x| + 2^-23 |x Phi(x)| over a dense grid of [-12, 12] and
    geometric grids down to 1e-6 on both sides (the relative bound is tightest near 0)."""
    x = np.concatenate([np.linspace(-12, 12, 2000001), -np.geomspace(1e-6, 12, 200001),
                        np.geomspace(1e-6, 12, 200001)]).astype(F32)
    X = x.astype(np.float64)
    exact = X * 0.5 * erfc(-X / math.sqrt(2.0))
    err = np.abs(gelu(x).astype(np.float64) - exact)
    assert np.all(err <= 3e-7 * np.abs(X) + 2.0 ** -23 * np.abs(exact))


def test_large_arguments_saturate():
    """erf rounds to 1 for |x| beyond about 5.8: GELU(x) = x for large positive x, 0 for large
    negative x, up to the largest FP32 values."""
    xs = np.concatenate([np.linspace(6.0, 60.0, 20001), np.geomspace(60.0, 3e38, 2001)]).astype(F32)
    assert np.array_equal(gelu(xs), xs)
    assert not np.any(gelu(-xs))


def test_special_values():
    g = gelu(np.array([0.0, -0.0, np.inf, np.nan], dtype=F32))
    assert g[0] == 0.0 and g[1] == 0.0 and g[2] == np.inf and np.isnan(g[3])
