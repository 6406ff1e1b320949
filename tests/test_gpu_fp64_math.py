"""The FP64 reciprocal and square root of the stage kernels (Newton-Raphson from the FP32
hardware approximations, two corrections) against CUDA's correctly rounded division and sqrt:
within one unit in the last place over the ranges the kernels meet (the trace factor
1/(rho (3 - rho)) and 1/rho for 0 < rho < 3, the sound speed sqrt(p_alpha'(rho)) of the
modified pressure), and equal to CUDA's results outside the Newton iteration's domain."""
import numpy as np
import pytest

from paper_1912_12059_gb300 import nsk

pytestmark = pytest.mark.gpu


def _ulps(a, b):
    """Distance in units in the last place of two arrays of positive finite doubles."""
    return np.abs(a.view(np.int64) - b.view(np.int64))


def _eval(gpu, fn, x):
    import torch

    xt = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(gpu)
    y = torch.empty_like(xt)
    nsk._test_hook_math(fn, xt, y)
    want = 1.0 / xt if fn == 0 else torch.sqrt(xt)
    torch.cuda.synchronize()
    return y.cpu().numpy(), want.cpu().numpy()


def _pa_prime(rho, T=0.85, alpha=1e3):
    return 24.0 * T / (3.0 - rho) ** 2 - 6.0 * rho + alpha * rho


def test_reciprocal_within_one_ulp(gpu):
    rng = np.random.default_rng(1)
    rho = rng.uniform(1e-3, 3.0 - 1e-3, 400000)
    x = np.concatenate([10.0 ** rng.uniform(-30, 30, 400000), rho, rho * (3.0 - rho),
                        np.nextafter(1.0, 2.0) ** np.arange(1000)])
    got, want = _eval(gpu, 0, x)
    d = _ulps(got, want)
    assert d.max() <= 1, (int(d.max()), x[d.argmax()])


def test_sqrt_within_one_ulp(gpu):
    rng = np.random.default_rng(2)
    rho = rng.uniform(0.02, 2.98, 200000)
    x = np.concatenate([10.0 ** rng.uniform(-30, 30, 400000)] +
                       [_pa_prime(rho, alpha=a) for a in (0.5, 2.0, 100.0, 1e3, 1e4)])
    x = x[x > 0]
    got, want = _eval(gpu, 1, x)
    d = _ulps(got, want)
    assert d.max() <= 1, (int(d.max()), x[d.argmax()])


@pytest.mark.parametrize("fn", [0, 1])
def test_outside_the_domain_cuda_decides(gpu, fn):
    x = np.array([0.0, 1e-310, 2.0 ** -121, 2.0 ** -120.5, 2.0 ** 120, 2.0 ** 121, 1e300, np.inf, np.nan, -1.0, -0.0])
    got, want = _eval(gpu, fn, x)
    same = (got == want) | (np.isnan(got) & np.isnan(want))
    assert same.all(), (x[~same], got[~same], want[~same])
