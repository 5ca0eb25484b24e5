"""The FP64 face kernel forms its quotients from an FP32 reciprocal seed, one
Newton-Raphson step and one residual correction (Markstein's refinement)
instead of the FP64 division sequence.  This checks the method's error bound
on the host: with a seed of relative error up to 2^-22 (the FP32 reciprocal
approximation and the rounding of the divisor to FP32 together), the result
stays within 0.51 units in the last place of the exact quotient, i.e. it
differs from the correctly rounded a / b by at most one unit in rare ties.
The fused multiply-adds are emulated in extended precision."""
import numpy as np
import pytest


def _fma(x, y, z):
    return (np.longdouble(x) * np.longdouble(y) + np.longdouble(z)).astype(np.float64)


@pytest.mark.skipif(np.finfo(np.longdouble).nmant < 63, reason="needs an extended long double for the fma emulation")
def test_newton_residual_quotient_within_half_ulp():
    rng = np.random.default_rng(1)
    n = 400_000
    a = rng.uniform(-1, 1, n) * 10 ** rng.uniform(-20, 20, n)
    b = rng.uniform(0.5, 1, n) * 10 ** rng.uniform(-29, 29, n) * np.sign(rng.uniform(-1, 1, n))
    seed = (np.float32(1) / b.astype(np.float32)).astype(np.float64) * (1 + rng.uniform(-1, 1, n) * 2.0 ** -22)
    y = _fma(seed, _fma(-b, seed, 1.0), seed)
    q = a * y
    q = _fma(y, _fma(-b, q, a), q)
    exact = np.longdouble(a) / np.longdouble(b)
    ulp = np.spacing(np.abs(exact.astype(np.float64)))
    err = np.abs((np.longdouble(q) - exact).astype(np.float64)) / ulp
    assert err.max() < 0.51
    # the IEEE quotient, for scale: correctly rounded
    ieee = np.abs((np.longdouble(a / b) - exact).astype(np.float64)) / ulp
    assert ieee.max() <= 0.5 + 1e-12
