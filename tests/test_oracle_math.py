"""Pins for the oracle's elementary functions against the exact values (mpmath at 120
bits): error bounds in units in the last place, not bit equality with any libm."""
import math

import mpmath as mp
import numpy as np

mp.mp.prec = 120


def _ulp_err(got, exact):
    e = float(exact)
    return abs(mp.mpf(got) - exact) / math.ulp(e) if e != 0 else abs(got)


def test_exp_error_bound(oracle):
    rng = np.random.default_rng(0)
    xs = np.concatenate([np.linspace(-10, 0, 4001), rng.uniform(-708, 709, 4000),
                         rng.uniform(-1e-6, 1e-6, 200), [0.0, -1.0, 1.0, -708.0, 709.0]])
    worst = max(_ulp_err(oracle.exp(x), mp.exp(mp.mpf(float(x)))) for x in xs)
    assert worst <= 1.0, worst
    assert oracle.exp(0.0) == 1.0
    assert oracle.exp(-709.0) == 0.0 and math.isinf(oracle.exp(710.0))


def test_log_error_bound(oracle):
    rng = np.random.default_rng(1)
    xs = np.concatenate([np.exp(rng.uniform(np.log(2.0**-53), np.log(1e300), 6000)),
                         np.linspace(0.5, 2.0, 3001), 1.0 + rng.uniform(-1e-8, 1e-8, 200),
                         [2.0**-53, 1 - 2.0**-53, 10.0, 1e6]])
    worst = max(_ulp_err(oracle.log(x), mp.log(mp.mpf(float(x)))) for x in xs)
    assert worst <= 2.0, worst  # the plain atanh-series form measures 1.67 ulp at worst
    assert oracle.log(1.0) == 0.0
    assert oracle.log(2.0) == float(mp.log(2))


def test_log_factorial(oracle):
    for k in range(0, 16):
        assert abs(oracle.log_factorial(k) - float(mp.log(mp.factorial(k)))) <= 2 * math.ulp(max(1.0, math.lgamma(k + 1)))
    ks = list(range(16, 200)) + [10**3, 12345, 10**5, 10**6, 10**7, 2**31]
    for k in ks:
        exact = mp.loggamma(k + 1)
        assert abs(oracle.log_factorial(k) - exact) / exact < 4e-16, k
