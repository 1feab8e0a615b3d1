"""The reciprocal the FP64 pivot chains use (the precision-block downdate, the
symmetric sweeps of the closed-form stage and of the block builds; no GPU
needed): two Newton-Raphson steps x <- x + x (1 - v x) from the FP32
reciprocal.  Each step squares the relative error, 2^-23 -> 2^-46 -> below the
FP64 rounding, so the result lies within two units in the last place of 1/v
over the pivots' range (the degeneracy floor 1e-12 up to large precision
entries).  Emulated with separately rounded FP64 operations (the kernel fuses
the multiply-adds, which only rounds less)."""
import numpy as np


def rcp_newton(v):
    x = (np.float32(1.0) / v.astype(np.float32)).astype(np.float64)
    for _ in range(2):
        x = x + x * (1.0 - v * x)
    return x


def test_newton_reciprocal_within_two_ulps():
    rng = np.random.default_rng(5)
    v = np.concatenate([10.0 ** rng.uniform(-12, 12, 200000), rng.uniform(0.5, 2.0, 100000),
                        np.array([1e-12, 1.0, 2.0, 3.0, 1e12, np.nextafter(1.0, 2.0)])])
    x = rcp_newton(v)
    exact = 1.0 / v
    assert np.max(np.abs(x - exact) / np.spacing(exact)) <= 2.0


def test_one_step_is_not_enough():
    # the second step is needed: after one the relative error is still ~2^-46
    v = np.random.default_rng(6).uniform(1.0, 2.0, 10000)
    x0 = (np.float32(1.0) / v.astype(np.float32)).astype(np.float64)
    x1 = x0 + x0 * (1.0 - v * x0)
    assert np.max(np.abs(x1 * v - 1.0)) > 1e-15
