"""Error bound of the Newton-refined reciprocal and cube root that the lane
kernel's step control uses (an FP32 seed refined by one Newton-Raphson step in
FP64). The same arithmetic in numpy: FP32 seed (correctly rounded
reciprocal, float32 cube root), one FP64 Newton step; the relative error must
stay below 1e-12 over the FP32 normal range the kernel admits."""
import numpy as np


def rcp_newton(x):
    r0 = (np.float32(1.0) / x.astype(np.float32)).astype(np.float64)
    return r0 + r0 * (1.0 - x * r0)


def cbrt_newton(a):
    c0 = np.cbrt(a.astype(np.float32)).astype(np.float64)
    return c0 + (a * rcp_newton(c0 * c0) - c0) / 3.0


def test_newton_reciprocal_and_cube_root_error_bound():
    rng = np.random.default_rng(11)
    x = np.exp(rng.uniform(np.log(2.0 ** -119), np.log(2.0 ** 119), 200000))
    e_r = np.abs(rcp_newton(x) * x - 1.0)
    e_c = np.abs(cbrt_newton(x) / np.cbrt(x) - 1.0)
    assert e_r.max() < 1e-13, e_r.max()
    assert e_c.max() < 1e-12, e_c.max()
