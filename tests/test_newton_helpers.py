"""Error bound of the Newton-refined reciprocal, cube root and inverse sixth,
fifth and fourth roots that the kernels' step control uses (a low-precision
seed refined by one Newton-Raphson step in FP64). The same arithmetic in
numpy with seeds at the edge of their error (the approximate FP64
reciprocal, float32 cube root and power) and one FP64 Newton step: the
relative error must stay within a few 1e-12 over the FP32 normal range the
kernels admit."""
import os

import numpy as np
import pytest


# the kernels seed the reciprocal with rcp.approx.ftz.f64, whose relative
# error was measured below 2^-19.94 on GB300; the mirror uses a seed pushed
# to that error (both signs), the worst case the Newton step has to absorb
SEED_ERR = 2.0 ** -19.9


def rcp_newton(x, seed_sign=1.0):
    r0 = (1.0 / x) * (1.0 + seed_sign * SEED_ERR)
    return r0 + r0 * (1.0 - x * r0)


def cbrt_newton(a, seed_sign=1.0):
    c0 = np.cbrt(a.astype(np.float32)).astype(np.float64)
    return c0 + (a * rcp_newton(c0 * c0, seed_sign) - c0) / 3.0


def test_newton_reciprocal_and_cube_root_error_bound():
    rng = np.random.default_rng(11)
    x = np.exp(rng.uniform(np.log(2.0 ** -119), np.log(2.0 ** 119), 200000))
    for sg in (1.0, -1.0):
        e_r = np.abs(rcp_newton(x, sg) * x - 1.0)
        e_c = np.abs(cbrt_newton(x, sg) / np.cbrt(x) - 1.0)
        assert e_r.max() < 2e-12, e_r.max()
        assert e_c.max() < 2e-12, e_c.max()


def rpow_newton(x, p, seed_ulps=0):
    """x^(-1/p): FP32 seed (numpy's float32 power, optionally pushed by a few
    ulp to the edge of CUDA's stated powf error), one FP64 Newton step."""
    y0 = np.power(x.astype(np.float32), np.float32(-1.0 / p))
    if seed_ulps:
        y0 = y0 * np.float32(1.0 + seed_ulps * 2.0 ** -23)
    y0 = y0.astype(np.float64)
    u = 1.0 - x * y0 ** p
    return y0 + y0 * u / p


def test_newton_inverse_roots_error_bound():
    rng = np.random.default_rng(12)
    x = np.exp(rng.uniform(np.log(2.0 ** -119), np.log(2.0 ** 119), 200000))
    for p in (6, 5, 4):
        exact = x ** (-1.0 / p)
        for ulps in (0, 4, -4):
            e = np.abs(rpow_newton(x, p, ulps) / exact - 1.0)
            assert e.max() < 5e-12, (p, ulps, e.max())


@pytest.mark.gpu
def test_gpu_approximate_reciprocal_seed_bound(tmp_path):
    """The seed error that the mirror above assumes, measured on the device:
    rcp.approx.ftz.f64 within 2^-19.9, and within 2e-12 after one Newton step."""
    import shutil
    import subprocess
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    src = os.path.join(os.path.dirname(__file__), "probes", "rcp_approx.cu")
    exe = str(tmp_path / "rcp_approx")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-o", exe, src],
                   check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    seed, refined = float(out[0]), float(out[1])
    assert seed < SEED_ERR, seed
    assert refined < 2e-12, refined
