"""The kernels' reciprocal, reciprocal square root and square root against the IEEE operations:
FP64 (hardware seeds refined by two Newton-Raphson steps) within 2 ulp, FP32 (single
hardware approximations) within their documented error (2 ulp for rcp and rsqrt, a few ulp
for sqrt). Arguments: log-uniform positives over 1e-30 .. 1e30 (FP64) and the float range."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def ulps(a, b, dtype):
    return np.abs(a - b) / np.spacing(np.abs(b).astype(dtype)).astype(np.float64)


def test_fp64_and_fp32_reciprocals_and_roots():
    import paper_1711_09272_gb300 as P
    r = W.SplitMix64(5).uniforms(200000)
    x = np.concatenate([10.0 ** (60 * r - 30), [1.0, 2.0, 0.5, 3.0, 1e-300 * 1e290, 7.0 / 3.0]])
    out = P.roeam_math_check(x)
    assert np.max(ulps(out[:, 0], 1.0 / x, np.float64)) <= 2
    assert np.max(ulps(out[:, 1], 1.0 / np.sqrt(x), np.float64)) <= 2
    assert np.max(ulps(out[:, 2], np.sqrt(x), np.float64)) <= 2
    xf = x.astype(np.float32)
    ok = (xf > 1e-30) & (xf < 1e30)
    xf = xf[ok].astype(np.float64)
    assert np.max(ulps(out[ok, 3], 1.0 / xf, np.float32)) <= 2
    assert np.max(ulps(out[ok, 4], 1.0 / np.sqrt(xf), np.float32)) <= 3
    assert np.max(ulps(out[ok, 5], np.sqrt(xf), np.float32)) <= 4
    assert P.roeam_math_check(np.array([0.0]))[0, 2] == 0.0     # sqrt(0) = 0 (a fluid at rest)
