"""The library's FP64 reciprocal, inverse square root and square root.

They are seeded by the FP32 hardware approximations and refined by two
Newton-Raphson steps in FP64 (each step squares the relative error:
2^-22 -> 2^-44 -> below 2^-53), then rounded once more, so each may differ
from the correctly rounded IEEE result by a few units in the last place.  The
bound tested here is 2 ulp of the IEEE result over a sweep of 43 decades plus
random mantissas, and exact IEEE results where the argument takes the IEEE
path (outside [1e-30, 1e30], where the FP32 seed would overflow or underflow).
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

import paper_1411_0814_gb300 as rsm  # noqa: E402


def ulps(got, want):
    return np.abs(got - want) / np.spacing(np.abs(want))


def test_fp64_reciprocal_and_square_roots_within_2_ulp():
    rng = np.random.default_rng(5)
    x = np.concatenate([np.logspace(-29.9, 29.9, 200001), rng.uniform(0.5, 1.0, 100000) * 2.0 ** rng.integers(-90, 90, 100000),
                        1.0 + np.arange(-512, 512) * 2.0 ** -52, [1.0, 2.0, 4.0, 0.25, 3.0, 1e-30 * 1.0001, 1e30 * 0.9999]])
    out = rsm.check_fp64_math(torch.from_numpy(x).cuda()).cpu().numpy()
    r_rcp, r_rsq, r_sqrt = ulps(out[0], 1.0 / x), ulps(out[1], 1.0 / np.sqrt(x)), ulps(out[2], np.sqrt(x))
    print(f"max ulp: rcp {r_rcp.max():.2f} rsqrt {r_rsq.max():.2f} sqrt {r_sqrt.max():.2f}; "
          f"exact fraction rcp {np.mean(r_rcp == 0):.3f} sqrt {np.mean(r_sqrt == 0):.3f}")
    assert r_rcp.max() <= 2.0
    assert r_rsq.max() <= 2.0
    assert r_sqrt.max() <= 2.0
    # negative arguments of the reciprocal
    neg = -x[::97]
    o = rsm.check_fp64_math(torch.from_numpy(np.ascontiguousarray(neg)).cuda()).cpu().numpy()
    assert ulps(o[0], 1.0 / neg).max() <= 2.0


def test_fp64_math_ieee_path_outside_the_seed_range():
    x = np.array([1e-300, 1e-31, 1e31, 1e300, 5e-324, 1.7e308])
    out = rsm.check_fp64_math(torch.from_numpy(x).cuda()).cpu().numpy()
    with np.errstate(over="ignore", divide="ignore"):
        want_rcp = 1.0 / x
    assert np.array_equal(out[0], want_rcp)
    assert np.array_equal(out[2], np.sqrt(x))
    assert ulps(out[1], 1.0 / np.sqrt(x)).max() <= 1.0  # 1 / sqrt(x): two IEEE roundings
