"""The exact test's refined reciprocal and square root (hardware estimates refined by one
Newton-Raphson step each, used for the roots s/a and c/s of a hit's interval) against the CUDA
runtime's correctly rounded 1/x and sqrt(x) and against numpy's (IEEE, correctly rounded), over
the refinements' whole range.

Bound: the estimates are good to about 2^-20 relative; one Newton step squares a reciprocal
estimate's error (x y' = 1 - eps^2) and leaves 1.5 eps^2 for the square root, so both results
must lie within 2^-38 (a few 1e-12) of the correctly rounded values. Two quotients and a square
root then move a root by under 1e-11 of its size, a hundredth of the search's 1e-9 interval
tolerance. A step dropped or wrongly signed leaves the raw estimate's 2^-20 and fails."""
import numpy as np
import pytest

from paper_1410_2698_gb300 import api

pytestmark = pytest.mark.gpu

REFINED_REL = 2.0 ** -38  # one Newton step from an estimate good to ~2^-20


def _inputs():
    rng = np.random.default_rng(1410)
    wide = np.exp2(rng.uniform(-999.0, 999.0, 200_000))           # every exponent of the range
    typical = np.exp(rng.uniform(np.log(1e-12), np.log(1e12), 200_000))  # a, |s|, disc in practice
    pow2 = np.exp2(np.arange(-999, 999, dtype=np.float64))         # exact powers of two
    near = np.concatenate([np.nextafter(pow2, 0.0), np.nextafter(pow2, np.inf)])
    mant = 1.0 + np.arange(4096) / 4096.0                          # the mantissa range at 2^0
    x = np.concatenate([wide, typical, pow2, near, mant, -wide[:1000], -typical[:1000]])
    return x


def test_refined_estimates_match_correct_rounding():
    x = _inputs()
    r = api.ts_eval_refined_estimates(x)
    # the runtime's references are the correctly rounded values numpy also computes
    assert np.array_equal(r["rcp_ref"], 1.0 / x)
    pos = x > 0
    assert np.array_equal(r["sqrt_ref"][pos], np.sqrt(x[pos]))
    e_rcp = np.abs(r["rcp_est"] - r["rcp_ref"]) / np.abs(r["rcp_ref"])
    e_sqrt = np.abs(r["sqrt_est"][pos] - r["sqrt_ref"][pos]) / r["sqrt_ref"][pos]
    assert np.all(np.isfinite(r["rcp_est"])), "an estimate in range came back non-finite"
    assert e_rcp.max() <= REFINED_REL, f"reciprocal: 2^{np.log2(e_rcp.max()):.2f}"
    assert e_sqrt.max() <= REFINED_REL, f"square root: 2^{np.log2(e_sqrt.max()):.2f}"
    # negative inputs: the reciprocal keeps its sign; the square root is not evaluated
    assert np.all(r["rcp_est"][~pos] < 0) and np.all(np.isnan(r["sqrt_est"][~pos]))


def test_refined_estimates_reject_values_outside_their_range():
    x = np.array([0.0, 5e-324, 1e-305, 2.0 ** -1001, 2.0 ** 1000, 1e305, 1.7e308])
    r = api.ts_eval_refined_estimates(x)
    assert np.all(np.isnan(r["rcp_est"])) and np.all(np.isnan(r["sqrt_est"]))
    inside = np.array([2.0 ** -1000, 2.0 ** 999.5])
    r = api.ts_eval_refined_estimates(inside)
    assert np.all(np.isfinite(r["rcp_est"])) and np.all(np.isfinite(r["sqrt_est"]))
