"""Tolerances for comparing two runs that trace the same particles but may
add their contributions in a different order.

Which lane traces which particle depends on the dynamic work queue, so the
per-lane partial sums of the Eq. 4 estimator differ from run to run while
every particle's contribution x_i = s_i L_i is the same.  FP32 lanes sum with
Kahan compensation, whose error is at most 2u sum |x_i| (u = 2^-24); FP64
lanes sum plainly, at most (n - 1) u sum |x_i| (u = 2^-53).  With the
particle count N and the relative standard error r of the mean,
sum |x_i| / |sum x_i| <= sqrt(N sum x_i^2) / |sum x_i| = sqrt(1 + N r^2),
and two runs can differ by twice the bound.  Cross-lane accumulation is FP64
and adds a negligible term.
"""
import math


def sum_order_rtol(result, precision, key="kappa"):
    n = max(int(result["particles"]), 1)
    value = abs(result[key])
    if value == 0.0:
        return 0.0
    rel = abs(result[key + "_se"]) / value
    spread = math.sqrt(1.0 + n * rel * rel)
    if precision == "fp32":
        return 2.0 * 2.0 * 2.0 ** -24 * spread
    return 2.0 * n * 2.0 ** -53 * spread


def lane_sum_error(precision, n):
    """Bound on the relative error (against sum |x_i|) of one lane's sum."""
    return 2.0 * 2.0 ** -24 if precision == "fp32" else n * 2.0 ** -53


def sum_atol(sum_x2, n, precision, runs=2):
    """Absolute tolerance on sum x_i between results assembled from `runs`
    separately summed runs: each contributes at most lane_sum_error times
    sum |x_i| <= sqrt(n sum x_i^2)."""
    n = max(int(n), 1)
    return runs * lane_sum_error(precision, n) * math.sqrt(n * sum_x2)
