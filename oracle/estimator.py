"""Nonadaptive Monte Carlo estimator -- oracle side (test infrastructure).

Sec. 2 (item 2) and Sec. 3: a_G is the mean of w = f/p over points drawn
from the per-graph density p of Eq. (1); its statistical error is the
standard deviation of the mean.  Independent runs (Calc 1 and Calc 2 of
Sec. 3, or replicas over disjoint counter ranges) combine by inverse-variance
weighting when they are separate estimates, or by pooling the raw moments
when they are pieces of one sample.
"""
from __future__ import annotations

import math

import numpy as np

from .graphs import deg_table
from .pdf import f_table, sample_points
from .philox import uniforms


def neumaier_sum(xs):
    """Compensated sum in double (Neumaier's variant of Kahan summation)."""
    s = 0.0
    c = 0.0
    for x in xs:
        x = float(x)
        t = s + x
        if abs(s) >= abs(x):
            c += (s - t) + x
        else:
            c += (x - t) + s
        s = t
    return s + c


def moments_to_result(sw, sw2, n):
    mean = sw / n
    var = max(0.0, sw2 / n - mean * mean) / (n - 1) if n > 1 else 0.0
    return {"value": mean, "variance": var, "sigma": math.sqrt(var), "n": n}


def weights(integrand, g, stream_id, seed, begin, n, deg=None):
    N = g.n_lines
    deg = deg if deg is not None else deg_table(g)
    F = f_table(deg, N)
    u = uniforms(np.arange(begin, begin + n, dtype=np.uint64), stream_id, seed, 2 * (N - 1))
    x, lp, _ = sample_points(u, deg, F, N)
    return integrand(x) * np.exp(-lp)


def mc_estimate(integrand, g, stream_id, seed, n, begin=0, batch=20000, deg=None):
    sw = []
    sw2 = []
    for b0 in range(begin, begin + n, batch):
        w = weights(integrand, g, stream_id, seed, b0, min(batch, begin + n - b0), deg)
        sw.extend(w)
        sw2.extend(w * w)
    return moments_to_result(neumaier_sum(sw), neumaier_sum(sw2), n)


def combine_inverse_variance(vals, sigmas):
    """Statistical combination of independent estimates (Sec. 3: Calc 1 and
    Calc 2 combined into one value)."""
    w = [1.0 / s ** 2 for s in sigmas]
    v = sum(wi * x for wi, x in zip(w, vals)) / sum(w)
    return v, math.sqrt(1.0 / sum(w))
