"""Tunable density and the gradient of the second moment -- oracle side.

The paper's density (Eq. (1)) is nonadaptive; the tunable version used here
reshapes it without biasing the estimator:
  Deg_theta(S) = max(d_min, Deg(S) + sum_{l in S} alpha_l),
  first walk step weighted by exp(beta_j):
  Z(theta) = sum_j exp(beta_j) F(E \\ j) / Deg(E \\ j),
  log p(z) = beta_{j1} - log Z + sum_l Deg(S_l) log t_l - sum_i log z_i.
The variance of the estimator is M2 - (mean)^2 with M2 = E_p[(f/p)^2], whose
gradient is -E_p[w^2 d log p / d theta] (w = f/p).  This module computes it
on given points, with d log Z / d theta by complex-step differentiation of
the F recursion (Im log Z(theta + i h e_m) / h), an independent route from
the reverse pass the CUDA library uses.

Weights: w = f/p with f in long double at every point (the estimator's rule
is to use each point's accurate value, re-evaluated at higher precision
where the FP64 value loses digits to the cancellation between forest terms;
the long-double value is that accurate value at every point of the graphs
tested).  A non-finite w counts as 0.
"""
from __future__ import annotations

import cmath
import math

import numpy as np

from .philox import uniforms


def deg_theta(deg0, alpha, N, d_min=0.05):
    """(Deg_theta table, active mask) for real or complex alpha; the clamp
    compares real parts."""
    M = 1 << N
    deg = [0.0] * M
    act = [False] * M
    for m in range(1, M - 1):
        v = deg0[m] + sum(alpha[l] for l in range(N) if m >> l & 1)
        if (v.real if isinstance(v, complex) else v) > d_min:
            deg[m] = v
            act[m] = True
        else:
            deg[m] = d_min
    return deg, act


def log_z(deg0, alpha, beta, N, d_min=0.05):
    deg, _ = deg_theta(deg0, alpha, N, d_min)
    M = 1 << N
    F = [0.0] * M
    for m in range(1, M - 1):
        bits = [l for l in range(N) if m >> l & 1]
        if len(bits) == 1:
            F[m] = 1.0
            continue
        F[m] = sum(F[m & ~(1 << j)] / deg[m & ~(1 << j)] for j in bits)
    Z = sum(cmath.exp(beta[j]) * F[(M - 1) & ~(1 << j)] / deg[(M - 1) & ~(1 << j)] for j in range(N))
    return cmath.log(Z)


def dlogz_complex_step(deg0, alpha, beta, N, d_min=0.05, h=1e-30):
    ga, gb = np.zeros(N), np.zeros(N)
    for m in range(N):
        a = [complex(x) for x in alpha]
        a[m] += 1j * h
        ga[m] = log_z(deg0, a, [complex(x) for x in beta], N, d_min).imag / h
        b = [complex(x) for x in beta]
        b[m] += 1j * h
        gb[m] = log_z(deg0, [complex(x) for x in alpha], b, N, d_min).imag / h
    return ga, gb


def tables(deg0, alpha, beta, N, d_min=0.05):
    """Real tables for the sampler: Deg_theta, F (with F(E) = Z), log Z."""
    deg, act = deg_theta(deg0, alpha, N, d_min)
    M = 1 << N
    F = [0.0] * M
    for m in range(1, M - 1):
        bits = [l for l in range(N) if m >> l & 1]
        F[m] = 1.0 if len(bits) == 1 else sum(F[m & ~(1 << j)] / deg[m & ~(1 << j)] for j in bits)
    return deg, act, F


def sample_theta(u, deg0, alpha, beta, N, d_min=0.05):
    """Points of the tuned density: the first walk step picks line j with
    probability exp(beta_j) F(E\\j) / (Deg(E\\j) Z), later steps as in Eq. (1);
    t_l = u^(1/Deg_theta(S_l)).  Returns (x, log p, order, Deg, active, Z)."""
    deg, act, F = tables(deg0, alpha, beta, N, d_min)
    full = (1 << N) - 1
    wts = [math.exp(beta[j]) * F[full & ~(1 << j)] / deg[full & ~(1 << j)] for j in range(N)]
    Z = sum(wts)
    B = u.shape[0]
    xs = np.zeros((B, N))
    lps = np.zeros(B)
    orders = np.zeros((B, N), dtype=np.int64)
    for b in range(B):
        s = full
        order = []
        for l in range(N - 1):
            cand = [j for j in range(N) if s >> j & 1]
            if l == 0:
                w = [wts[j] for j in cand]
                tot = Z
            else:
                w = [F[s & ~(1 << j)] / deg[s & ~(1 << j)] for j in cand]
                tot = F[s]
            target = u[b, l] * tot
            cum = 0.0
            pick = cand[-1]
            for j, wj in zip(cand, w):
                cum += wj
                if target < cum:
                    pick = j
                    break
            order.append(pick)
            s &= ~(1 << pick)
        order.append([j for j in range(N) if s >> j & 1][0])
        s = full
        logx = 0.0
        lpb = beta[order[0]] - math.log(Z)
        xs[b, order[0]] = 1.0
        for l in range(1, N):
            s &= ~(1 << order[l - 1])
            lu = math.log(u[b, N - 1 + (l - 1)])
            lt = lu / deg[s]
            logx += lt
            xs[b, order[l]] = math.exp(logx)
            lpb += lu - logx
        lps[b] = lpb
        orders[b] = order
    return xs, lps, orders, deg, act, Z


def m2_grad(integrand, g, stream_id, seed, begin, n, alpha, beta, d_min=0.05, deg0=None,
            dtype=np.longdouble):
    """(M2 estimate, dM2/dalpha, dM2/dbeta) on samples [begin, begin+n)."""
    from .graphs import deg_table
    N = g.n_lines
    deg0 = deg0 if deg0 is not None else deg_table(g)
    u = uniforms(np.arange(begin, begin + n, dtype=np.uint64), stream_id, seed, 2 * (N - 1))
    x, lp, order, deg, act, Z = sample_theta(u, deg0, alpha, beta, N, d_min)
    w = np.asarray(integrand(x, dtype=dtype), dtype=np.float64) * np.exp(-lp)
    w = np.where(np.isfinite(w), w, 0.0)
    w2 = w * w
    ga_s = np.zeros(N)
    gb_s = np.zeros(N)
    for b in range(n):
        s = (1 << N) - 1
        cum = 0.0
        for r in range(N):
            if r > 0:
                s &= ~(1 << order[b][r - 1])
                if act[s]:
                    cum += math.log(x[b, order[b][r]] / x[b, order[b][r - 1]])
            ga_s[order[b][r]] += w2[b] * cum
        gb_s[order[b][0]] += w2[b]
    M2 = float(np.sum(w2)) / n
    dla, dlb = dlogz_complex_step(deg0, alpha, beta, N, d_min)
    ga = -(ga_s / n - M2 * dla)
    gb = -(gb_s / n - M2 * dlb)
    return M2, ga, gb
