"""Hepp sectors and the Deg-based density of Eq. (1) -- oracle side.

Sec. 2 splits the Feynman-parameter simplex into Hepp sectors
z_{j1} >= z_{j2} >= ... >= z_{jM} and uses, in each sector, the density

    p(z) = C * prod_{l=2..M} (z_{jl} / z_{j(l-1)})^{Deg({jl..jM})} / (z_1...z_M)

(Eq. (1)), which is homogeneous of degree -M, so the simplex integral of p
equals its integral over the slice z_{j1} = 1 (Cheng-Wu).  With t_l =
z_{jl}/z_{j(l-1)} the sector integral factorises into prod_l 1/Deg(S_l),
S_l = {jl..jM}.  Hence:

* normaliser Z = 1/C = F(E) with F({x}) = 1 and
  F(S) = sum_{j in S} F(S \\ {j}) / Deg(S \\ {j});
* sampling: walk S = E -> S \\ {j} with probability
  F(S\\{j}) / (Deg(S\\{j}) F(S)), then t_l = u^(1/Deg(S_l)).

Subsets are bitmasks over line indices.  Ties in the walk's inverse CDF are
resolved by scanning j in ascending line index.
"""
from __future__ import annotations

import math
from itertools import permutations

import numpy as np


def f_table(deg, N: int):
    """F over all non-empty subsets (list indexed by bitmask)."""
    F = [0.0] * (1 << N)
    for mask in range(1, 1 << N):
        bits = [l for l in range(N) if mask >> l & 1]
        if len(bits) == 1:
            F[mask] = 1.0
            continue
        acc = 0.0
        for j in bits:
            r = mask & ~(1 << j)
            acc += F[r] / deg[r]
        F[mask] = acc
    return F


def normaliser_bruteforce(deg, N: int) -> float:
    """Z by summing prod_l 1/Deg(S_l) over all N! sectors (small N only)."""
    full = (1 << N) - 1
    z = 0.0
    for perm in permutations(range(N)):
        s = full
        prod = 1.0
        for j in perm[:-1]:
            s &= ~(1 << j)
            prod /= deg[s]
        z += prod
    return z


def density(z, deg, logZ: float) -> float:
    """log p(z) of Eq. (1) evaluated directly at the point z (any positive
    scaling of a simplex point: p is homogeneous of degree -M).  The sector is
    read off by sorting z in decreasing order."""
    z = np.asarray(z, dtype=np.float64)
    N = z.size
    order = sorted(range(N), key=lambda i: -z[i])
    s = (1 << N) - 1
    lp = -logZ
    for l in range(1, N):
        s &= ~(1 << order[l - 1])
        lp += deg[s] * (math.log(z[order[l]]) - math.log(z[order[l - 1]]))
    lp -= float(np.sum(np.log(z)))
    return lp


def sample_points(u, deg, F, N: int):
    """Map uniforms u[:, 0:2(N-1)] to points.

    Draws 0..N-2 choose the sector (one per walk level), draws N-1..2N-3
    give t_2..t_N.  Returns (x, logp, order): x is scaled so that its largest
    component is 1, logp is log p(x) accumulated along the walk, order is the
    sector permutation j1..jN.
    """
    u = np.atleast_2d(u)
    B = u.shape[0]
    full = (1 << N) - 1
    logZ = math.log(F[full])
    x = np.zeros((B, N))
    logp = np.zeros(B)
    orders = np.zeros((B, N), dtype=np.int64)
    for b in range(B):
        s = full
        order = []
        for l in range(N - 1):
            target = u[b, l] * F[s]
            cum = 0.0
            pick = None
            last = None
            for j in range(N):
                if not (s >> j & 1):
                    continue
                r = s & ~(1 << j)
                cum += F[r] / deg[r]
                last = j
                if target < cum:
                    pick = j
                    break
            if pick is None:
                pick = last
            order.append(pick)
            s &= ~(1 << pick)
        order.append([j for j in range(N) if s >> j & 1][0])
        # radial part
        s = full
        logx = 0.0
        lp = -logZ
        x[b, order[0]] = 1.0
        for l in range(1, N):
            s &= ~(1 << order[l - 1])
            d = deg[s]
            lu = math.log(u[b, N - 1 + (l - 1)])
            logt = lu / d
            logx += logt
            x[b, order[l]] = math.exp(logx)
            lp += d * logt - logx
        logp[b] = lp
        orders[b] = order
    return x, logp, orders
