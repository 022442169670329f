"""MRG32k3a combined multiple-recursive generator -- oracle side (test
infrastructure).

Sec. 3 of the paper runs Calc 1 with the MRG32k3a generator of the CURAND
library and Calc 2 with Philox4x32-10, as two independent checks of one
integration.  MRG32k3a is L'Ecuyer's generator ("Good parameters and
implementations for combined multiple recursive random number generators",
Operations Research 47 (1999)): two order-3 linear recurrences

    x1[n] = (1403580 x1[n-2] - 810728 x1[n-3])  mod m1,  m1 = 2^32 - 209
    x2[n] = ( 527612 x2[n-1] - 1370589 x2[n-3]) mod m2,  m2 = 2^32 - 22853

combined as z[n] = (x1[n] - x2[n]) mod m1 and mapped to the uniform
u[n] = z[n] / (m1 + 1), or m1 / (m1 + 1) where z[n] = 0, strictly inside
(0, 1); as in L'Ecuyer's implementation the division is a product with the
double nearest 1 / (m1 + 1).  The state is (x[n-3], x[n-2], x[n-1]) for each recurrence, and one
step is a 3x3 matrix product modulo m, so a jump of k steps is a product
with the k-th matrix power (L'Ecuyer, Simard, Chen, Kelton, "An
object-oriented random-number package with many long streams and
substreams", Operations Research 50 (2002)).

Stream layout used by both sides of this project (stated here as a
definition, not shared code): start from the state with all six words
12345 and advance by

    position = seed * 2^127 + (diagram id) * 2^96 + sample * 2^5 + draw,

so that every (seed, diagram, sample) owns 32 consecutive draws (a sample
uses 2(N - 1) <= 28 of them: draw d of a sample is its d-th uniform, in the
order the Philox layout uses).  The jump here is an exact integer matrix
power computed by repeated squaring with Python integers.
"""
from __future__ import annotations

import numpy as np

M1 = 4294967087          # 2^32 - 209
M2 = 4294944443          # 2^32 - 22853
A12, A13 = 1403580, 810728
A21, A23 = 527612, 1370589
SEED0 = (12345, 12345, 12345)
SAMPLE_SHIFT = 5         # 32 draws per sample
DIAG_SHIFT = 96
SEED_SHIFT = 127
# the double nearest 1 / (m1 + 1); both sides multiply by it
NORM = 1.0 / (M1 + 1)


def matrices():
    """One-step transition matrices (A1 mod m1, A2 mod m2) acting on the
    state column (x[n-3], x[n-2], x[n-1])."""
    a1 = [[0, 1, 0], [0, 0, 1], [(-A13) % M1, A12 % M1, 0]]
    a2 = [[0, 1, 0], [0, 0, 1], [(-A23) % M2, 0, A21 % M2]]
    return a1, a2


def mat_mul(a, b, m):
    return [[sum(a[i][k] * b[k][j] for k in range(3)) % m for j in range(3)] for i in range(3)]


def mat_vec(a, v, m):
    return [sum(a[i][k] * v[k] for k in range(3)) % m for i in range(3)]


def mat_pow(a, k, m):
    """a^k mod m for an integer k >= 0, by repeated squaring."""
    r = [[int(i == j) for j in range(3)] for i in range(3)]
    p = [row[:] for row in a]
    while k:
        if k & 1:
            r = mat_mul(r, p, m)
        p = mat_mul(p, p, m)
        k >>= 1
    return r


def step(s1, s2):
    """One step of both recurrences from the states (x[n-3], x[n-2], x[n-1]):
    returns the new states and the output uniform of step n."""
    p1 = (A12 * s1[1] - A13 * s1[0]) % M1
    p2 = (A21 * s2[2] - A23 * s2[0]) % M2
    z = (p1 - p2) % M1
    u = float(z if z > 0 else M1) * NORM
    return (s1[1], s1[2], p1), (s2[1], s2[2], p2), u


def state_at(position: int):
    """State after `position` steps from the all-12345 state (jump ahead)."""
    a1, a2 = matrices()
    s1 = mat_vec(mat_pow(a1, position, M1), list(SEED0), M1)
    s2 = mat_vec(mat_pow(a2, position, M2), list(SEED0), M2)
    return tuple(s1), tuple(s2)


def draws(seed: int, diagram_id: int, sample: int, n_draws: int):
    """The n_draws uniforms of one sample (n_draws <= 32)."""
    assert 0 <= n_draws <= (1 << SAMPLE_SHIFT)
    pos = (int(seed) << SEED_SHIFT) + (int(diagram_id) << DIAG_SHIFT) + (int(sample) << SAMPLE_SHIFT)
    s1, s2 = state_at(pos)
    out = []
    for _ in range(n_draws):
        s1, s2, u = step(s1, s2)
        out.append(u)
    return out


def uniforms(sample_idx, diagram_id: int, seed: int, n_draws: int):
    """Uniform draws [len(sample_idx), n_draws] for the given samples (the
    same call shape as the Philox oracle's uniforms).  A sample that follows
    the previous one is reached by running the recurrence through the
    previous sample's 32 positions; any other by a jump."""
    assert 0 <= n_draws <= (1 << SAMPLE_SHIFT)
    s = np.asarray(sample_idx, dtype=np.uint64).ravel()
    out = np.empty((s.size, n_draws), dtype=np.float64)
    base = (int(seed) << SEED_SHIFT) + (int(diagram_id) << DIAG_SHIFT)
    prev, st = None, None
    for r, i in enumerate(s):
        i = int(i)
        if prev is not None and i == prev + 1:
            s1, s2 = st
        else:
            s1, s2 = state_at(base + (i << SAMPLE_SHIFT))
        row = []
        for d in range(1 << SAMPLE_SHIFT):
            s1, s2, u = step(s1, s2)
            if d < n_draws:
                row.append(u)
        out[r] = row
        prev, st = i, (s1, s2)
    return out
