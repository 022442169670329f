"""Oracle pins: the MRG32k3a generator (Sec. 3, Calc 1).

L'Ecuyer (1999) chose the two component recurrences of MRG32k3a so that
each has a primitive characteristic polynomial: the order of its one-step
matrix modulo m_j is exactly m_j^3 - 1, the largest possible, and the
combined generator's period is (m1^3 - 1)(m2^3 - 1)/2.  That property fixes
the multipliers, their signs and the moduli: a wrong one gives a
polynomial that is not primitive, whose matrix has a smaller order (checked
here against every prime factor of m_j^3 - 1, which sympy factors).  The
jump-ahead by matrix powers is checked against stepping the recurrence, and
the uniform map against its definition."""
import numpy as np
import pytest

from oracle import mrg32k3a as m

sympy = pytest.importorskip("sympy")

IDENT = [[1, 0, 0], [0, 1, 0], [0, 0, 1]]


@pytest.mark.parametrize("comp", [0, 1])
def test_each_component_has_full_period(comp):
    a = m.matrices()[comp]
    mod = (m.M1, m.M2)[comp]
    order = mod ** 3 - 1
    assert m.mat_pow(a, order, mod) == IDENT
    for q in sympy.factorint(order):
        assert m.mat_pow(a, order // q, mod) != IDENT, q


def _full_period(a, mod):
    order = mod ** 3 - 1
    return m.mat_pow(a, order, mod) == IDENT and all(
        m.mat_pow(a, order // q, mod) != IDENT for q in sympy.factorint(order))


@pytest.mark.parametrize("name,comp,row", [
    ("sign of 810728", 0, [810728, 1403580, 0]),
    ("lags of component 1 swapped", 0, [(-810728) % m.M1, 0, 1403580]),
    ("multipliers of component 1 swapped", 0, [1403580, (-810728) % m.M1, 0]),
    ("sign of 1370589", 1, [1370589, 0, 527612]),
    ("lags of component 2 swapped", 1, [(-1370589) % m.M2, 527612, 0]),
])
def test_plausible_mistakes_lose_the_full_period(name, comp, row):
    """The pin is sharp for the mistakes a restatement is likely to make: a
    flipped sign, a swapped lag or swapped multipliers give a matrix whose
    order is below m^3 - 1."""
    mod = (m.M1, m.M2)[comp]
    assert _full_period(m.matrices()[comp], mod)
    assert not _full_period([[0, 1, 0], [0, 0, 1], row], mod), name


def test_component_two_needs_its_own_modulus():
    assert not _full_period(m.matrices()[1], m.M1)


def test_jump_ahead_equals_stepping():
    s1, s2 = m.SEED0, m.SEED0
    outs = []
    for _ in range(1300):
        s1, s2, u = m.step(s1, s2)
        outs.append(u)
        if len(outs) in (1, 31, 32, 1000, 1200):
            assert m.state_at(len(outs)) == (tuple(s1), tuple(s2))
    # draws of "sample" 37 of seed 0, diagram 0 are steps 37*32 .. 37*32+27
    assert m.draws(0, 0, 37, 28) == outs[37 * 32:37 * 32 + 28]


def test_jumps_compose():
    a1, a2 = m.matrices()
    p, k = (5 << 127) + (3 << 96) + (123456789 << 5), 977
    s1, s2 = m.state_at(p)
    t1 = m.mat_vec(m.mat_pow(a1, k, m.M1), list(s1), m.M1)
    t2 = m.mat_vec(m.mat_pow(a2, k, m.M2), list(s2), m.M2)
    assert m.state_at(p + k) == (tuple(t1), tuple(t2))


def test_uniform_map_and_moments():
    # z = 0 maps to m1/(m1+1); every output strictly inside (0, 1)
    s1 = (0, 0, 0)
    s2 = (0, 0, 0)
    assert m.step(s1, s2)[2] == m.M1 * m.NORM
    u = m.uniforms(np.arange(400), 2, 7, 28)
    assert u.shape == (400, 28)
    assert np.all((u > 0) & (u < 1))
    assert abs(u.mean() - 0.5) < 0.01
    assert abs(u.var() - 1 / 12) < 0.003
    # independent of the Philox stream of the same sample
    from oracle.philox import uniforms as pu
    assert abs(np.corrcoef(u.ravel(), pu(np.arange(400), 2, 7, 28).ravel())[0, 1]) < 0.03


def test_consecutive_samples_equal_jumps():
    idx = np.array([7, 8, 9, 10, 500, 501, 3], dtype=np.uint64)
    u = m.uniforms(idx, 4, 2, 28)
    for r, i in enumerate(idx):
        assert list(u[r]) == m.draws(2, 4, int(i), 28)


def test_stream_layout():
    u = m.uniforms(np.array([0, 5, 10**12]), 3, 11, 4)
    for r, s in enumerate((0, 5, 10**12)):
        pos = (11 << 127) + (3 << 96) + (s << 5)
        s1, s2 = m.state_at(pos)
        for d in range(4):
            s1, s2, x = m.step(s1, s2)
            assert u[r, d] == x
