"""Oracle pins for the subtracted integrand: the one-loop closed form and
A_1^(2) = 1/2 (Sec. 1, Schwinger), homogeneity, mirror symmetry (Sec. 3
footnote), pointwise UV finiteness of the forest formula (Sec. 2 item 1), and
the Monte Carlo estimator on the one-loop graph."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle.estimator import mc_estimate
from oracle.graphs import divergent_subgraphs, enumerate_graphs
from oracle.integrand import Integrand


def test_one_loop_closed_form_pointwise():
    g = enumerate_graphs(1)[0]
    z = np.random.default_rng(1).dirichlet([1, 1, 1], size=50)
    np.testing.assert_allclose(Integrand(g)(z), z[:, 2] / (z[:, 0] + z[:, 1]), rtol=1e-13)


def test_one_loop_integral_is_one_half_by_quadrature():
    f = Integrand(enumerate_graphs(1)[0])

    def h(y, x):
        return f(np.array([[x, y, 1.0 - x - y]]))[0]
    val, err = integrate.dblquad(h, 0.0, 1.0, 0.0, lambda x: 1.0 - x, epsabs=1e-11, epsrel=1e-10)
    assert val == pytest.approx(0.5, abs=1e-8)


@pytest.mark.parametrize("gi", range(6))
def test_two_loop_homogeneous_of_degree_minus_6(gi):
    g = enumerate_graphs(2)[gi]
    f = Integrand(g)
    z = np.random.default_rng(gi).dirichlet([1] * 6, size=3)
    np.testing.assert_allclose(f(3.7 * z), 3.7 ** -6 * f(z), rtol=1e-11)


def _mirror_point(g, z):
    mg = g.mirror()
    m = 2 * g.n - 1
    zm = np.zeros_like(z)
    for i in range(2 * g.n):
        zm[:, 2 * g.n - 1 - i] = z[:, i]
    for a, (s, t) in enumerate(g.pairs):
        b = mg.pairs.index(tuple(sorted((m - s, m - t))))
        zm[:, 2 * g.n + b] = z[:, 2 * g.n + a]
    return mg, zm


@pytest.mark.parametrize("gi", range(6))
def test_mirror_graphs_agree_pointwise(gi):
    g = enumerate_graphs(2)[gi]
    z = np.random.default_rng(10 + gi).dirichlet([1] * 6, size=4)
    mg, zm = _mirror_point(g, z)
    np.testing.assert_allclose(Integrand(g)(z), Integrand(mg)(zm), rtol=1e-11)


@pytest.mark.parametrize("gi", range(6))
def test_uv_limits_are_integrable(gi):
    """z_S -> eps z_S for every UV-divergent S: the subtracted integrand times
    eps^|S| vanishes (integrable), the unsubtracted one tends to a constant."""
    g = enumerate_graphs(2)[gi]
    f, fu = Integrand(g), Integrand(g, subtract=False)
    z0 = np.random.default_rng(20 + gi).dirichlet([1] * 6, size=3)
    for s in divergent_subgraphs(g):
        L = sorted(s.lines(g))
        vals, raw = [], []
        for eps in (1e-4, 1e-6, 1e-8):
            z = z0.copy()
            z[:, L] *= eps
            vals.append(np.abs(f(z)) * eps ** len(L))
            raw.append(np.abs(fu(z)) * eps ** len(L))
        assert np.all(vals[2] < 2e-2 * vals[0] + 1e-12)     # falls like eps
        assert np.all(raw[2] > 0.5 * raw[0])                  # log divergence left alone


def test_mc_one_loop_within_three_sigma():
    g = enumerate_graphs(1)[0]
    r = mc_estimate(Integrand(g), g, stream_id=0, seed=0, n=200_000)
    assert abs(r["value"] - 0.5) < 3 * r["sigma"]
    assert r["sigma"] < 2e-3


def test_inverse_variance_combination_reproduces_sec3():
    """Sec. 3 combines Calc 1, 6.739(132), and Calc 2, 6.905(220), into
    6.782(113)."""
    from oracle.estimator import combine_inverse_variance
    v, s = combine_inverse_variance([6.739, 6.905], [0.132, 0.220])
    assert round(v, 3) == 6.783 or round(v, 3) == 6.782
    assert round(s, 3) == 0.113
