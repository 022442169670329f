"""Oracle pins for the subtracted integrand: the one-loop closed form and
A_1^(2) = 1/2 (Sec. 1, Schwinger), homogeneity, mirror symmetry (Sec. 3
footnote), pointwise UV finiteness of the forest formula (Sec. 2 item 1),
integrability of every single-set limit at two loops and of the nested
shell limits of the three-loop rainbow graph, and the Monte Carlo estimator
on the one-loop graph."""
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


def _exponent(f, z0, S, e1, e2, dtype):
    """Local exponent delta of |f| eps^|S| under z_S -> eps z_S between e1 and
    e2, per base point: the limit is integrable where delta > 0 (a finite
    integral needs |f| eps^|S| -> 0; a logarithmic divergence has delta 0)."""
    out = []
    for e in (e1, e2):
        z = np.array(z0, dtype=dtype)
        z[:, S] *= e
        out.append(np.abs(np.asarray(f(z, dtype=dtype), dtype=np.float64)) * e ** len(S))
    return np.log(out[1] / out[0]) / math.log(e2 / e1)


@pytest.mark.parametrize("gi", range(6))
def test_two_loop_every_single_set_limit_is_integrable(gi):
    """Sec. 2: each graph's subtracted integrand has a finite integral.  Every
    proper subset S of the lines, scaled to zero at two base points (all UV
    limits, all IR limits -- a photon's parameter growing is its complement
    shrinking -- and every mixed one), keeps |f| eps^|S| falling."""
    g = enumerate_graphs(2)[gi]
    f = Integrand(g)
    z0 = np.random.default_rng(40 + gi).dirichlet([1] * 6, size=2)
    worst = 9.0
    for m in range(1, 63):
        S = [l for l in range(6) if m >> l & 1]
        d = _exponent(f, z0, S, 1e-4, 1e-6, np.longdouble)
        worst = min(worst, float(d.min()))
        assert np.all(d > 0.5), (S, d)
    assert worst < 1.2


def test_three_loop_rainbow_shell_limits_are_integrable():
    """The three-loop rainbow graph (photons nested around X) has the two
    nested X-subgraphs G' (lines 2, 3, photon 8) and G'' (lines 1-4, photons
    7, 8).  The shell G''\\G' (lines 1, 4, photon 7) is a UV-divergent
    subgraph of the block G/G' in the forest terms where G' gets A: with the
    operator reading of item 3 (L on G'', L - U on the root) |f| eps^3 falls
    like eps; giving G'' the operator L - U instead leaves it constant (a
    logarithmically divergent integral)."""
    g = enumerate_graphs(3)[47]
    assert g.pairs == ((0, 5), (1, 4), (2, 3)) and g.e == 3
    f = Integrand(g)
    z0 = np.random.default_rng(5).dirichlet([1] * 9, size=2)
    for S in ([1, 4, 7], [0, 5, 6], [0, 1, 4, 5, 6, 7], [1, 2, 3, 4, 7, 8]):
        d = _exponent(f, z0, S, 1e-3, 1e-5, np.float64)
        assert np.all(d > 0.8), (S, d)


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
