"""Oracle pins: graph polynomials (Kirchhoff, derivative identity, one-loop
closed forms) and the F2(0) projection on vertices of known form."""
import numpy as np
import pytest

from oracle import dirac
from oracle.graphs import enumerate_graphs
from oracle.integrand import TermEvaluator
from oracle.polys import polynomials, spanning_tree_u


def _main_term(g):
    ev = TermEvaluator(g, "q", "F2", [])
    return ev


@pytest.mark.parametrize("n", [1, 2, 3])
def test_u_is_kirchhoff_spanning_tree_sum(n):
    rng = np.random.default_rng(n)
    for g in enumerate_graphs(n)[:8]:
        ev = _main_term(g)
        z = rng.random(g.n_lines) + 0.1
        P = polynomials(z, ev.eta, ev.alpha, ev.beta, ev.kappa, ev.mass2)
        edges = [g.line_ends(l) for l in range(g.n_lines)]
        assert P["U"][0] == pytest.approx(spanning_tree_u(edges, 2 * g.n + 1, z), rel=1e-12)


@pytest.mark.parametrize("n", [4, 5])
def test_extended_precision_u_and_adjugate(n):
    """The long-double path (cofactor expansion) at four and five loops:
    U against the spanning-tree sum, adj against det * inverse."""
    rng = np.random.default_rng(10 + n)
    for g in enumerate_graphs(n)[:: 97 if n == 4 else 1201][:4]:
        ev = _main_term(g)
        z = rng.random(g.n_lines) + 0.1
        P = polynomials(z, ev.eta, ev.alpha, ev.beta, ev.kappa, ev.mass2, dtype=np.longdouble)
        P64 = polynomials(z, ev.eta, ev.alpha, ev.beta, ev.kappa, ev.mass2)
        edges = [g.line_ends(l) for l in range(g.n_lines)]
        assert float(P["U"][0]) == pytest.approx(spanning_tree_u(edges, 2 * g.n + 1, z), rel=1e-13)
        np.testing.assert_allclose(P["adj"][0].astype(float), P64["adj"][0], rtol=1e-10, atol=1e-14)


def test_b_diagonal_is_derivative_of_u():
    g = enumerate_graphs(2)[1]
    ev = _main_term(g)
    z = np.array([0.3, 0.2, 0.5, 0.7, 0.4, 0.9])
    P = polynomials(z, ev.eta, ev.alpha, ev.beta, ev.kappa, ev.mass2)
    for i in range(g.n_elec):
        h = 1e-6
        zp, zm = z.copy(), z.copy()
        zp[i] += h
        zm[i] -= h
        up = polynomials(zp, ev.eta, ev.alpha, ev.beta, ev.kappa, ev.mass2)["U"][0]
        um = polynomials(zm, ev.eta, ev.alpha, ev.beta, ev.kappa, ev.mass2)["U"][0]
        bii = ev.eta[i] @ P["adj"][0] @ ev.eta[i]
        assert bii == pytest.approx((up - um) / (2 * h), rel=1e-8)


def test_one_loop_closed_forms():
    g = enumerate_graphs(1)[0]
    ev = _main_term(g)
    z = np.array([[0.2, 0.3, 0.5], [0.1, 0.6, 0.3]])
    P = polynomials(z, ev.eta, ev.alpha, ev.beta, ev.kappa, ev.mass2)
    U = z.sum(1)
    np.testing.assert_allclose(P["U"], U)
    np.testing.assert_allclose(P["A"][:, 0], z[:, 2] / U)
    np.testing.assert_allclose(P["V"], (z[:, 0] + z[:, 1]) ** 2 / U)


def _sigma(m, n):
    return 0.5j * (dirac.GAMMA[m] @ dirac.GAMMA[n] - dirac.GAMMA[n] @ dirac.GAMMA[m])


def test_f2_projection_on_known_vertices():
    rng = np.random.default_rng(0)
    for _ in range(5):
        a, b, c = rng.normal(size=3)
        G = np.array([a * dirac.GAMMA[m] for m in range(4)])
        H = np.zeros((4, 3, 4, 4), complex)
        for m in range(4):
            for j in range(3):
                # b i sigma^{mu nu} q_nu / 2m  +  c q^mu (no moment)
                H[m, j] = -b * 1j * _sigma(m, j + 1) / 2 + (c * dirac.ONE if m == j + 1 else 0)
        # structures that vanish between on-shell spinors
        Pm = dirac.GAMMA[0] - dirac.ONE
        G2 = G + np.array([Pm @ dirac.GAMMA[m] @ Pm + (Pm if m == 0 else 0) for m in range(4)])
        assert dirac.f2_of_vertex(G, H).real == pytest.approx(b, abs=1e-13)
        assert dirac.f2_of_vertex(G2, H).real == pytest.approx(b, abs=1e-13)
        assert dirac.l_of_vertex(G).real == pytest.approx(a, abs=1e-13)
        assert dirac.gamma_mu_coeff(G).real == pytest.approx(a, abs=1e-13)
