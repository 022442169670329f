"""Oracle pins for the tunable density and the gradient of the second
moment: at theta = 0 the tuned sampler is the Eq. (1) sampler; the complex-step
d log Z / d theta matches central differences; on the one-loop graph the
score-function gradient estimate matches the derivative of M2(theta) computed
by deterministic quadrature (2-dim simplex)."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle.adjoint import dlogz_complex_step, log_z, m2_grad, sample_theta
from oracle.graphs import deg_table, enumerate_graphs
from oracle.integrand import Integrand
from oracle.pdf import f_table, sample_points
from oracle.philox import uniforms


def test_theta_zero_is_eq1_sampler():
    g = enumerate_graphs(2)[1]
    N = g.n_lines
    deg = deg_table(g)
    u = uniforms(np.arange(200), 1, 3, 2 * (N - 1))
    x0, lp0, o0 = sample_points(u, deg, f_table(deg, N), N)
    x1, lp1, o1, *_ = sample_theta(u, deg, [0.0] * N, [0.0] * N, N)
    np.testing.assert_array_equal(o0, o1)
    np.testing.assert_allclose(x0, x1, rtol=1e-14)
    np.testing.assert_allclose(lp0, lp1, rtol=1e-13, atol=1e-13)


def test_complex_step_matches_central_differences():
    g = enumerate_graphs(2)[4]
    N = g.n_lines
    deg = deg_table(g)
    rng = np.random.default_rng(0)
    a = list(0.1 * rng.normal(size=N))
    b = list(0.3 * rng.normal(size=N))
    ga, gb = dlogz_complex_step(deg, a, b, N)
    h = 1e-6
    for m in range(N):
        ap, am = list(a), list(a)
        ap[m] += h
        am[m] -= h
        fd = (log_z(deg, ap, b, N).real - log_z(deg, am, b, N).real) / (2 * h)
        assert ga[m] == pytest.approx(fd, rel=1e-6, abs=1e-9)
        bp, bm = list(b), list(b)
        bp[m] += h
        bm[m] -= h
        fd = (log_z(deg, a, bp, N).real - log_z(deg, a, bm, N).real) / (2 * h)
        assert gb[m] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def _m2_quadrature(alpha, beta):
    """M2(theta) = int f^2 / p over the one-loop simplex."""
    from oracle.adjoint import tables
    g = enumerate_graphs(1)[0]
    deg0 = deg_table(g)
    deg, act, F = tables(deg0, alpha, beta, 3)
    full = 7
    Z = sum(math.exp(beta[j]) * F[full & ~(1 << j)] / deg[full & ~(1 << j)] for j in range(3))

    def logp(z):
        order = sorted(range(3), key=lambda i: -z[i])
        s = full
        lp = beta[order[0]] - math.log(Z)
        for l in range(1, 3):
            s &= ~(1 << order[l - 1])
            lp += deg[s] * (math.log(z[order[l]]) - math.log(z[order[l - 1]]))
        return lp - sum(math.log(v) for v in z)

    def h(y, x):
        z = np.array([x, y, 1.0 - x - y])
        if np.any(z <= 0):
            return 0.0
        f = z[2] / (z[0] + z[1])
        return f * f * math.exp(-logp(z))
    v, _ = integrate.dblquad(h, 0, 1, 0, lambda x: 1 - x, epsabs=1e-12, epsrel=1e-10)
    return v


def test_one_loop_gradient_matches_quadrature_derivative():
    g = enumerate_graphs(1)[0]
    alpha = [0.2, -0.1, 0.15]
    beta = [0.1, 0.0, -0.2]
    f = Integrand(g)
    # score-function estimate over batches, for its error bar
    est = [m2_grad(f, g, 0, 1, b * 20000, 20000, alpha, beta, dtype=np.float64) for b in range(8)]
    m2 = np.mean([e[0] for e in est])
    ga = np.mean([e[1] for e in est], axis=0)
    ga_se = np.std([e[1] for e in est], axis=0, ddof=1) / math.sqrt(len(est))
    assert m2 == pytest.approx(_m2_quadrature(alpha, beta), rel=0.02)
    h = 1e-3
    for m in (0, 2):
        ap, am = list(alpha), list(alpha)
        ap[m] += h
        am[m] -= h
        fd = (_m2_quadrature(ap, beta) - _m2_quadrature(am, beta)) / (2 * h)
        assert abs(ga[m] - fd) < 4 * ga_se[m] + 1e-3 * abs(fd), (m, ga[m], fd, ga_se[m])
