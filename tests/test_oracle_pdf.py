"""Oracle pins: the Eq. (1) density, its normaliser and the sector walk."""
import math

import numpy as np
import pytest
from scipy import integrate, stats

from oracle.graphs import deg_table, enumerate_graphs
from oracle.pdf import density, f_table, normaliser_bruteforce, sample_points
from oracle.philox import uniforms


@pytest.mark.parametrize("gi", range(6))
def test_normaliser_dp_equals_sum_over_sectors(gi):
    g = enumerate_graphs(2)[gi]
    deg = deg_table(g)
    F = f_table(deg, g.n_lines)
    assert F[-1] == pytest.approx(normaliser_bruteforce(deg, g.n_lines), rel=1e-13)


def test_density_integrates_to_one_by_quadrature():
    # N = 3: p on the 2-simplex with arbitrary positive Deg, by 2-d quadrature
    deg = [0.0, 1.7, 0.6, 2.2, 0.9, 1.3, 0.45, 0.0]
    F = f_table(deg, 3)
    lz = math.log(F[-1])

    def p(y, x):
        z = np.array([x, y, 1.0 - x - y])
        if np.any(z <= 0):
            return 0.0
        return math.exp(density(z, deg, lz))
    val, err = integrate.dblquad(p, 0.0, 1.0, 0.0, lambda x: 1.0 - x, epsabs=1e-10, epsrel=1e-9)
    assert val == pytest.approx(1.0, abs=1e-6)


def test_walk_density_equals_eq1_at_the_point():
    g = enumerate_graphs(2)[2]
    N = g.n_lines
    deg = deg_table(g)
    F = f_table(deg, N)
    u = uniforms(np.arange(300), 7, 99, 2 * (N - 1))
    x, lp, order = sample_points(u, deg, F, N)
    for i in range(300):
        assert np.argsort(-x[i]).tolist() == order[i].tolist()
        assert lp[i] == pytest.approx(density(x[i], deg, math.log(F[-1])), rel=1e-12, abs=1e-12)


def test_sector_frequencies_chi2_and_radial_ks():
    deg = [0.0, 1.7, 0.6, 2.2, 0.9, 1.3, 0.45, 0.0]
    F = f_table(deg, 3)
    n = 20000
    u = uniforms(np.arange(n), 0, 5, 4)
    x, lp, order = sample_points(u, deg, F, 3)
    # predicted sector probability: prod_l 1/Deg(S_l) / Z
    counts, probs = [], []
    from itertools import permutations
    for perm in permutations(range(3)):
        s = 7
        pr = 1.0
        for j in perm[:-1]:
            s &= ~(1 << j)
            pr /= deg[s]
        probs.append(pr / F[-1])
        counts.append(int(np.sum(np.all(order == np.array(perm), axis=1))))
    chi2, pval = stats.chisquare(counts, np.array(probs) * n)
    assert pval > 1e-3
    # t_2 = z_j2 / z_j1 ~ Beta(Deg(S_2), 1) within sector (0, 1, 2)
    m = np.all(order == np.array([0, 1, 2]), axis=1)
    t2 = x[m, 1] / x[m, 0]
    assert stats.kstest(t2, stats.beta(deg[0b110], 1).cdf).pvalue > 1e-3
