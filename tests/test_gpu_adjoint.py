"""GPU tests of the density adjoint: the library's M2 and dM2/dtheta equal the
oracle's score-function estimate on the same Philox points; the tuned density
samples from the oracle's tuned sampler point for point; gradient descent
through the torch.autograd.Function lowers the second moment while the mean
stays within its error."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1905_08007_b300 as q                         # noqa: E402
from paper_1905_08007_b300.tune import pdf_grad, tune, _set_params   # noqa: E402
from oracle.adjoint import m2_grad, sample_theta           # noqa: E402
from oracle.graphs import deg_table, enumerate_graphs as o_enum  # noqa: E402
from oracle.integrand import Integrand                     # noqa: E402
from oracle.philox import uniforms                         # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return q.Context(0)


THETA = {3: ([0.2, -0.1, 0.15], [0.1, 0.0, -0.2]),
         6: ([0.1, -0.05, 0.2, 0.0, -0.1, 0.05], [0.2, -0.1, 0.0, 0.1, -0.2, 0.3])}


@pytest.mark.parametrize("n,gi", [(1, 0), (2, 0), (2, 4)])
def test_tuned_points_match_oracle(ctx, n, gi):
    g = q.enumerate_graphs(n)[gi]
    og = o_enum(n)[gi]
    d = ctx.load(g)
    a, b = THETA[og.n_lines]
    _set_params(d, a, b)
    z, f, lp, fl = d.dump_points(0, 777, seed=2)
    N = og.n_lines
    u = uniforms(np.arange(777), g.stream_id, 2, 2 * (N - 1))
    x, lpo, *_ = sample_theta(u, deg_table(og), a, b, N)
    np.testing.assert_allclose(z.cpu().numpy(), x, rtol=1e-12)
    np.testing.assert_allclose(lp.cpu().numpy(), lpo, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("n,gi,tol", [(1, 0, 1e-10), (2, 0, 1e-6), (2, 4, 1e-6)])
def test_gradient_matches_oracle_on_same_points(ctx, n, gi, tol):
    g = q.enumerate_graphs(n)[gi]
    og = o_enum(n)[gi]
    d = ctx.load(g)
    a, b = THETA[og.n_lines]
    cnt = 1500 + 17
    m2, ga, gb = pdf_grad(d, a, b, cnt, seed=7, begin=123)
    m2o, gao, gbo = m2_grad(Integrand(og), og, g.stream_id, 7, 123, cnt, a, b)
    assert m2 == pytest.approx(m2o, rel=tol)
    scale = max(np.max(np.abs(gao)), np.max(np.abs(gbo)))
    np.testing.assert_allclose(ga, gao, rtol=tol, atol=tol * scale)
    np.testing.assert_allclose(gb, gbo, rtol=tol, atol=tol * scale)


def test_tuning_lowers_second_moment_unbiased(ctx):
    g = q.enumerate_graphs(2)[1]
    d = ctx.load(g)
    before = d.integrate(1 << 24, seed=21)
    a, b, hist = tune(d, steps=12, n=1 << 21, lr=0.08)
    after = d.integrate(1 << 24, seed=21)
    assert after.variance < before.variance
    assert abs(after.value - before.value) < 4 * math.sqrt(after.variance + before.variance)


def test_calibrated_deg_caps_rule_and_matches_oracle_sampler(ctx):
    """Calibrated Deg: never above the rule, positive, and the oracle samples
    the same points from the table read back from the library."""
    from oracle.pdf import f_table, sample_points
    g = q.enumerate_graphs(2)[3]
    og = o_enum(2)[3]
    d = ctx.load(g)
    rule = d.deg_table()
    d.calibrate_deg(n_base=8, seed=1)
    cal = d.deg_table()
    N = og.n_lines
    assert all(0 < cal[m] <= rule[m] + 1e-15 for m in range(1, (1 << N) - 1))
    # the complement of the self-energy subgraph (lines 0, 1, 3, 4) is lowered
    assert cal[0b011011] < rule[0b011011]
    z, f, lp, fl = d.dump_points(0, 500, seed=4)
    u = uniforms(np.arange(500), g.stream_id, 4, 2 * (N - 1))
    x, lpo, _ = sample_points(u, cal, f_table(cal, N), N)
    np.testing.assert_allclose(z.cpu().numpy(), x, rtol=1e-12)
    np.testing.assert_allclose(lp.cpu().numpy(), lpo, rtol=1e-12, atol=1e-12)


def test_gradient_at_flagged_points_uses_double_double():
    """Threshold 1e-12 on a self-energy graph: most points fail the FP64
    estimate.  The adjoint then sums their double-double values (as the
    estimator does), and M2 and its gradient match the long-double oracle
    far below the FP64 cancellation noise those points carry."""
    c = q.Context(0, threshold=1e-12)
    g = q.enumerate_graphs(2)[4]
    og = o_enum(2)[4]
    d = c.load(g)
    a, b = THETA[og.n_lines]
    _set_params(d, a, b)
    cnt = 1200 + 9
    _, _, _, fl = d.dump_points(123, cnt, seed=7)
    assert (fl.cpu().numpy() != 0).mean() > 0.1
    m2, ga, gb = pdf_grad(d, a, b, cnt, seed=7, begin=123)
    m2o, gao, gbo = m2_grad(Integrand(og), og, g.stream_id, 7, 123, cnt, a, b)
    assert m2 == pytest.approx(m2o, rel=1e-9)
    scale = max(np.max(np.abs(gao)), np.max(np.abs(gbo)))
    np.testing.assert_allclose(ga, gao, rtol=1e-9, atol=1e-9 * scale)
    np.testing.assert_allclose(gb, gbo, rtol=1e-9, atol=1e-9 * scale)


@pytest.mark.parametrize("gi", [0, 1])
def test_adjoint_matches_finite_differences_two_loops(ctx, gi):
    """Two-loop graphs: for every component of theta, the central difference
    (M2(theta + h e_m) - M2(theta - h e_m)) / 2h with common random numbers
    (the same Philox counters on both sides, so the difference keeps little
    noise) agrees with the adjoint's score-function estimate of dM2/dtheta_m
    within 3 sigma, sigma from 8 independent batches of each."""
    g = q.enumerate_graphs(2)[gi]
    d = ctx.load(g)
    N = d.n_lines
    a0, b0 = THETA[N]
    theta = np.array(list(a0) + list(b0))
    h, n, B = 0.02, 1 << 21, 8
    adj = np.zeros((B, 2 * N))
    fd = np.zeros((B, 2 * N))
    for b in range(B):
        begin = 5_000_000 + b * n
        _, ga, gb = pdf_grad(d, theta[:N], theta[N:], n, seed=11, begin=begin)
        adj[b] = ga + gb
        for m in range(2 * N):
            tp, tm = theta.copy(), theta.copy()
            tp[m] += h
            tm[m] -= h
            mp, _, _ = pdf_grad(d, tp[:N], tp[N:], n, seed=11, begin=begin)
            mm, _, _ = pdf_grad(d, tm[:N], tm[N:], n, seed=11, begin=begin)
            fd[b, m] = (mp - mm) / (2 * h)
    ma, mf = adj.mean(0), fd.mean(0)
    se = np.sqrt(adj.var(0, ddof=1) / B + fd.var(0, ddof=1) / B)
    assert np.all(np.abs(ma - mf) <= 3 * se + 1e-3 * np.abs(mf)), (ma, mf, se)
