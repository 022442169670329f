"""GPU parity tests through the C ABI: the CUDA path against the CPU oracle
on the same Philox points (points, Eq. (1) density, integrand), sized to span
several blocks and a ragged tail, plus sampled points at the end of the
1e8-sample range the bench uses; estimator checks against A_1^(2) = 1/2.

Tolerances: points and log p to 1e-12 (both sides draw the same counters and
take the sector decisions in FP64 with the same tables and order; log/exp
differ by ulps); integrand to 1e-12 relative on points whose rounding-error
estimate is below the threshold (the forest terms cancel, so the error of
both FP64 evaluations grows with sum|t|/|f|, which is what the flag bounds).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1905_08007_b300 as q                     # noqa: E402
from oracle.graphs import deg_table, enumerate_graphs as o_enum   # noqa: E402
from oracle.integrand import Integrand                 # noqa: E402
from oracle.pdf import density, f_table, sample_points # noqa: E402
from oracle.philox import uniforms                     # noqa: E402

GRAPHS = [(1, 0)] + [(2, i) for i in range(6)]


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    # threshold 1e-12: every point the FP64 path accepts must be good to 1e-12
    return q.Context(0, threshold=1e-12)


def _oracle_points(og, stream, seed, begin, n):
    N = og.n_lines
    deg = deg_table(og)
    F = f_table(deg, N)
    u = uniforms(np.arange(begin, begin + n, dtype=np.uint64), stream, seed, 2 * (N - 1))
    x, lp, _ = sample_points(u, deg, F, N)
    return x, lp, deg, math.log(F[-1])


@pytest.mark.parametrize("n,gi", GRAPHS)
@pytest.mark.parametrize("begin,count", [(0, 512 + 37), (10**8 - 333, 333)])
def test_points_density_integrand_match_oracle(ctx, n, gi, begin, count):
    g = q.enumerate_graphs(n)[gi]
    og = o_enum(n)[gi]
    d = ctx.load(g)
    z, f, lp, fl = d.dump_points(begin, count, seed=0)
    z, f, lp, fl = z.cpu().numpy(), f.cpu().numpy(), lp.cpu().numpy(), fl.cpu().numpy()
    xo, lpo, deg, logZ = _oracle_points(og, g.stream_id, 0, begin, count)
    # same sector for every point (an integer decision taken in FP64 on both sides)
    assert np.array_equal(np.argsort(-z, axis=1, kind="stable"), np.argsort(-xo, axis=1, kind="stable"))
    np.testing.assert_allclose(z, xo, rtol=1e-12, atol=0)
    np.testing.assert_allclose(lp, lpo, rtol=1e-12, atol=1e-12)
    # density of Eq. (1) re-evaluated directly at the GPU's point
    lpd = np.array([density(z[i], deg, logZ) for i in range(0, count, 7)])
    np.testing.assert_allclose(lp[::7], lpd, rtol=1e-12, atol=1e-12)
    # integrand at the GPU's own point.  Both sides in FP64 on every point:
    # they round differently where the forest terms cancel, so this broad
    # check uses 1e-9 on the points the GPU accepts in FP64
    fo = Integrand(og)(z)
    ok = fl == 0
    # at 1e-12 the self-energy graphs flag most points (their forest terms
    # cancel to many digits); the flagged ones are checked in double-double
    assert ok.mean() > 0.15
    rel = np.abs(f[ok] - fo[ok]) / np.abs(fo[ok])
    assert rel.max() < 1e-9, rel.max()
    # strict check, 1e-12 relative, on a subsample: accepted FP64 values and
    # double-double values of flagged points against the long-double oracle;
    # where the two disagree (the oracle's own V = sum z - sum z A^2 cancels
    # at IR corners, even in long double) the arbiter is the oracle in
    # arbitrary precision (mpmath, 34 digits) on every such point
    sub = np.arange(0, count, 10)
    fld = Integrand(og)(z[sub], dtype=np.longdouble).astype(np.float64)
    zt = torch.tensor(z[sub], dtype=torch.float64, device="cuda")
    fdd = d.eval_points(zt, prec=1).cpu().numpy()
    gpu = np.where(ok[sub], f[sub], fdd)
    rel = np.abs(gpu - fld) / np.abs(fld)
    _arbitrate(og, z[sub], gpu, rel)


def _arbitrate(og, zs, gpu, rel, tol=1e-12, cap=64):
    """Every point where the GPU value and the long-double oracle differ by
    more than tol is settled by the oracle in 34-digit mpmath (the long-double
    oracle loses digits of its own where its V = sum z - sum z A^2 cancels).
    More than ``cap`` such points fail outright.  Returns (points settled by
    mpmath, largest verified relative error)."""
    import mpmath
    idx = np.nonzero(rel > tol)[0]
    assert len(idx) <= cap, f"{len(idx)} points above {tol} against the long-double oracle"
    worst = float(np.max(rel[rel <= tol])) if np.any(rel <= tol) else 0.0
    if len(idx) == 0:
        return 0, worst
    with mpmath.workdps(34):
        zo = np.array([[mpmath.mpf(float(v)) for v in zs[i]] for i in idx], dtype=object)
        ref = Integrand(og)(zo, dtype=object)
        for j, i in enumerate(idx):
            r = float(abs(mpmath.mpf(float(gpu[i])) - ref[j]) / abs(ref[j]))
            assert r < tol, (int(i), r, gpu[i], float(ref[j]))
            worst = max(worst, r)
    print(f"{og.pairs} e={og.e}: {len(rel)} points at {tol:g}, {len(idx)} settled by mpmath, "
          f"largest verified error {worst:.2e}")
    return len(idx), worst


@pytest.mark.parametrize("n,gi", GRAPHS)
def test_double_double_agrees_with_fp64_and_oracle(ctx, n, gi):
    g = q.enumerate_graphs(n)[gi]
    d = ctx.load(g)
    z, f, lp, fl = d.dump_points(0, 512, seed=3)
    fdd = d.eval_points(z, prec=1).cpu().numpy()
    f64 = d.eval_points(z, prec=0).cpu().numpy()
    ok = fl.cpu().numpy() == 0
    # separate kernels may fuse multiply-adds differently: equal to the error bound
    np.testing.assert_allclose(f64[ok], f.cpu().numpy()[ok], rtol=1e-12)
    np.testing.assert_allclose(f64[ok], fdd[ok], rtol=1e-12)
    sub = np.arange(0, 512, 16)
    og = o_enum(n)[gi]
    zz = z.cpu().numpy()[sub]
    fld = Integrand(og)(zz, dtype=np.longdouble).astype(np.float64)
    rel = np.abs(fdd[sub] - fld) / np.abs(fld)
    _arbitrate(og, zz, fdd[sub], rel)


def test_one_loop_estimate_is_one_half(ctx):
    d = ctx.load(q.enumerate_graphs(1)[0])
    r = d.integrate(10**7, seed=0)
    assert abs(r.value - 0.5) < 3 * r.sigma, (r.value, r.sigma)
    assert r.n == 10**7 and r.n_unstable == 0


def test_estimate_matches_oracle_sums_small(ctx):
    """Same samples, same moments: GPU sum of w vs the oracle's."""
    from oracle.estimator import mc_estimate
    g = q.enumerate_graphs(2)[4]
    d = ctx.load(g)
    n = 20000 + 123
    r = d.integrate(n, seed=5)
    ro = mc_estimate(Integrand(o_enum(2)[4]), o_enum(2)[4], g.stream_id, 5, n)
    # the GPU re-evaluates ill-conditioned points in double-double, the oracle
    # keeps its FP64 values there (relative errors up to ~1e-7 on a few
    # percent of points), so the sums agree to that level
    assert r.value == pytest.approx(ro["value"], rel=1e-6)
    assert r.variance == pytest.approx(ro["variance"], rel=1e-6)


def test_replicas_merge_to_single_run(ctx):
    d = ctx.load(q.enumerate_graphs(2)[1])
    full = d.integrate(3_000_000, seed=9)
    a = d.integrate(1_000_000, seed=9, begin=0)
    b = d.integrate(2_000_000, seed=9, begin=1_000_000)
    m = q.merge_results(a, b)
    assert m.n == full.n
    assert m.value == pytest.approx(full.value, rel=1e-12)
    assert m.variance == pytest.approx(full.variance, rel=1e-10)


def test_launch_shape_changes_only_rounding(ctx):
    d = ctx.load(q.enumerate_graphs(2)[3])
    r1 = d.integrate(500_000, seed=2)
    ctx.set_launch(128, 97)
    r2 = d.integrate(500_000, seed=2)
    ctx.set_launch(256, 0)
    assert r2.value == pytest.approx(r1.value, rel=1e-12)


def test_empty_range_and_bad_arguments(ctx):
    d = ctx.load(q.enumerate_graphs(1)[0])
    r = d.integrate(0, seed=0)
    assert r.n == 0 and r.value == 0.0
    with pytest.raises(q.QedError):
        ctx.set_launch(100, 0)
    with pytest.raises(q.QedError):
        ctx.load(q.Graph(2, ((0, 1), (2, 3)), 2))
    with pytest.raises(q.QedError):
        ctx.load(q.enumerate_graphs(1)[0], deg=np.zeros(8))


def test_queue_overflow_rescan_matches_chunked_runs():
    """More flagged points than the context's queue holds (2^22): the
    double-double kernel re-scans the chunk and replaces the first pass.
    The same samples in chunks that never overflow give the same estimate;
    the flag decisions are taken by different kernels there, so the flagged
    counts may differ by points at the threshold itself."""
    c = q.Context(0, threshold=1e-15)
    d = c.load(q.enumerate_graphs(2)[4])
    n = 6_000_011
    full = d.integrate(n, seed=17, begin=3)
    assert full.n_flagged > (1 << 22)
    parts = [d.integrate(2_000_000, seed=17, begin=3), d.integrate(2_000_000, seed=17, begin=2_000_003),
             d.integrate(2_000_011, seed=17, begin=4_000_003)]
    m = q.merge_results(q.merge_results(parts[0], parts[1]), parts[2])
    assert m.n == full.n
    assert abs(m.n_flagged - full.n_flagged) <= 1e-5 * n
    assert m.value == pytest.approx(full.value, rel=1e-10)
    assert m.variance == pytest.approx(full.variance, rel=1e-9)
