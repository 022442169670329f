"""FP64 interval arithmetic on the bytecode integrands (Sec. 3: the round-off
of the numerical subtraction is removed with interval arithmetic), through
the C ABI.

* Enclosure: at Eq. (1) points of two-, three- and four-loop graphs the
  interval [lo, hi] contains the double-double value of the same program
  (the same FP64 constants, ~2^-104 kappa accurate) up to the final
  rounding of that value to FP64, and, at two loops, the oracle's integrand
  in 34-digit mpmath up to the rounding of the program's constants (a few
  ulp of the sum of the absolute values of the monomials, bounded here by
  the interval's own width or 1e-15).
* Sharpness: where the FP64 estimate accepts a point at 1e-12, the interval
  is narrow too (relative width below 1e-9), so the interval rule does not
  send well-conditioned points to the double-double pass wholesale.
* The interval flag rule: an integration in which every point is evaluated
  in interval arithmetic and the rest re-evaluated in double-double gives,
  on the same samples, the estimate rule's value within the thresholds.
"""
from pathlib import Path

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1905_08007_b300 as q                     # noqa: E402
from oracle.graphs import enumerate_graphs as o_enum   # noqa: E402
from oracle.integrand import Integrand                 # noqa: E402

GOLD = Path(__file__).parent / "golden"


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return q.Context(0, threshold=1e-12, prefer_programs=True)


def _ulp(x):
    return np.spacing(np.abs(x))


def _check_encloses_dd(d, z):
    lo, hi = d.eval_interval(z)
    fdd = d.eval_points(z, prec=1)
    lo, hi, fdd = lo.cpu().numpy(), hi.cpu().numpy(), fdd.cpu().numpy()
    fin = np.isfinite(lo) & np.isfinite(hi)
    assert fin.mean() > 0.9
    assert np.all(lo[fin] <= hi[fin])
    slack = 2 * _ulp(fdd[fin])
    assert np.all(lo[fin] - slack <= fdd[fin]) and np.all(fdd[fin] <= hi[fin] + slack)
    return lo, hi, fdd, fin


@pytest.mark.parametrize("gi", range(4))
def test_two_loop_interval_encloses_dd_and_the_oracle(ctx, gi):
    # the programs exist for one graph of each mirror pair
    g = q.enumerate_graphs(2, reduced=True)[gi]
    d = ctx.load(g)
    z, f, lp, fl = d.dump_points(0, 700, seed=5)
    lo, hi, fdd, fin = _check_encloses_dd(d, z)
    # the oracle in 34-digit arithmetic on a subsample
    import mpmath
    og = next(x for x in o_enum(2) if (tuple(x.pairs), x.e) == (tuple(g.pairs), g.e))
    zz = z.cpu().numpy()
    # the 34-digit oracle takes seconds per two-loop point: four points
    idx = [i for i in range(0, 700, 175) if fin[i]]
    with mpmath.workdps(34):
        zo = np.array([[mpmath.mpf(float(v)) for v in zz[i]] for i in idx], dtype=object)
        ref = Integrand(og)(zo, dtype=object)
    for j, i in enumerate(idx):
        ex = float(ref[j])
        slack = max(hi[i] - lo[i], 1e-15 * abs(ex))
        assert lo[i] - slack <= ex <= hi[i] + slack, (i, lo[i], hi[i], ex)
    # sharpness where the estimate accepts the point
    ok = (fl.cpu().numpy() == 0) & fin
    if ok.any():
        mid = 0.5 * (lo[ok] + hi[ok])
        assert np.all((hi[ok] - lo[ok]) <= 1e-9 * np.abs(mid))


@pytest.mark.parametrize("gi", [0, 13, 27])
def test_three_loop_interval_encloses_dd(ctx, gi):
    g = q.enumerate_graphs(3, reduced=True)[gi]
    d = ctx.load(g)
    z = d.dump_points(10**6, 300, seed=2)[0]
    _check_encloses_dd(d, z)


def test_four_loop_interval_encloses_dd(ctx):
    rows = [ln.split() for ln in (GOLD / "four_loop_points.txt").read_text().splitlines()
            if ln and not ln.startswith("#")]
    gis = sorted({int(r[0]) for r in rows})[:6]
    c4 = q.Context(0, threshold=1e-12)
    every = q.enumerate_graphs(4)
    for gi in gis:
        d = c4.load(every[gi])
        z = d.dump_points(0, 64, seed=0)[0]
        lo, hi, fdd, fin = _check_encloses_dd(d, z)
        rel = (hi[fin] - lo[fin]) / np.abs(0.5 * (lo[fin] + hi[fin]))
        assert np.median(rel) < 1e-6


def test_degenerate_inputs(ctx):
    d = ctx.load(q.enumerate_graphs(2)[1])
    z = torch.empty((0, d.n_lines), dtype=torch.float64, device="cuda")
    lo, hi = d.eval_interval(z)
    assert lo.numel() == 0
    # a compiled integrand has no interval evaluation
    cc = q.Context(0, programs=False)
    dc = cc.load(q.enumerate_graphs(2)[1])
    with pytest.raises(q.QedError):
        dc.eval_interval(torch.ones((4, dc.n_lines), dtype=torch.float64, device="cuda"))
    cc.set_flag_rule("interval")
    with pytest.raises(q.QedError):
        dc.integrate(1000)


@pytest.mark.parametrize("gi", [1, 3])
def test_interval_rule_integration_matches_estimate_rule(gi):
    g = q.enumerate_graphs(2, reduced=True)[gi]
    res = {}
    for rule in ("estimate", "interval"):
        c = q.Context(0, threshold=1e-9, prefer_programs=True, flag_rule=rule)
        res[rule] = c.load(g).integrate(1 << 21, seed=9)
    a, b = res["estimate"], res["interval"]
    assert a.n == b.n == 1 << 21
    # same samples; accepted values agree to the thresholds, flagged ones
    # are re-evaluated in double-double either way
    assert b.value == pytest.approx(a.value, rel=1e-6, abs=1e-9)
    assert b.variance == pytest.approx(a.variance, rel=1e-4)
    assert b.n_flagged >= 0 and b.n_unstable <= max(10, 2 * a.n_unstable + 10)
    print(f"graph {gi}: flagged estimate {a.n_flagged}, interval {b.n_flagged}; "
          f"unstable {a.n_unstable} / {b.n_unstable}")
