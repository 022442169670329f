"""The two-loop lepton-loop-free total against its closed form
(197/144 + pi^2/12 - pi^2 ln2/2 + 3 zeta(3)/4) - (119/36 - pi^2/3): the
Petermann-Sommerfield A_1^(4) (Sec. 1) minus its vacuum-polarisation part,
from 1e8 samples per graph on the GPU, within 3 sigma."""
import math

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1905_08007_b300 as q   # noqa: E402

ZETA3 = 1.2020569031595942
TARGET = (197 / 144 + math.pi ** 2 / 12 - math.pi ** 2 * math.log(2) / 2 + 3 * ZETA3 / 4) \
    - (119 / 36 - math.pi ** 2 / 3)


def test_closed_form_value():
    assert TARGET == pytest.approx(-0.34416638743829586, abs=1e-15)


def test_two_loop_total_within_three_sigma():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    ctx = q.Context(0)
    tot, var = 0.0, 0.0
    per = []
    for g in q.enumerate_graphs(2):
        r = ctx.load(g).integrate(10**8, seed=0)
        per.append((g.pairs, g.e, r.value, r.sigma, r.n_flagged, r.n_unstable))
        tot += r.value
        var += r.variance
    sig = math.sqrt(var)
    print("per-graph", per)
    print(f"total {tot:.6f} +- {sig:.6f}  target {TARGET:.6f}")
    assert abs(tot - TARGET) < 3 * sig, (tot, sig, per)


def test_two_loop_total_calibrated_tuned_batched():
    """Same closed form from the production path: Deg calibrated on the
    integrand's limits, densities gradient-tuned, all six graphs in the
    persistent batched launch with variance-driven allocation.  With finite
    variance the error bar is ~5e-4 at 6e8 samples, a tight pin of the
    subtraction reading."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1905_08007_b300.tune import tune
    ctx = q.Context(0)
    ds = [ctx.load(g) for g in q.enumerate_graphs(2)]
    for d in ds:
        d.calibrate_deg(n_base=8, seed=5)
        tune(d, steps=10, n=1 << 21, lr=0.08, seed=7)
    res = ctx.integrate_batch(ds, 6 * 10**8, seed=3, policy="variance", rounds=4, chunk=1 << 18)
    tot = sum(r.value for r in res)
    sig = math.sqrt(sum(r.variance for r in res))
    print(f"calibrated+tuned total {tot:.6f} +- {sig:.6f}  target {TARGET:.6f}")
    assert sig < 2e-3
    assert abs(tot - TARGET) < 3 * sig, (tot, sig)
