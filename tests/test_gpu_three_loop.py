"""Three-loop graphs (9 lines, 8-dim simplex): per-point parity of the CUDA
path with the oracle -- every graph at stored oracle points in long double
(tests/golden/three_loop_points.txt), a subset of graphs at fresh points --
and the batched persistent launch over all 50 graphs with 1e9 samples in
total and variance-driven allocation, checked against the per-graph path on
the same counters."""
import math
from pathlib import Path

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1905_08007_b300 as q                      # noqa: E402
from oracle.graphs import deg_table, enumerate_graphs as o_enum   # noqa: E402
from oracle.integrand import Integrand                  # noqa: E402
from oracle.pdf import f_table, sample_points           # noqa: E402
from oracle.philox import uniforms                      # noqa: E402

ROOT = Path(__file__).resolve().parents[1]
SUBSET = [0, 9, 19, 29, 39, 49]
GOLDEN3 = Path(__file__).resolve().parent / "golden" / "three_loop_points.txt"


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = q.Context(0, threshold=1e-12)
    try:
        c.load(q.enumerate_graphs(3)[0])
    except q.QedError as e:
        if e.code == -6:
            pytest.skip("library built without three-loop integrands")
        raise
    return c


def _golden3():
    byg = {}
    for ln in GOLDEN3.read_text().splitlines():
        if ln and not ln.startswith("#"):
            r = ln.split()
            byg.setdefault(int(r[0]), []).append(r)
    return byg


def test_three_loop_points_match_stored_oracle(ctx):
    """Every three-loop graph at the stored oracle points (tests/golden,
    written by make_three_loop.py from oracle/ alone): the GPU's points and
    log p to 1e-12, its accepted FP64 values (threshold 1e-12) to 1e-12, and
    its double-double values at every point to 1e-12 plus the long-double
    oracle's own rounding, 16 * 2^-64 * kappa, with kappa the condition
    number sum|monomials| / |f| of the integrand's program at that point.
    Points outside that are settled by the oracle in 34-digit mpmath."""
    from tests.test_programs import interpret, read_programs, _name
    from tests.test_gpu_parity import _arbitrate
    progs = read_programs(ROOT / "paper_1905_08007_b300" / "csrc" / "_gen" / "vm_n3.bin.z")
    gs = q.enumerate_graphs(3)
    ogs = o_enum(3)
    n_fp64 = n_dd = 0
    for gi, rs in sorted(_golden3().items()):
        d = ctx.load(gs[gi])
        z, f, lp, fl = [], [], [], []
        for r in rs:
            a, b, c_, e = d.dump_points(int(r[1]), 1, seed=0)
            z.append(a.cpu().numpy()[0]); f.append(b.item()); lp.append(c_.item()); fl.append(e.item())
        z, f, lp, fl = np.array(z), np.array(f), np.array(lp), np.array(fl)
        zo = np.array([[float(v) for v in r[3:12]] for r in rs])
        lpo = np.array([float(r[2]) for r in rs])
        fo = np.array([np.longdouble(r[12]) for r in rs])
        np.testing.assert_allclose(z, zo, rtol=1e-12, atol=0)
        np.testing.assert_allclose(lp, lpo, rtol=1e-12, atol=1e-12)
        fo64 = fo.astype(np.float64)
        ok = fl == 0
        rel = np.abs(f - fo64) / np.abs(fo64)
        if np.any(rel[ok] > 1e-12):
            _arbitrate(ogs[gi], zo[ok], f[ok], rel[ok], cap=2)
        n_fp64 += int(ok.sum())
        fdd = d.eval_points(torch.tensor(zo, device="cuda"), prec=1).cpu().numpy()
        # the mirror-reduced program set holds one of each mirror pair
        g = ogs[gi]
        name = _name(g) if _name(g) in progs else _name(g.mirror())
        zp = zo if _name(g) in progs else _mirror_z(g, zo)
        fp, W = interpret(progs[name], zp, np.longdouble)
        kappa = (W / np.abs(fp)).astype(np.float64)
        tol = 1e-12 + 16 * 2.0 ** -64 * kappa
        rdd = np.abs(fdd - fo64) / np.abs(fo64)
        bad = rdd > tol
        if np.any(bad):
            _arbitrate(ogs[gi], zo[bad], fdd[bad], np.full(int(bad.sum()), 1.0), cap=2)
        n_dd += len(rs)
    assert n_fp64 >= 100 and n_dd == 400
    print(f"three-loop points: {n_fp64} accepted FP64 values and {n_dd} double-double values at 1e-12")


def _mirror_z(g, z):
    """z of graph g re-indexed as the point of its mirror graph (electron line
    i -> 2n-1-i, photons re-matched)."""
    mg = g.mirror()
    m = 2 * g.n - 1
    zm = np.zeros_like(z)
    for i in range(2 * g.n):
        zm[:, 2 * g.n - 1 - i] = z[:, i]
    for a, (s, t) in enumerate(g.pairs):
        b = mg.pairs.index(tuple(sorted((m - s, m - t))))
        zm[:, 2 * g.n + b] = z[:, 2 * g.n + a]
    return zm


@pytest.mark.parametrize("gi", SUBSET)
@pytest.mark.parametrize("begin,count", [(0, 24), (10**9 - 8, 8)])
def test_three_loop_points_match_oracle(ctx, gi, begin, count):
    """Fresh points (not stored) on a subset of graphs: points and log p to
    1e-12; integrand values at every point within 1e-9 of the FP64 oracle
    where the GPU accepts FP64 (both sides round in FP64; the strict 1e-12
    comparison against long double is the stored-points test)."""
    g = q.enumerate_graphs(3)[gi]
    og = o_enum(3)[gi]
    d = ctx.load(g)
    z, f, lp, fl = d.dump_points(begin, count, seed=0)
    z, f, lp, fl = z.cpu().numpy(), f.cpu().numpy(), lp.cpu().numpy(), fl.cpu().numpy()
    N = og.n_lines
    deg = deg_table(og)
    u = uniforms(np.arange(begin, begin + count, dtype=np.uint64), g.stream_id, 0, 2 * (N - 1))
    x, lpo, _ = sample_points(u, deg, f_table(deg, N), N)
    np.testing.assert_allclose(z, x, rtol=1e-12)
    np.testing.assert_allclose(lp, lpo, rtol=1e-12, atol=1e-12)
    fo = Integrand(og)(z)
    ok = fl == 0
    assert np.all(np.abs(f[ok] - fo[ok]) <= 1e-9 * np.abs(fo[ok]))


def test_three_loop_batched_config(ctx):
    """1e9 samples over the three-loop set in the persistent launch: the 28
    mirror-reduced graphs with their bytecode programs (mirror weights), the
    path the bench runs; each graph's batch result equals its per-graph
    integration of the same counters."""
    c = q.Context(0, prefer_programs=True)
    gs = q.enumerate_graphs(3, reduced=True)
    ds = [c.load(g) for g in gs]
    res = c.integrate_batch(ds, 10**9, seed=0, policy="variance", rounds=4, chunk=1 << 14)
    assert sum(r.n for r in res) >= 10**9
    assert all(math.isfinite(r.value) and r.n > 0 for r in res)
    rate = sum(r.n for r in res) / res[0].seconds
    print(f"three-loop set (bytecode): {rate:.3e} samples/s, "
          f"flagged {sum(r.n_flagged for r in res) / sum(r.n for r in res):.4f}")
    for i in (0, 13):
        ref = ds[i].integrate(res[i].n, seed=0, begin=0)
        assert res[i].value == pytest.approx(ref.value, rel=1e-9, abs=1e-12)


def test_three_loop_compiled_batch(ctx):
    """The compiled three-loop integrands in the persistent launch (all 50
    graphs, 5e7 samples; their double-double versions spill registers, so
    the bench runs three loops on the bytecode path)."""
    c = q.Context(0)
    ds = [c.load(g) for g in q.enumerate_graphs(3)]
    res = c.integrate_batch(ds, 5 * 10**7, seed=0, policy="variance", rounds=2, chunk=1 << 18)
    assert sum(r.n for r in res) >= 5 * 10**7
    assert all(math.isfinite(r.value) and r.n > 0 for r in res)
    ref = ds[25].integrate(res[25].n, seed=0, begin=0)
    assert res[25].value == pytest.approx(ref.value, rel=1e-10)
