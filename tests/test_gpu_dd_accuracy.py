"""Accuracy of the double-double re-evaluation against the arbitrary-precision
oracle (mpmath, 34 digits) on the points the FP64 path flags, on the two
self-energy graphs (where the forest terms cancel most), for the compiled
integrands and for the bytecode programs in the interpreter kernels (whose
double-double multiply-add has one two-sum).  Prints the maximum and median
relative error of the double-double values and of the FP64 values on the
same points."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1905_08007_b300 as q                      # noqa: E402
from oracle.graphs import enumerate_graphs as o_enum    # noqa: E402
from oracle.integrand import Integrand                  # noqa: E402


@pytest.mark.parametrize("programs", [False, True], ids=["compiled", "bytecode"])
@pytest.mark.parametrize("gi", [3, 5])
def test_flagged_points_double_double_vs_mpmath(gi, programs):
    import mpmath
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    ctx = q.Context(0, threshold=1e-12, prefer_programs=programs)
    g = q.enumerate_graphs(2)[gi]
    og = o_enum(2)[gi]
    d = ctx.load(g)
    if programs and d.integrand_id == q.Context(0).load(g).integrand_id:
        pytest.skip("programs exist for one graph of each mirror pair; this one is the other")
    z, f, lp, fl = d.dump_points(0, 4000, seed=17)
    flagged = np.nonzero(fl.cpu().numpy() & 1)[0][:6]
    assert flagged.size >= 6
    zf = z[flagged]
    fdd = d.eval_points(zf, prec=1).cpu().numpy()
    f64 = f.cpu().numpy()[flagged]
    with mpmath.workdps(34):
        zo = np.array([[mpmath.mpf(float(v)) for v in row] for row in zf.cpu().numpy()], dtype=object)
        ref = Integrand(og)(zo, dtype=object)
        e_dd = np.array([float(abs(mpmath.mpf(float(a)) - b) / abs(b)) for a, b in zip(fdd, ref)])
        e_64 = np.array([float(abs(mpmath.mpf(float(a)) - b) / abs(b)) for a, b in zip(f64, ref)])
    print(f"graph {og.pairs} e={og.e} ({'bytecode' if programs else 'compiled'}): {flagged.size} flagged points; double-double rel. error "
          f"max {e_dd.max():.2e} median {np.median(e_dd):.2e}; FP64 max {e_64.max():.2e} "
          f"median {np.median(e_64):.2e}")
    assert e_dd.max() < 1e-12
