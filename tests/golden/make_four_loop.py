"""Writes four_loop_points.txt: oracle values of four-loop integrands at the
points that Eq. (1)'s sampler draws from given Philox counters (seed 0,
stream id = the graph's index in the full enumeration).  Calls only oracle/.

    python tests/golden/make_four_loop.py

Graphs: one per forest-structure size in the mirror-reduced four-loop set
(1, 3, 8, 16 and 46 forest terms).  Columns: graph index, counter, log p,
z[0..11], f in long double (20 significant digits).
"""
import multiprocessing as mp
import sys
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

GRAPHS = [85, 113, 23, 442, 514]
COUNTERS = [0, 1, 2, 3, 4, 5, 1_000_000_007]


def rows(gi):
    from oracle.graphs import deg_table, enumerate_graphs
    from oracle.integrand import Integrand
    from oracle.pdf import f_table, sample_points
    from oracle.philox import uniforms
    g = enumerate_graphs(4)[gi]
    N = g.n_lines
    deg = deg_table(g)
    u = uniforms(np.array(COUNTERS, dtype=np.uint64), gi, 0, 2 * (N - 1))
    x, lp, _ = sample_points(u, deg, f_table(deg, N), N)
    f = Integrand(g)(x, dtype=np.longdouble)
    out = []
    for k, c in enumerate(COUNTERS):
        zs = " ".join(repr(float(v)) for v in x[k])
        out.append(f"{gi} {c} {float(lp[k])!r} {zs} {np.format_float_scientific(f[k], precision=19)}")
    return out


if __name__ == "__main__":
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(GRAPHS)) as pool:
        res = pool.map(rows, GRAPHS)
    path = Path(__file__).with_name("four_loop_points.txt")
    with open(path, "w") as fh:
        fh.write("# four-loop integrand at Eq. (1) points (oracle, long double); written by make_four_loop.py\n")
        fh.write("# graph counter logp z0..z11 f\n")
        for r in res:
            fh.write("\n".join(r) + "\n")
    print(path)
