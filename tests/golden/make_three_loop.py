"""Writes three_loop_points.txt: oracle values of every three-loop integrand
(all 50 graphs) at the points that Eq. (1)'s sampler draws from given Philox
counters (seed 0, stream id = the graph's index, default Deg table).  Calls
only oracle/.

    python tests/golden/make_three_loop.py [--procs 6]

Columns: graph index, counter, log p, z[0..8], f in long double (20
significant digits).
"""
import argparse
import multiprocessing as mp
import sys
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

COUNTERS = [0, 1, 2, 3, 4, 5, 999_999, 10**9 - 1]
OUT = Path(__file__).with_name("three_loop_points.txt")


def rows(gi):
    from oracle.graphs import deg_table, enumerate_graphs
    from oracle.integrand import Integrand
    from oracle.pdf import f_table, sample_points
    from oracle.philox import uniforms
    g = enumerate_graphs(3)[gi]
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=6)
    a = ap.parse_args()
    ctx = mp.get_context("spawn")
    with ctx.Pool(a.procs) as pool:
        res = pool.map(rows, range(50), chunksize=1)
    with open(OUT, "w") as fh:
        fh.write("# three-loop integrand at Eq. (1) points (oracle, long double); written by make_three_loop.py\n")
        fh.write("# graph counter logp z0..z8 f\n")
        for r in res:
            fh.write("\n".join(r) + "\n")
    print(OUT)


if __name__ == "__main__":
    main()
