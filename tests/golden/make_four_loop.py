"""Writes four_loop_points.txt: oracle values of the four-loop integrands at
the points that Eq. (1)'s sampler draws from given Philox counters (seed 0,
stream id = the graph's index in the full enumeration) with the Deg table
Deg(s) = -omega(I-closure(s)), else 0.5, floored at 0.05 (deg_table with
omega_factor 1: the file was written before Deg took half of -omega; any
positive table serves parity, and the tests give the library the same one).
Calls only oracle/.

    python tests/golden/make_four_loop.py [--procs 6] [--graphs G ...] [--counters C ...]

With --graphs / --counters only those rows are computed and they replace
the rows of the same (graph, counter) in the existing file (the others are
kept).

Graphs: every mirror-reduced four-loop graph (269; Sec. 3 counts the
mirror-reduced set), each at the counters in COUNTERS.  The oracle needs a few
minutes per point, so rows are appended to four_loop_points.partial as they
finish and a rerun resumes from it; the complete set is then written sorted.
Columns: graph index, counter, log p, z[0..11], f in long double (20
significant digits).
"""
import argparse
import multiprocessing as mp
import sys
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

COUNTERS = [0, 1_000_000_007]
OUT = Path(__file__).with_name("four_loop_points.txt")
PARTIAL = Path(__file__).with_name("four_loop_points.partial")


def graphs():
    from oracle.graphs import enumerate_graphs, enumerate_reduced
    full = enumerate_graphs(4)
    index = {g.key(): i for i, g in enumerate(full)}
    return [index[g.key()] for g in enumerate_reduced(4)]


def row(job):
    gi, c = job
    from oracle.graphs import deg_table, enumerate_graphs
    from oracle.integrand import Integrand
    from oracle.pdf import f_table, sample_points
    from oracle.philox import uniforms
    g = enumerate_graphs(4)[gi]
    N = g.n_lines
    deg = deg_table(g, omega_factor=1.0)
    u = uniforms(np.array([c], dtype=np.uint64), gi, 0, 2 * (N - 1))
    x, lp, _ = sample_points(u, deg, f_table(deg, N), N)
    f = Integrand(g)(x, dtype=np.longdouble)
    zs = " ".join(repr(float(v)) for v in x[0])
    return f"{gi} {c} {float(lp[0])!r} {zs} {np.format_float_scientific(f[0], precision=19)}"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=6)
    ap.add_argument("--graphs", type=int, nargs="*", default=None)
    ap.add_argument("--counters", type=int, nargs="*", default=None)
    ap.add_argument("--merge-only", action="store_true",
                    help="write the rows finished so far (the .partial file) into the file and stop")
    a = ap.parse_args()
    gis = a.graphs if a.graphs else graphs()
    counters = a.counters if a.counters else COUNTERS
    keep = {}
    if (a.graphs or a.counters) and OUT.exists():
        for ln in OUT.read_text().splitlines():
            p = ln.split()
            if len(p) == 16 and not ln.startswith("#"):
                keep[(int(p[0]), int(p[1]))] = ln
    done = {}
    if PARTIAL.exists():
        for ln in PARTIAL.read_text().splitlines():
            p = ln.split()
            if len(p) == 16:
                done[(int(p[0]), int(p[1]))] = ln
    jobs = [] if a.merge_only else [(gi, c) for gi in gis for c in counters if (gi, c) not in done]
    ctx = mp.get_context("spawn")
    with ctx.Pool(a.procs) as pool, open(PARTIAL, "a") as fh:
        for ln in pool.imap_unordered(row, jobs):
            fh.write(ln + "\n")
            fh.flush()
            p = ln.split()
            done[(int(p[0]), int(p[1]))] = ln
    if a.merge_only and OUT.exists():
        for ln in OUT.read_text().splitlines():
            p = ln.split()
            if len(p) == 16 and not ln.startswith("#"):
                keep.setdefault((int(p[0]), int(p[1])), ln)
    keep.update(done)
    done = keep
    keys = sorted(done)
    with open(OUT, "w") as fh:
        fh.write("# four-loop integrand at Eq. (1) points (oracle, long double); written by make_four_loop.py\n")
        fh.write("# Deg table: -omega(I-closure) (oracle deg_table with omega_factor 1), c_div 0.5, d_min 0.05\n")
        fh.write("# graph counter logp z0..z11 f\n")
        for k in keys:
            fh.write(done[k] + "\n")
    PARTIAL.unlink()
    print(OUT, len(keys), "rows")


if __name__ == "__main__":
    main()
