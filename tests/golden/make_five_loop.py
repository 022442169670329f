"""Writes five_loop_points.txt: oracle values of five-loop integrands (15
lines) at the points that Eq. (1)'s sampler draws from given Philox counters
(seed 0, stream id = the graph's index in the full enumeration, the Deg
rule's table).  Calls only oracle/.

    python tests/golden/make_five_loop.py [--procs 4] [--graphs G ...] [--counters C ...]

Graphs: by default five graphs of the 64-graph five-loop workload
(five_loop_subset.txt) whose programs take the generator a few minutes, at
the counters in COUNTERS; the oracle needs about four minutes per
five-loop point in float64 (an hour or more in long double), so the values
are float64.  Rows are appended to five_loop_points.partial as they finish
and a rerun resumes from it; with
--graphs / --counters the new rows replace the rows of the same (graph,
counter) in the existing file.  Columns: graph index, counter, log p,
z[0..14], f in float64 (17 significant digits).
"""
import argparse
import multiprocessing as mp
import sys
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

COUNTERS = [0, 1_000_000_007]
OUT = Path(__file__).with_name("five_loop_points.txt")
PARTIAL = Path(__file__).with_name("five_loop_points.partial")


def graphs():
    return [91, 158, 203, 1518, 1610]


def row(job):
    gi, c = job
    from oracle.graphs import deg_table, enumerate_graphs
    from oracle.integrand import Integrand
    from oracle.pdf import f_table, sample_points
    from oracle.philox import uniforms
    g = enumerate_graphs(5)[gi]
    N = g.n_lines
    deg = deg_table(g)
    u = uniforms(np.array([c], dtype=np.uint64), gi, 0, 2 * (N - 1))
    x, lp, _ = sample_points(u, deg, f_table(deg, N), N)
    # float64: a long-double five-loop point takes the oracle an hour or more
    f = Integrand(g)(x, dtype=np.float64)
    zs = " ".join(repr(float(v)) for v in x[0])
    return f"{gi} {c} {float(lp[0])!r} {zs} {np.format_float_scientific(f[0], precision=19)}"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=4)
    ap.add_argument("--graphs", type=int, nargs="*", default=None)
    ap.add_argument("--counters", type=int, nargs="*", default=None)
    a = ap.parse_args()
    gis = a.graphs if a.graphs else graphs()
    counters = a.counters if a.counters else COUNTERS
    keep = {}
    if (a.graphs or a.counters) and OUT.exists():
        for ln in OUT.read_text().splitlines():
            p = ln.split()
            if len(p) == 19 and not ln.startswith("#"):
                keep[(int(p[0]), int(p[1]))] = ln
    done = {}
    if PARTIAL.exists():
        for ln in PARTIAL.read_text().splitlines():
            p = ln.split()
            if len(p) == 19:
                done[(int(p[0]), int(p[1]))] = ln
    jobs = [(gi, c) for gi in gis for c in counters if (gi, c) not in done]
    ctx = mp.get_context("spawn")
    with ctx.Pool(a.procs) as pool, open(PARTIAL, "a") as fh:
        for ln in pool.imap_unordered(row, jobs):
            fh.write(ln + "\n")
            fh.flush()
            p = ln.split()
            done[(int(p[0]), int(p[1]))] = ln
    keep.update(done)
    done = keep
    keys = sorted(done)
    with open(OUT, "w") as fh:
        fh.write("# five-loop integrand at Eq. (1) points (oracle, float64); written by make_five_loop.py\n")
        fh.write("# Deg table: the Deg rule (oracle deg_table), c_div 0.5, d_min 0.05; f in float64\n")
        fh.write("# graph counter logp z0..z14 f\n")
        for k in keys:
            fh.write(done[k] + "\n")
    PARTIAL.unlink()
    print(OUT, len(keys), "rows")


if __name__ == "__main__":
    main()
