"""Write three_loop_limit_scan.txt: the local exponent of every single-set
limit of every mirror-reduced three-loop graph, from the oracle alone.

Sec. 2: after the subtraction every graph's integrand has a finite integral
point by point in parameter space; a limit z_S -> eps z_S (S a proper subset
of the lines: ultraviolet limits where S shrinks, infrared limits where its
complement grows -- an I-closure's complement shrinking is the infrared
corner of Eq. (1)'s Deg rule -- and every mixed one) is integrable when
|f| eps^|S| -> 0.  The local exponent

    delta_S = log(|f(eps2)| eps2^|S| / (|f(eps1)| eps1^|S|)) / log(eps2 / eps1)

at eps1 = 1e-3, eps2 = 1e-5 is positive for an integrable limit (a
logarithmic divergence has delta 0).  Two base points per graph, drawn from
a fixed Dirichlet(1, ..., 1) generator (numpy seed 60 + graph index).

    python tests/golden/make_three_loop_scan.py [--jobs 8]

Runs the oracle in float64 over all 511 - 1 proper subsets of the 9 lines of
the 28 mirror-reduced graphs (about 57000 integrand evaluations, in batches
of 128 points to bound the memory of the vectorised oracle; an hour or so
on 8 cores).  Finished graphs are appended to three_loop_limit_scan.partial
and a rerun resumes from it.  Line format: graph index (full enumeration),
subset bitmask, delta at base point 0, delta at base point 1.
"""
from __future__ import annotations

import argparse
import math
import multiprocessing as mp
import sys
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
sys.path.insert(0, str(HERE.parents[1]))

EPS = (1e-3, 1e-5)
N = 9
BATCH = 128
PARTIAL = HERE / "three_loop_limit_scan.partial"


def reduced_indices():
    from oracle.graphs import enumerate_graphs
    gs = enumerate_graphs(3)
    out = []
    for i, g in enumerate(gs):
        m = g.mirror()
        if not (m.key() < g.key()):
            out.append(i)
    return out


def base_points(gi):
    return np.random.default_rng(60 + gi).dirichlet([1.0] * N, size=2)


def scan_graph(gi, masks=None):
    """[(mask, delta0, delta1)] for graph gi of the full three-loop list."""
    from oracle.graphs import enumerate_graphs
    from oracle.integrand import Integrand
    g = enumerate_graphs(3)[gi]
    f = Integrand(g)
    z0 = base_points(gi)
    masks = list(range(1, (1 << N) - 1)) if masks is None else list(masks)
    pts = []
    for m in masks:
        for e in EPS:
            z = z0.copy()
            for l in range(N):
                if m >> l & 1:
                    z[:, l] *= e
            pts.append(z)
    allz = np.concatenate(pts, axis=0)
    vals = np.concatenate([np.abs(f(allz[i:i + BATCH])) for i in range(0, len(allz), BATCH)])
    out = []
    k = 0
    for m in masks:
        s = bin(m).count("1")
        a = vals[k:k + 2] * EPS[0] ** s
        b = vals[k + 2:k + 4] * EPS[1] ** s
        k += 4
        d = np.log(b / a) / math.log(EPS[1] / EPS[0])
        out.append((m, float(d[0]), float(d[1])))
    return out


def _job(gi):
    return gi, scan_graph(gi)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=8)
    ap.add_argument("--out", default=str(HERE / "three_loop_limit_scan.txt"))
    a = ap.parse_args(argv)
    gis = reduced_indices()
    done = {}
    if PARTIAL.exists():
        for ln in PARTIAL.read_text().splitlines():
            gi, m, d0, d1 = ln.split()
            done.setdefault(int(gi), []).append(ln)
    todo = [g for g in gis if len(done.get(g, [])) != (1 << N) - 2]
    with mp.get_context("spawn").Pool(a.jobs) as pool:
        for gi, rows in pool.imap_unordered(_job, todo):
            text = "".join(f"{gi} {m} {d0:.6f} {d1:.6f}\n" for m, d0, d1 in rows)
            with open(PARTIAL, "a") as fh:
                fh.write(text)
            done[gi] = text.splitlines()
            print(f"graph {gi} done ({len(done)}/{len(gis)})", flush=True)
    lines = ["# local exponent delta of |f| eps^|S| under z_S -> eps z_S between eps = 1e-3 and 1e-5,",
             "# two base points per graph (Dirichlet(1,...,1), numpy seed 60 + graph index); written by",
             "# tests/golden/make_three_loop_scan.py from the oracle (float64)",
             "# graph_index subset_mask delta_point0 delta_point1"]
    for gi in gis:
        lines.extend(sorted(done[gi], key=lambda ln: int(ln.split()[1])))
    Path(a.out).write_text("\n".join(lines) + "\n")
    PARTIAL.unlink()
    print(f"wrote {a.out}: {len(gis)} graphs")


if __name__ == "__main__":
    main()
