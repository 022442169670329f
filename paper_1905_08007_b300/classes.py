"""Per-class totals of a graph set (Sec. 3, Table 1).

The paper splits the lepton-loop-free vertex graphs of an order into
gauge-invariant classes (k, m, n): k photons with ends on both sides of the
external photon vertex, m on one side and n on the other (m >= n), and gives
per class the value sum_j a_j, the number of graphs N_diag (a graph and its
mirror image counted once), sum_j |a_j| and max_j |a_j|.  For a
mirror-reduced set with mirror weights (2 for the representative of a pair,
1 for a self-mirror graph), a_j = weight_j x value_j is the contribution of
graph j with both orientations and the row's graph count is N_diag; for a
set that holds both orientations (weights 1) a_j is one orientation's value.
The class sigma adds the graphs' variances.  The class of a graph comes from
the library (qed_gauge_class).
"""
from __future__ import annotations

import math

from ._lib import gauge_class


def class_table(graphs, results, weights=None):
    """Rows {k, m, n, graphs, value, sigma, sum_abs, max_abs}, in decreasing
    order of the graph count, from per-graph results and weights."""
    weights = weights if weights is not None else [1.0] * len(graphs)
    acc = {}
    for g, r, w in zip(graphs, results, weights):
        a = w * r.value
        row = acc.setdefault(gauge_class(g), [0, 0.0, 0.0, 0.0, 0.0])
        row[0] += 1
        row[1] += a
        row[2] += w * w * r.variance
        row[3] += abs(a)
        row[4] = max(row[4], abs(a))
    out = [{"k": k, "m": m, "n": n, "graphs": c, "value": v, "sigma": math.sqrt(var), "sum_abs": sa,
            "max_abs": mx} for (k, m, n), (c, v, var, sa, mx) in acc.items()]
    out.sort(key=lambda r: (-r["graphs"], -r["k"]))
    return out
