"""Host logic of the per-class totals (Sec. 3, Table 1): the library's
gauge-invariant classes of the mirror-reduced five-loop set have Table 1's
N_diag counts, and the class rows add up to the set total."""
from pathlib import Path

import pytest

import paper_1905_08007_b300 as q

GOLD = Path(__file__).parent / "golden"


def _table1():
    rows = {}
    for ln in (GOLD / "table1_ndiag.txt").read_text().splitlines():
        if ln.startswith("#") or not ln.strip():
            continue
        k, m, n, c = (int(x) for x in ln.split())
        rows[(k, m, n)] = c
    return rows


def _fake(values):
    return [q.Result(v, 0.01 * (i + 1), (v, 0.0), (v * v, 0.0), 100, 0, 0, 0.0) for i, v in enumerate(values)]


def test_five_loop_classes_have_table1_counts():
    gs = q.enumerate_graphs(5, reduced=True)
    assert len(gs) == 3213
    rows = q.class_table(gs, _fake([1.0] * len(gs)))
    assert {(r["k"], r["m"], r["n"]): r["graphs"] for r in rows} == _table1()


def test_class_rows_add_up():
    gs = q.enumerate_graphs(4, reduced=True)
    vals = [((-1) ** i) * (0.1 + i % 7) for i in range(len(gs))]
    w = [2.0 if i % 3 else 1.0 for i in range(len(gs))]
    res = _fake(vals)
    rows = q.class_table(gs, res, w)
    assert sum(r["graphs"] for r in rows) == len(gs)
    assert sum(r["value"] for r in rows) == pytest.approx(sum(a * b for a, b in zip(w, vals)))
    assert sum(r["sum_abs"] for r in rows) == pytest.approx(sum(abs(a * b) for a, b in zip(w, vals)))
    assert max(r["max_abs"] for r in rows) == pytest.approx(max(abs(a * b) for a, b in zip(w, vals)))
    var = sum(r["sigma"] ** 2 for r in rows)
    assert var == pytest.approx(sum(a * a * r.variance for a, r in zip(w, res)))
