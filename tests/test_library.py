"""Host-side checks of the native library that need no GPU: it loads, exports
every symbol include/qedmc.h declares, enumerates the same graphs as the
oracle, and fails loudly (QED_ECUDA) when no GPU is present."""
import re
from pathlib import Path

import pytest

import paper_1905_08007_b300 as q
from oracle.graphs import enumerate_graphs as oracle_enum

ROOT = Path(__file__).resolve().parents[1]


def _declared():
    txt = (ROOT / "include" / "qedmc.h").read_text()
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*\*?(qed_\w+)\s*\(", txt, re.M)))


def test_library_exports_every_declared_symbol():
    L = q.load_library()
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_enumeration_matches_oracle(n):
    a = [(g.pairs, g.e) for g in q.enumerate_graphs(n)]
    b = [(g.pairs, g.e) for g in oracle_enum(n)]
    assert a == b
    assert [g.stream_id for g in q.enumerate_graphs(n)] == list(range(len(a)))


def test_gauge_class_matches_oracle():
    for g, o in zip(q.enumerate_graphs(3), oracle_enum(3)):
        assert q.gauge_class(g) == o.gauge_class()


def test_invalid_graph_rejected_without_gpu():
    with pytest.raises(q.QedError):
        q.gauge_class(q.Graph(2, ((0, 1), (2, 3)), 3))   # external-leg self-energy is still a graph shape
    with pytest.raises(q.QedError):
        q.gauge_class(q.Graph(2, ((0, 1), (1, 3)), 2))   # vertex used twice


def test_context_fails_loudly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(q.QedError) as ei:
        q.Context(0)
    assert ei.value.code == -3
