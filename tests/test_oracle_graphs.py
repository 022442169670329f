"""Oracle pins: the graph set against Sec. 3 / Table 1 and brute force."""
from collections import Counter
from itertools import combinations
from pathlib import Path

import pytest

from oracle.graphs import (divergent_subgraphs, enumerate_graphs, enumerate_reduced, forests,
                           i_closure, omega, deg_table)

GOLD = Path(__file__).parent / "golden"


def test_counts_all_orders():
    assert [len(enumerate_graphs(n)) for n in range(1, 6)] == [1, 6, 50, 518, 6354]
    # Sec. 3: "3213 integrands" at 5 loops, mirror pairs counted once
    assert [len(enumerate_reduced(n)) for n in range(1, 6)] == [1, 4, 28, 269, 3213]


def test_table1_class_counts():
    want = {}
    for line in (GOLD / "table1_ndiag.txt").read_text().splitlines():
        if line.startswith("#") or not line.strip():
            continue
        k, m, n, c = map(int, line.split())
        want[(k, m, n)] = c
    got = Counter(g.gauge_class() for g in enumerate_reduced(5))
    assert dict(got) == want
    assert sum(want.values()) == 3213


def test_mirror_is_involution_and_preserves_class():
    for g in enumerate_graphs(3):
        m = g.mirror()
        assert m.mirror().key() == g.key()
        assert m.gauge_class() == g.gauge_class()
        assert m.key() in {h.key() for h in enumerate_graphs(3)}


def _is_1pi_connected(g, lines):
    """Brute force: connected and no line whose removal disconnects it."""
    def comps(ls):
        parent = {}

        def f(x):
            while parent[x] != x:
                x = parent[x]
            return x
        for l in ls:
            for v in g.line_ends(l):
                parent.setdefault(v, v)
        for l in ls:
            a, b = (f(v) for v in g.line_ends(l))
            if a != b:
                parent[a] = b
        return len({f(v) for v in parent}), set(parent)
    c, verts = comps(lines)
    if c != 1:
        return False
    for l in lines:
        rest = [x for x in lines if x != l]
        if not rest:
            return False
        c2, v2 = comps(rest)
        if c2 != 1 or v2 != verts:
            return False
    return True


@pytest.mark.parametrize("n", [1, 2, 3])
def test_divergent_subgraphs_brute_force(n):
    """The proper one-particle-irreducible connected line sets with
    omega >= 0, found by brute force over all subsets, are exactly the
    segment construction (self-energy and vertex-like subgraphs)."""
    for g in enumerate_graphs(n):
        N = g.n_lines
        full = frozenset(range(N))
        want = set()
        for r in range(2, N):
            for s in combinations(range(N), r):
                s = frozenset(s)
                if omega(g, s) < 0 or not _is_1pi_connected(g, s):
                    continue
                want.add(s)
        got = {s.lines(g) for s in divergent_subgraphs(g)}
        assert got == want
        for s in divergent_subgraphs(g):
            assert omega(g, s.lines(g)) == (1 if s.kind == "SE" else 0)


def test_omega_special_cases():
    g = enumerate_graphs(1)[0]
    # one electron line: -1; the photon: -2; the whole one-loop vertex: 0
    assert omega(g, [0]) == -1
    assert omega(g, [2]) == -2
    assert omega(g, [0, 1, 2]) == 0
    # I-closure of the two electron lines adds the photon
    assert i_closure(g, [0, 1]) == frozenset({0, 1, 2})


def test_deg_positive():
    for g in enumerate_graphs(2):
        d = deg_table(g)
        assert all(x > 0 for x in d[1:-1])


def test_forests_are_nested_or_disjoint():
    for g in enumerate_graphs(3):
        for F in forests(g):
            ls = [s.lines(g) for s in F]
            for a, b in combinations(ls, 2):
                assert a <= b or b <= a or not (a & b)
