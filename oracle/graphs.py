"""Diagram set, subgraphs and Deg -- oracle side (test infrastructure only).

Sec. 3 of the paper counts the 5-loop vertex graphs without lepton loops
(3213 integrands, Table 1 per class, mirror pairs counted once).  A graph is an
open electron line carrying 2n photon vertices plus the external-photon
vertex X; the n internal photons pair the 2n photon vertices.

Conventions (shared only by definition with the CUDA side, no code shared):

* photon vertices are numbered 0..2n-1 along the electron flow; X sits after
  the first ``e`` of them (1 <= e <= 2n-1);
* the 2n+1 vertices in line order are "positions" 0..2n, X at position e;
  photon vertex v sits at position v if v < e, else v+1;
* electron line i (0..2n-1) joins positions i and i+1;
* photon a (0..n-1, ordered by first endpoint) joins photon vertices
  (s_a, t_a), s_a < t_a;
* line index for the PDF / Feynman parameters: electron lines 0..2n-1 first,
  then photon lines 2n..3n-1.
"""
from __future__ import annotations

from dataclasses import dataclass
from functools import lru_cache
from itertools import combinations


def perfect_matchings(vs):
    """All perfect matchings of the tuple ``vs`` as tuples of sorted pairs."""
    if not vs:
        yield ()
        return
    a = vs[0]
    for i in range(1, len(vs)):
        b = vs[i]
        rest = vs[1:i] + vs[i + 1:]
        for m in perfect_matchings(rest):
            yield ((a, b),) + m


@dataclass(frozen=True)
class Graph:
    n: int                      # loop order = number of internal photons
    pairs: tuple                # ((s_0,t_0),...,(s_{n-1},t_{n-1})) sorted by s
    e: int                      # external vertex after e photon vertices

    # ---- geometry -------------------------------------------------------
    @property
    def n_lines(self) -> int:
        return 3 * self.n

    @property
    def n_elec(self) -> int:
        return 2 * self.n

    def pos(self, v: int) -> int:
        """Position (0..2n) on the electron line of photon vertex v."""
        return v if v < self.e else v + 1

    def photon_positions(self, a: int):
        s, t = self.pairs[a]
        return self.pos(s), self.pos(t)

    def line_ends(self, l: int):
        """Endpoints (as positions) of PDF line l."""
        if l < self.n_elec:
            return (l, l + 1)
        return self.photon_positions(l - self.n_elec)

    def span(self, a: int):
        """Electron lines carrying photon a's loop momentum."""
        ps, pt = self.photon_positions(a)
        return tuple(range(ps, pt))

    # ---- labels -----------------------------------------------------------
    def mirror(self) -> "Graph":
        """Reverse the electron line (Sec. 3 footnote: equal contribution)."""
        m = 2 * self.n - 1
        pr = tuple(sorted(tuple(sorted((m - s, m - t))) for s, t in self.pairs))
        return Graph(self.n, pr, 2 * self.n - self.e)

    def key(self):
        return (self.pairs, self.e)

    def is_self_mirror(self) -> bool:
        return self.mirror().key() == self.key()

    def canonical(self) -> "Graph":
        mg = self.mirror()
        return self if self.key() <= mg.key() else mg

    def gauge_class(self):
        """(k, m, n): photons spanning X, left of X, right of X, with m >= n
        after mirroring (Sec. 3, Table 1)."""
        k = left = right = 0
        for s, t in self.pairs:
            if t < self.e:
                left += 1
            elif s >= self.e:
                right += 1
            else:
                k += 1
        return (k, max(left, right), min(left, right))


def _closed(pairs, vset):
    for s, t in pairs:
        if (s in vset) != (t in vset):
            return False
    return True


def admissible(n: int, pairs, e: int) -> bool:
    """No self-energy insertion on an external leg and one-particle
    irreducible: no prefix {0..k-1} with k <= e and no suffix {k..2n-1} with
    k >= e may be closed under the photon pairing."""
    for k in range(1, e + 1):
        if _closed(pairs, set(range(k))):
            return False
    for k in range(e, 2 * n):
        if _closed(pairs, set(range(k, 2 * n))):
            return False
    return True


@lru_cache(maxsize=None)
def enumerate_graphs(n: int):
    """All lepton-loop-free vertex graphs of order n (both orientations)."""
    out = []
    for m in perfect_matchings(tuple(range(2 * n))):
        pairs = tuple(sorted(m))
        for e in range(1, 2 * n):
            if admissible(n, pairs, e):
                out.append(Graph(n, pairs, e))
    return tuple(out)


@lru_cache(maxsize=None)
def enumerate_reduced(n: int):
    """Mirror-reduced set: one representative (lexicographically smaller key)
    per mirror pair; self-mirror graphs appear once."""
    seen = {}
    for g in enumerate_graphs(n):
        c = g.canonical()
        seen.setdefault(c.key(), c)
    return tuple(sorted(seen.values(), key=lambda g: g.key()))


# ---------------------------------------------------------------------------
# UV degree, I-closure, Deg (Sec. 2, Eq. (1) and the text after it)
# ---------------------------------------------------------------------------

def omega(g: Graph, s) -> int:
    """UV degree of divergence of the line set s (Feynman gauge, d=4):
    4 L(s) - 2 #photons(s) - #electrons(s), where L(s) is the cycle rank of
    the subgraph formed by the lines of s and their end vertices."""
    s = list(s)
    if not s:
        return 0
    parent = {}

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for l in s:
        for v in g.line_ends(l):
            parent.setdefault(v, v)
    comps = len(parent)
    for l in s:
        a, b = g.line_ends(l)
        ra, rb = find(a), find(b)
        if ra != rb:
            parent[ra] = rb
            comps -= 1
    loops = len(s) - len(parent) + comps
    n_ph = sum(1 for l in s if l >= g.n_elec)
    n_el = len(s) - n_ph
    return 4 * loops - 2 * n_ph - n_el


def i_closure(g: Graph, s) -> frozenset:
    """s together with every photon whose connecting electron path lies in s
    (Sec. 2, definition of the I-closure)."""
    s = set(s)
    out = set(s)
    for a in range(g.n):
        if set(g.span(a)) <= s:
            out.add(g.n_elec + a)
    return frozenset(out)


def deg_default(g: Graph, s, c_div: float = 0.5, d_min: float = 0.05, omega_factor: float = 0.5) -> float:
    """Deg(s) reading: half of -omega of the I-closure when that is positive,
    else the constant c_div for sets whose closure is UV divergent, floored
    at d_min.  omega counts powers of momentum; in the Feynman parameters of
    s the integrand scales with half that power (a parameter goes like the
    inverse square of its line's momentum), which is the exponent the bound
    of Eq. (1) needs, and it makes Deg fractional (1/2 for one electron
    line), as the text after Eq. (1) says Deg can be.  Parity unpinned as to
    the value: any positive Deg gives an unbiased estimator.  omega_factor
    = 1 gives the earlier reading Deg = -omega (too steep by two, kept to
    reproduce points stored with it)."""
    w = -omega(g, i_closure(g, s))
    d = omega_factor * float(w) if w > 0 else c_div
    return max(d, d_min)


def deg_table(g: Graph, c_div: float = 0.5, d_min: float = 0.05, omega_factor: float = 0.5):
    """Deg over all subsets of lines as a list indexed by bitmask; entries
    for the empty and the full set are unused and set to 0."""
    N = g.n_lines
    full = (1 << N) - 1
    tab = [0.0] * (1 << N)
    for mask in range(1, full):
        s = [l for l in range(N) if mask >> l & 1]
        tab[mask] = deg_default(g, s, c_div, d_min, omega_factor)
    return tab


# ---------------------------------------------------------------------------
# UV-divergent subgraphs and forests (Sec. 2: linear operators on the
# amplitudes of UV-divergent subdiagrams)
# ---------------------------------------------------------------------------

@dataclass(frozen=True)
class Subgraph:
    a: int            # first electron line of the segment
    b: int            # last electron line of the segment (inclusive)
    photons: tuple    # internal photons
    kind: str         # "SE" (omega=1) or "V" (omega=0)
    has_x: bool       # contains the external vertex (I-set)

    def lines(self, g: Graph) -> frozenset:
        return frozenset(range(self.a, self.b + 1)) | frozenset(
            g.n_elec + p for p in self.photons)


def divergent_subgraphs(g: Graph):
    """Proper 1PI subgraphs with omega >= 0.  Without lepton loops each is a
    contiguous electron segment with the photons internal to it; SE-like
    ones have no photon leg (omega = 1), vertex-like ones exactly one (the
    external photon or an internal photon of g; omega = 0)."""
    out = []
    for a in range(g.n_elec):
        for b in range(a, g.n_elec):
            if a == 0 and b == g.n_elec - 1:
                continue
            pos = set(range(a, b + 2))
            inside = [i for i in range(g.n) if set(g.photon_positions(i)) <= pos]
            legs = 0
            for p in pos:
                if p == g.e:
                    legs += 1
                    continue
                v = p if p < g.e else p - 1
                partner = [t if s == v else s for s, t in g.pairs if v in (s, t)][0]
                if g.pos(partner) not in pos:
                    legs += 1
            if legs > 1:
                continue
            spanned = set()
            for i in inside:
                spanned |= set(g.span(i))
            if not set(range(a, b + 1)) <= spanned:
                continue          # an internal bridge: not 1PI
            kind = "SE" if legs == 0 else "V"
            out.append(Subgraph(a, b, tuple(inside), kind, g.e in pos and kind == "V"))
    return tuple(out)


def is_forest(g: Graph, subs) -> bool:
    ls = [s.lines(g) for s in subs]
    for x, y in combinations(ls, 2):
        if not (x <= y or y <= x or not (x & y)):
            return False
    return True


def forests(g: Graph):
    """All forests (sets of pairwise nested-or-disjoint divergent
    subgraphs), the empty forest included."""
    subs = divergent_subgraphs(g)
    out = []
    for r in range(len(subs) + 1):
        for c in combinations(subs, r):
            if is_forest(g, c):
                out.append(c)
    return out
