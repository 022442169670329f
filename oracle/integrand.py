"""Per-diagram subtracted AMM integrand -- oracle side (test infrastructure).

What is computed (Sec. 2 items 1-4).  The paper does not print the operator
definitions (it defers them to its references); the reading below is this
project's own: Feynman gauge and m = 1, the F2(0) projection of item 1, the
four operators U, L, A of item 2 with their kinematics, and the combination
rule of item 3.

1. Unsubtracted integrand M_G(z).  Feynman gauge, m = 1, alpha/pi units.  For
   an n-loop vertex graph with 3n lines, after Feynman parametrisation and the
   loop integrations,

     M_G = (-1)^n 4^-n sum_{k<n} (-1)^k Gamma(n-k) U^-2 V^(k-n) (2U)^-k
           sum_{k contractions} prod B_ij  F2[ Dirac string ],

   where each electron line contributes (Q_l-slash + 1) or, when contracted
   with another line, gamma^rho ... gamma_rho; photons contract their two
   vertices; F2 is the q -> 0 magnetic projection of ``dirac``.

2. Forest terms.  Each UV-divergent subgraph S in a forest is replaced by an
   operator value, computed as a "block": the lines of S keep their own loop
   momenta but no longer carry the momenta of the enclosing loops, and see a
   fixed external momentum:
     U (vertex-like S)  : Gamma_mu(0, 0) = c gamma_mu            (kin "0")
     U (self-energy S)  : Sigma -> dm_os + (k-slash - m) b(0)     (kins "p"
                          and "k": on-shell mass part, zero-momentum slope)
     L (vertex-like)    : on-shell forward vertex constant         (kin "p")
     A (vertex-like, X) : F2(0) of S                               (kin "q")
   A block's scalar multiplies the enclosing string, in which S appears as one
   vertex (vertex-like S) or as the identity / the factor (k-slash - m)
   (self-energy S).  All blocks of one term share the Feynman parameters of
   G; their loop momenta decouple, so Lambda is block diagonal and the single
   Gamma(n-k) V^(k-n) factor with V = sum of the blocks' V reproduces the
   product of the blocks' separate integrals.

3. Combination (forest-like formula):
     A~_G = sum_F (-1)^|F| [ T(F; G) + sum_{G' in F, X in G'} T(F; G') ],
   T(F; G'): G' gets A, the root G gets (L - U) when G' != G, every element
   of F strictly containing G' gets L, every other element of F gets U.
   (An element S with G' < S < G is both a link of the infrared chain,
   (L - U), and the ultraviolet counterterm, U, of the block that encloses
   it; the two add to L.  With (L - U) alone the block G/G' keeps the
   logarithmic divergence of its subgraph S/G' -- the shell limit of the
   three-loop rainbow graph, pinned by a test.)

Parity unpinned as to the operator reading itself except through the tests
that tie it to A_1^(2) = 1/2, the two-loop closed form, the UV/IR finiteness
scans and mirror symmetry.
"""
from __future__ import annotations

import math
import string as _string
from dataclasses import dataclass, field
from itertools import product as _iproduct

import numpy as np

from . import dirac
from .graphs import Graph, Subgraph, forests
from .polys import polynomials, b_matrix

GAMMA_STACK = np.array(dirac.GAMMA)                     # [mu, 4, 4]
GAMMA_SPATIAL_NEG = -np.array(dirac.GAMMA[1:])          # -gamma^j, j=1..3
GAMMA_LOWER = np.array([dirac.METRIC[m] * dirac.GAMMA[m] for m in range(4)])  # gamma_nu


# ---------------------------------------------------------------------------
# term description
# ---------------------------------------------------------------------------

@dataclass
class Block:
    a: int                 # first electron line of the segment
    b: int                 # last electron line
    kind: str              # "root", "V", "SE"
    kin: str               # "q", "p", "0", "k"
    proj: str              # "F2", "L", "UV", "SEmass", "SEwf"
    photons: tuple = ()
    children: list = field(default_factory=list)
    parent: "Block" = None

    def contains_pos(self, v):
        return self.a <= v <= self.b + 1

    def contains_line(self, l):
        return self.a <= l <= self.b


def build_blocks(g: Graph, root_kin, root_proj, subs):
    """subs: list of (Subgraph, kin, proj).  Returns (root, all blocks)."""
    root = Block(0, g.n_elec - 1, "root", root_kin, root_proj, tuple(range(g.n)))
    blocks = [root]
    for s, kin, proj in subs:
        blocks.append(Block(s.a, s.b, s.kind, kin, proj, s.photons))
    # parent = smallest strictly containing block
    for bl in blocks[1:]:
        best = root
        for other in blocks[1:]:
            if other is bl:
                continue
            if other.a <= bl.a and bl.b <= other.b and (other.b - other.a) > (bl.b - bl.a):
                if (other.b - other.a) < (best.b - best.a):
                    best = other
        bl.parent = best
        best.children.append(bl)
    for bl in blocks:
        bl.children.sort(key=lambda c: c.a)
    return root, blocks


def _min_block_line(blocks, l):
    best = blocks[0]
    for bl in blocks:
        if bl.contains_line(l) and (bl.b - bl.a) < (best.b - best.a):
            best = bl
    return best


def _min_block_photon(g, blocks, a):
    ps, pt = g.photon_positions(a)
    best = blocks[0]
    for bl in blocks:
        if bl.contains_pos(ps) and bl.contains_pos(pt) and (bl.b - bl.a) < (best.b - best.a):
            best = bl
    return best


# ---------------------------------------------------------------------------
# Dirac chains via einsum
# ---------------------------------------------------------------------------

_LET = _string.ascii_letters
_PAIR_LABELS = "abdefghiklmnopqtuvwxyABCDEFGHIKLOPQRSTUVWXY"


def _chain(items, pairs, out_free, Bn=1, ctype=complex):
    """Product items[-1] ... items[0] of 4x4 factors, built right to left.

    items: list of (array, has_batch, free) where array is [B,4,4] (batch),
    [4,4], or [F,4,4] / [B,F,4,4] carrying the named free index ``free``;
    array None marks a gamma slot contracted with its partner in ``pairs``
    (a Feynman-gauge photon or a contracted loop-momentum pair: sum over
    alpha of gamma^alpha ... gamma_alpha).
    Returns array [B, *out_free, 4, 4].
    """
    partner = {}
    for (i, j) in pairs:
        partner[i] = j
        partner[j] = i
    # R dims: [B, open axes..., 4, 4]; open axes are free indices or the
    # alpha of a pair whose second gamma is still to come.
    R = np.broadcast_to(np.eye(4, dtype=ctype), (Bn, 4, 4)).copy()
    names = []

    def lmul(M, R, nb):
        # M: [B?, F?, 4, 4] with nb = number of leading batch dims of M (0/1)
        if nb:
            M = M.reshape((M.shape[0],) + (1,) * len(names) + M.shape[1:])
        return np.matmul(M, R) if M.ndim == R.ndim else np.matmul(M, R[..., None, :, :])

    for t, (arr, has_batch, free) in enumerate(items):
        if arr is None:
            j = partner[t]
            lab = _PAIR_LABELS[min(t, j)]
            if j > t:      # open the pair: gamma^alpha, alpha as a new axis
                R = np.matmul(GAMMA_STACK, R[..., None, :, :])
                names.append(lab)
                continue
            k = names.index(lab)
            Rk = np.moveaxis(R, 1 + k, -3)            # [..., alpha, 4, 4]
            R = np.matmul(GAMMA_LOWER, Rk).sum(axis=-3)
            names.pop(k)
            continue
        if free is None:
            if has_batch:
                R = np.matmul(arr.reshape((arr.shape[0],) + (1,) * len(names) + (4, 4)), R)
            else:
                R = np.matmul(arr, R)
        else:
            if has_batch:
                A = arr.reshape((arr.shape[0],) + (1,) * len(names) + arr.shape[1:])
            else:
                A = arr
            R = np.matmul(A, R[..., None, :, :])
            names.append(free)
    assert sorted(names) == sorted(out_free), (names, out_free)
    perm = [0] + [1 + names.index(f) for f in out_free] + [1 + len(names), 2 + len(names)]
    return np.transpose(R, perm)


def _pairings(idx):
    """All sets of disjoint pairs of the list idx (including the empty set)."""
    if len(idx) < 2:
        yield ()
        return
    first, rest = idx[0], idx[1:]
    for p in _pairings(rest):
        yield p
    for i in range(len(rest)):
        for p in _pairings(rest[:i] + rest[i + 1:]):
            yield ((first, rest[i]),) + p


class TermEvaluator:
    """Evaluates one forest term of one graph at a batch of points."""

    def __init__(self, g: Graph, root_kin, root_proj, subs):
        self.g = g
        self.root, self.blocks = build_blocks(g, root_kin, root_proj, subs)
        n = g.n
        L = g.n_lines
        self.mb_line = [_min_block_line(self.blocks, l) for l in range(g.n_elec)]
        self.mb_ph = [_min_block_photon(g, self.blocks, a) for a in range(n)]
        eta = np.zeros((L, n))
        for a in range(n):
            for l in g.span(a):
                if self.mb_line[l] is self.mb_ph[a]:
                    eta[l, a] = 1.0
            eta[g.n_elec + a, a] = 1.0
        alpha = np.zeros(L)
        beta = np.zeros(L)
        kappa = np.zeros(L)
        for l in range(g.n_elec):
            kin = self.mb_line[l].kin
            after_x = 1.0 if l >= g.e else 0.0
            if kin == "q":
                alpha[l], beta[l] = 1.0, after_x - 0.5
            elif kin == "p":
                alpha[l] = 1.0
            elif kin == "k":
                kappa[l] = 1.0
        mass2 = np.array([1.0] * g.n_elec + [0.0] * n)
        self.eta, self.alpha, self.beta, self.kappa, self.mass2 = eta, alpha, beta, kappa, mass2

    # ---- label of a vertex position inside block bl -------------------
    def _vertex_label(self, bl, v):
        g = self.g
        if v == g.e:
            return "mu"
        pv = v if v < g.e else v - 1
        a = [i for i, (s, t) in enumerate(g.pairs) if pv in (s, t)][0]
        if self.mb_ph[a] is bl:
            return ("ph", a)
        return "mu"

    def _leg_label(self, parent, child):
        """Label the child's replacement vertex carries in the parent."""
        g = self.g
        if child.contains_pos(g.e):
            return "mu"
        for v in range(child.a, child.b + 2):
            pv = v if v < g.e else v - 1
            a = [i for i, (s, t) in enumerate(g.pairs) if pv in (s, t)][0]
            ps, pt = g.photon_positions(a)
            if not (child.contains_pos(ps) and child.contains_pos(pt)):
                return ("ph", a) if self.mb_ph[a] is parent else "mu"
        raise ValueError("vertex-like block without a leg")

    def _sequence(self, bl):
        """Items of the block's own string in increasing position order."""
        seq = []
        v = bl.a
        children = {c.a: c for c in bl.children}
        while v <= bl.b + 1:
            if v in children:
                c = children[v]
                seq.append(("sub", c))
                v = c.b + 1
                if v <= bl.b:
                    seq.append(("line", v))
                v += 1
                continue
            seq.append(("vtx", self._vertex_label(bl, v)))
            if v <= bl.b:
                seq.append(("line", v))
            v += 1
        return seq

    # ---- evaluate ---------------------------------------------------------
    def __call__(self, z, dtype=np.float64):
        """dtype np.float64; np.longdouble; or object with mpmath numbers in z
        (arbitrary precision, the reference for re-evaluated points)."""
        self.dtype = dtype
        if dtype == np.float64:
            self.ctype = complex
        elif dtype == np.longdouble:
            self.ctype = np.clongdouble
        else:                      # object: mpmath numbers, exact to mp.dps
            self.ctype = object
        z = np.atleast_2d(np.asarray(z, dtype=dtype))
        P = polynomials(z, self.eta, self.alpha, self.beta, self.kappa, self.mass2, dtype=dtype)
        self.P = P
        U, V = P["U"], P["V"]
        n = self.g.n
        val = self._block_value(self.root, z)
        total = np.zeros(z.shape[0], dtype=dtype)
        for k in range(0, n):
            if k >= len(val):
                break
            total = total + ((-1) ** k) * math.gamma(n - k) * U ** -2.0 * V ** (k - n) \
                * (2.0 * U) ** (-k) * val[k]
        return ((-1) ** n) * 4.0 ** (-n) * total

    def _factor_matrix(self, A, C, K, minus_mass=False):
        """(A pslash + 1) (or (A pslash - 1)) with the q / k parts handled by
        the derivative pass; returns [B,4,4]."""
        B = A.shape[0]
        m = np.zeros((B, 4, 4), dtype=self.ctype)
        s = -1.0 if minus_mass else 1.0
        m[:, 0, 0] = m[:, 1, 1] = s + A
        m[:, 2, 2] = m[:, 3, 3] = s - A
        return m

    def _block_value(self, bl, z):
        P = self.P
        Bn = z.shape[0]
        seq = self._sequence(bl)
        # momentum-carrying factors: own lines and wf insertions
        mom = []            # (seq index, eta vector, A, C, K, minus_mass)
        child_vals = []
        for t, (kind, obj) in enumerate(seq):
            if kind == "line":
                l = obj
                mom.append((t, self.eta[l], P["A"][:, l], P["C"][:, l], P["K"][:, l], False))
            elif kind == "sub":
                c = obj
                child_vals.append(self._block_value(c, z))
                if c.kind == "SE" and c.proj == "SEwf":
                    l = c.a - 1
                    mom.append((t, self.eta[l], P["A"][:, l], P["C"][:, l], P["K"][:, l], True))
        photon_pairs = {}
        for t, (kind, obj) in enumerate(seq):
            lab = None
            if kind == "vtx":
                lab = obj
            elif kind == "sub" and obj.kind != "SE":
                lab = self._leg_label(bl, obj)
            if isinstance(lab, tuple):
                photon_pairs.setdefault(lab[1], []).append(t)
        ph_pairs = [tuple(v) for v in photon_pairs.values()]
        for pp in ph_pairs:
            assert len(pp) == 2
        own = {}
        mom_idx = list(range(len(mom)))
        for pat in _pairings(mom_idx):
            k = len(pat)
            coef = np.ones(Bn, dtype=self.dtype)
            for (i, j) in pat:
                coef = coef * b_matrix(P["adj"], mom[i][1], mom[j][1])
            if np.all(coef == 0.0):
                continue
            contracted = set()
            for (i, j) in pat:
                contracted.add(mom[i][0])
                contracted.add(mom[j][0])
            pairs = ph_pairs + [(mom[i][0], mom[j][0]) for (i, j) in pat]
            r = self._project(bl, seq, mom, contracted, pairs, Bn)
            own[k] = own.get(k, 0.0) + coef * r
        kmax = max(own.keys()) if own else 0
        vals = [own.get(k, np.zeros(Bn, dtype=self.dtype)) for k in range(kmax + 1)]
        for cv in child_vals:
            new = [np.zeros(Bn, dtype=self.dtype) for _ in range(len(vals) + len(cv) - 1)]
            for i, x in enumerate(vals):
                for j, y in enumerate(cv):
                    new[i + j] = new[i + j] + x * y
            vals = new
        return vals

    def _items(self, bl, seq, mom, contracted, Bn, deriv=None):
        """Build einsum items; deriv = (seq index, kind) replaces that factor
        by its q- or k-derivative gamma."""
        mom_by_t = {m[0]: m for m in mom}
        items = []
        for t, (kind, obj) in enumerate(seq):
            if t in contracted:
                items.append((None, False, None))
                continue
            if kind == "vtx" or (kind == "sub" and obj.kind != "SE"):
                lab = obj if kind == "vtx" else self._leg_label(bl, obj)
                if lab == "mu":
                    items.append((GAMMA_STACK, False, "M"))
                else:
                    items.append((None, False, None))
                continue
            if kind == "sub" and obj.proj == "SEmass":
                items.append((np.eye(4, dtype=complex), False, None))
                continue
            _, eta, A, C, K, minus = mom_by_t[t]
            if deriv is not None and deriv[0] == t:
                if deriv[1] == "q":
                    items.append((GAMMA_SPATIAL_NEG[None] * C[:, None, None, None], True, "J"))
                else:
                    items.append((GAMMA_LOWER[None] * K[:, None, None, None], True, "N"))
                continue
            items.append((self._factor_matrix(A, C, K, minus), True, None))
        return items

    def _project(self, bl, seq, mom, contracted, pairs, Bn):
        has_mu = any(
            (k == "vtx" and o == "mu") or (k == "sub" and o.kind != "SE" and self._leg_label(bl, o) == "mu")
            for k, o in seq)
        if bl.proj in ("F2", "L", "UV"):
            assert has_mu
            G = _chain(self._items(bl, seq, mom, contracted, Bn), pairs, ["M"], Bn, self.ctype)
            if bl.proj == "L":
                return np.real(dirac.l_of_vertex(G))
            if bl.proj == "UV":
                return np.real(dirac.gamma_mu_coeff(G))
            H = np.zeros((Bn, 4, 3, 4, 4), dtype=self.ctype)
            for (t, eta, A, C, K, minus) in mom:
                if t in contracted or np.all(C == 0.0):
                    continue
                H = H + _chain(self._items(bl, seq, mom, contracted, Bn, (t, "q")), pairs, ["M", "J"], Bn, self.ctype)
            return np.real(dirac.f2_of_vertex(G, H))
        if bl.proj == "SEmass":
            S = _chain(self._items(bl, seq, mom, contracted, Bn), pairs, [], Bn, self.ctype)
            return np.real(0.5 * np.trace(S[:, 0:2, 0:2], axis1=-2, axis2=-1))
        if bl.proj == "SEwf":
            D = np.zeros((Bn, 4, 4, 4), dtype=self.ctype)
            for (t, eta, A, C, K, minus) in mom:
                if t in contracted or np.all(K == 0.0):
                    continue
                D = D + _chain(self._items(bl, seq, mom, contracted, Bn, (t, "k")), pairs, ["N"], Bn, self.ctype)
            # D[nu] = dSigma/dk^nu = b gamma_nu (lower index): tr(gamma^nu D_nu) = 16 b
            acc = 0.0
            for nu in range(4):
                acc = acc + np.trace(dirac.GAMMA[nu] @ D[:, nu], axis1=-2, axis2=-1)
            return np.real(acc / 16.0)
        raise ValueError(bl.proj)


# ---------------------------------------------------------------------------
# forest formula
# ---------------------------------------------------------------------------

def _operator_choices(g, F, gprime):
    """Expand one T(F; G') into signed lists of (root_kin, root_proj, subs)."""
    opts_per = []
    for s in F:
        if gprime is not None and s == gprime:
            opts_per.append([(+1, (s, "q", "F2"))])
        elif gprime is not None and s.lines(g) > gprime.lines(g):
            # an element between G' and the root: (L - U) as a link of the
            # infrared chain plus U as the ultraviolet counterterm of the
            # block enclosing it -- together L
            opts_per.append([(+1, (s, "p", "L"))])
        elif s.kind == "SE":
            opts_per.append([(+1, (s, "p", "SEmass")), (+1, (s, "k", "SEwf"))])
        else:
            opts_per.append([(+1, (s, "0", "UV"))])
    if gprime is None:
        roots = [(+1, "q", "F2")]
    else:
        roots = [(+1, "p", "L"), (-1, "0", "UV")]
    out = []
    for rs, rk, rp in roots:
        for combo in _iproduct(*opts_per) if opts_per else [()]:
            sign = rs
            subs = []
            for sg, sub in combo:
                sign *= sg
                subs.append(sub)
            out.append((sign, rk, rp, subs))
    return out


def forest_terms(g: Graph):
    """All signed terms of A~_G as (sign, TermEvaluator, description)."""
    terms = []
    for F in forests(g):
        fsign = (-1) ** len(F)
        for gprime in [None] + [s for s in F if s.has_x]:
            for sign, rk, rp, subs in _operator_choices(g, F, gprime):
                desc = (tuple((s.a, s.b, kin, proj) for s, kin, proj in subs), rk, rp)
                terms.append((fsign * sign, TermEvaluator(g, rk, rp, subs), desc))
    return terms


class Integrand:
    """A~_G(z) for one graph, homogeneous of degree -3n in z."""

    def __init__(self, g: Graph, subtract: bool = True):
        self.g = g
        if subtract:
            self.terms = forest_terms(g)
        else:
            self.terms = [(1, TermEvaluator(g, "q", "F2", []), ((), "q", "F2"))]

    def __call__(self, z, return_terms=False, dtype=np.float64):
        z = np.atleast_2d(np.asarray(z, dtype=dtype))
        vals = [s * ev(z, dtype=dtype) for s, ev, _ in self.terms]
        tot = np.sum(vals, axis=0)
        if return_terms:
            return tot, vals
        return tot
