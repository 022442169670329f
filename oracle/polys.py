"""Feynman-parametric graph polynomials -- oracle side (test infrastructure).

Sec. 2 (item 4) writes each graph's contribution as one Feynman-parametric
integral.  The polynomials are the textbook ones, built here from an explicit
loop-momentum basis, line by line:

  k_l = sum_a eta_la ell_a + P_l           (line momentum; P_l external part)
  sum_l z_l (k_l^2 - m_l^2) = ell' Lambda ell' - V     after the shift
  Lambda_ab = sum_l z_l eta_la eta_lb,      U = det Lambda,
  J_a = sum_l z_l eta_la P_l,               Q_l = P_l - eta_l . Lambda^-1 J,
  V = sum_l z_l m_l^2 - sum_l z_l Q_l^2     (at q = 0, p^2 = m^2 = 1),
  B_ij = eta_i . adj(Lambda) . eta_j         (so <ell'_i ell'_j> ~ B_ij / U).

P_l = alpha_l p + beta_l q + kappa_l k, so Q_l = A_l p + C_l q + K_l k.

Everything is vectorised over a leading batch of sample points.
"""
from __future__ import annotations

import numpy as np


def _det_laplace(m):
    """Determinant of [B, k, k] by Laplace expansion along the first row."""
    k = m.shape[1]
    if k == 1:
        return m[:, 0, 0]
    if k == 2:
        return m[:, 0, 0] * m[:, 1, 1] - m[:, 0, 1] * m[:, 1, 0]
    tot = None
    for c in range(k):
        minor = np.delete(np.delete(m, 0, axis=1), c, axis=2)
        term = m[:, 0, c] * _det_laplace(minor)
        tot = term if tot is None else (tot + term if c % 2 == 0 else tot - term)
    return tot


def _det_adj_cofactor(lam):
    """Determinant and adjugate by cofactor expansion (any float dtype);
    used for the extended-precision mode.  adj[r, c] = (-1)^(r+c) times the
    minor of lam without row c and column r."""
    B, n, _ = lam.shape
    if n == 1:
        return lam[:, 0, 0].copy(), np.ones_like(lam)
    if n == 2:
        adj = np.empty_like(lam)
        adj[:, 0, 0] = lam[:, 1, 1]
        adj[:, 1, 1] = lam[:, 0, 0]
        adj[:, 0, 1] = -lam[:, 0, 1]
        adj[:, 1, 0] = -lam[:, 1, 0]
        return lam[:, 0, 0] * lam[:, 1, 1] - lam[:, 0, 1] * lam[:, 1, 0], adj
    if n == 3:
        adj = np.empty_like(lam)
        for r in range(3):
            for c in range(3):
                rr = [i for i in range(3) if i != c]
                cc = [j for j in range(3) if j != r]
                m = lam[:, rr][:, :, cc]
                adj[:, r, c] = (-1) ** (r + c) * (m[:, 0, 0] * m[:, 1, 1] - m[:, 0, 1] * m[:, 1, 0])
        det = lam[:, 0, 0] * adj[:, 0, 0] + lam[:, 0, 1] * adj[:, 1, 0] + lam[:, 0, 2] * adj[:, 2, 0]
        return det, adj
    adj = np.empty_like(lam)
    for r in range(n):
        for c in range(n):
            minor = np.delete(np.delete(lam, c, axis=1), r, axis=2)
            adj[:, r, c] = (-1) ** (r + c) * _det_laplace(minor)
    det = lam[:, 0, 0] * adj[:, 0, 0]
    for c in range(1, n):
        det = det + lam[:, 0, c] * adj[:, c, 0]
    return det, adj


def polynomials(z, eta, alpha, beta, kappa, mass2, dtype=np.float64):
    """z: [B, L]; eta: [L, n] (0/1 incidence); alpha/beta/kappa/mass2: [L].
    dtype: np.float64 (default) or np.longdouble (64-bit mantissa on x86).

    Returns dict with U [B], adj [B,n,n], A, C, K [B, L], V [B].
    """
    z = np.atleast_2d(np.asarray(z, dtype=dtype))
    eta = np.asarray(eta, dtype=dtype)
    n = eta.shape[1]
    lam = np.einsum("bl,la,lc->bac", z, eta, eta)
    if n == 0:
        U = np.ones(z.shape[0], dtype=dtype)
        inv = np.zeros((z.shape[0], 0, 0), dtype=dtype)
    elif dtype == np.float64:
        U = np.linalg.det(lam)
        inv = np.linalg.inv(lam)
    else:
        U, adj0 = _det_adj_cofactor(lam)
        inv = adj0 / U[:, None, None]
    adj = inv * U[:, None, None]
    out = {"U": U, "adj": adj, "inv": inv}
    for name, coef in (("A", alpha), ("C", beta), ("K", kappa)):
        coef = np.asarray(coef, dtype=dtype)
        J = np.einsum("bl,la,l->ba", z, eta, coef)
        shift = np.einsum("la,bac,bc->bl", eta, inv, J)
        out[name] = coef[None, :] - shift
    out["V"] = z @ np.asarray(mass2, dtype=dtype) - np.sum(z * out["A"] ** 2, axis=1)
    return out


def b_matrix(adj, eta_i, eta_j):
    """B_ij = eta_i . adj . eta_j for one pair of (possibly equal) factors."""
    return np.einsum("a,bac,c->b", eta_i, adj, eta_j)


def spanning_tree_u(g_edges, n_vertices, z):
    """U by brute force: sum over spanning trees T of prod_{l not in T} z_l
    (Kirchhoff); g_edges is a list of (u, v) vertex pairs.  Small graphs only."""
    from itertools import combinations
    L = len(g_edges)
    total = 0.0
    for tree in combinations(range(L), n_vertices - 1):
        parent = list(range(n_vertices))

        def find(x):
            while parent[x] != x:
                parent[x] = parent[parent[x]]
                x = parent[x]
            return x
        ok = True
        for l in tree:
            a, b = find(g_edges[l][0]), find(g_edges[l][1])
            if a == b:
                ok = False
                break
            parent[a] = b
        if ok:
            prod = 1.0
            for l in range(L):
                if l not in tree:
                    prod *= z[l]
            total += prod
    return total
