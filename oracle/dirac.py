"""Explicit 4x4 Dirac algebra and the F2(0) projection -- oracle side.

Everything is done with explicit matrices in the Dirac representation and in
the electron rest frame p = (m, 0, 0, 0), m = 1, metric (+,-,-,-).  This is
the plain textbook route (Bjorken-Drell spinors); the CUDA side derives its
coefficients by a different route and shares nothing with this file.

F2(0) of a vertex Gamma^mu(p, q) = G^mu + q^j H^mu_j + O(q^2)
(p = average of the in/out momenta, q = out - in, q along a spatial axis, so
p.q = 0 on shell) is read off the on-shell sandwich ubar(p+q/2) Gamma u(p-q/2)
expanded to first order in q with u(k) = sqrt(E+m) (chi, sigma.k/(E+m) chi):

* the charge:        ubar G^0 u = 2 F1 chi'^+ chi  ->  F1 = tr2(G^0_11) / 2;
* the magnetic term: the O(q) part of ubar Gamma^i u is
  2 chi'^+ [H^i_j,11 - (G^i_12 s_j + s_j G^i_21)/4] chi q^j
  = (F1 + F2) i (s x q)^i (plus terms along q^i that carry no moment),
  so F1 + F2 = (i/12) sum_{ijl} eps_ijl tr2(s_l X^i_j) with X^i_j the bracket
  times 2;
* F2 = (F1 + F2) - F1.

Blocks "11", "12", "21" are the upper-left, upper-right and lower-left 2x2
blocks; s_j are the Pauli matrices.
"""
from __future__ import annotations

import numpy as np

I2 = np.eye(2, dtype=complex)
SIG = [np.array([[0, 1], [1, 0]], dtype=complex),
       np.array([[0, -1j], [1j, 0]], dtype=complex),
       np.array([[1, 0], [0, -1]], dtype=complex)]
Z2 = np.zeros((2, 2), dtype=complex)

GAMMA = [np.block([[I2, Z2], [Z2, -I2]])] + [
    np.block([[Z2, s], [-s, Z2]]) for s in SIG]
METRIC = np.array([1.0, -1.0, -1.0, -1.0])
ONE = np.eye(4, dtype=complex)

# T[a,b,c,d] = sum_alpha g_{alpha alpha} (gamma^alpha)_{ab} (gamma^alpha)_{cd}:
# one Feynman-gauge photon (or one contracted loop-momentum pair) joining two
# places of a Dirac string.
TCON = sum(METRIC[a] * np.einsum("ab,cd->abcd", GAMMA[a], GAMMA[a]) for a in range(4))

EPS = np.zeros((3, 3, 3))
EPS[0, 1, 2] = EPS[1, 2, 0] = EPS[2, 0, 1] = 1.0
EPS[0, 2, 1] = EPS[2, 1, 0] = EPS[1, 0, 2] = -1.0


def slash_p(A):
    """A * pslash + 1 in the rest frame (A may be an array of samples)."""
    A = np.asarray(A, dtype=float)
    out = np.zeros(A.shape + (4, 4), dtype=complex)
    out[..., 0, 0] = out[..., 1, 1] = 1 + A
    out[..., 2, 2] = out[..., 3, 3] = 1 - A
    return out


def f2_from_parts(G0_11, Gi_12, Gi_21, Hij_11):
    """F2(0) from the blocks listed in the module docstring.

    G0_11: [..., 2, 2]; Gi_12, Gi_21: [..., 3, 2, 2] (i = x, y, z);
    Hij_11: [..., 3, 3, 2, 2] (H^i_j, derivative along q^j).
    """
    F1 = 0.5 * np.trace(G0_11, axis1=-2, axis2=-1)
    X = 2.0 * Hij_11.copy()
    for i in range(3):
        for j in range(3):
            X[..., i, j, :, :] -= 0.5 * (Gi_12[..., i, :, :] @ SIG[j] + SIG[j] @ Gi_21[..., i, :, :])
    mag = 0.0
    for i in range(3):
        for j in range(3):
            for l in range(3):
                if EPS[i, j, l] != 0.0:
                    mag = mag + EPS[i, j, l] * np.trace(SIG[l] @ X[..., i, j, :, :], axis1=-2, axis2=-1)
    # i/12 applied as (times i) then (divide by 12): exact in the extended
    # precision modes, where a rounded double 1/12 would be amplified by the
    # cancellation between (F1 + F2) and F1
    mag = mag * 1j / 12
    return mag - F1


def f2_of_vertex(G, H):
    """F2(0) from full 4x4 matrices G[mu] ([..., 4, 4, 4]) and
    H[mu][j] = dGamma^mu/dq^j ([..., 4, 3, 4, 4])."""
    return f2_from_parts(G[..., 0, 0:2, 0:2],
                         G[..., 1:4, 0:2, 2:4],
                         G[..., 1:4, 2:4, 0:2],
                         H[..., 1:4, :, 0:2, 0:2])


def l_of_vertex(G):
    """On-shell forward vertex constant: the coefficient of gamma^mu of
    Gamma^mu(p, 0) between on-shell spinors, read off the charge component
    (the F1 of the q=0 vertex)."""
    return 0.5 * np.trace(G[..., 0, 0:2, 0:2], axis1=-2, axis2=-1)


def gamma_mu_coeff(G):
    """c for a vertex at zero external momenta, G^mu = c gamma^mu
    (no vector is available, so the form is exact): tr(gamma_mu G^mu)/16."""
    acc = 0.0
    for mu in range(4):
        acc = acc + METRIC[mu] * np.trace(GAMMA[mu] @ G[..., mu, :, :], axis1=-2, axis2=-1)
    return acc / 16.0
