"""Philox4x32-10 counter-based generator -- oracle side (test infrastructure).

Sec. 3 of the paper runs Calc 2 with the Philox_4x32_10 generator.  The
generator is Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11: a 4x32-bit counter, a 2x32-bit key, ten rounds, each round two
32x32->64 multiplies by fixed odd multipliers followed by a word permutation
with key xor; the key is bumped by two Weyl constants between rounds.

Stream layout used by both sides of this project (stated here as a
definition, not shared code):
  counter = (sample lo32, sample hi32, diagram id, block), key = (seed lo32,
  seed hi32); draw d of a sample uses block d // 2, words 2*(d % 2) and
  2*(d % 2) + 1; u = ((((w_hi << 32) | w_lo) >> 12) + 0.5) * 2**-52: 52 random
  bits, every value exactly representable and strictly inside (0,1) (a
  53-bit version would round its top value to 1.0).
"""
from __future__ import annotations

import numpy as np

MULT0 = 0xD2511F53
MULT1 = 0xCD9E8D57
WEYL0 = 0x9E3779B9
WEYL1 = 0xBB67AE85
M32 = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """Scalar reference: ctr = 4 ints, key = 2 ints -> 4 ints."""
    c0, c1, c2, c3 = (int(x) & M32 for x in ctr)
    k0, k1 = (int(x) & M32 for x in key)
    for r in range(10):
        p0 = MULT0 * c0
        p1 = MULT1 * c2
        hi0, lo0 = p0 >> 32, p0 & M32
        hi1, lo1 = p1 >> 32, p1 & M32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & M32, lo1, (hi0 ^ c3 ^ k1) & M32, lo0
        k0 = (k0 + WEYL0) & M32
        k1 = (k1 + WEYL1) & M32
    return (c0, c1, c2, c3)


def philox_np(c0, c1, c2, c3, k0, k1):
    """Vectorised over numpy uint64 arrays holding 32-bit values."""
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) & np.uint64(M32) for x in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & np.uint64(M32)
    k1 = np.asarray(k1, dtype=np.uint64) & np.uint64(M32)
    m32 = np.uint64(M32)
    s32 = np.uint64(32)
    for r in range(10):
        p0 = np.uint64(MULT0) * c0
        p1 = np.uint64(MULT1) * c2
        hi0, lo0 = p0 >> s32, p0 & m32
        hi1, lo1 = p1 >> s32, p1 & m32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & m32, lo1, (hi0 ^ c3 ^ k1) & m32, lo0
        k0 = (k0 + np.uint64(WEYL0)) & m32
        k1 = (k1 + np.uint64(WEYL1)) & m32
    return c0, c1, c2, c3


def words_to_uniform(w_hi, w_lo):
    """Two 32-bit words -> one double strictly inside (0,1), 52 random bits."""
    w_hi = np.asarray(w_hi, dtype=np.uint64)
    w_lo = np.asarray(w_lo, dtype=np.uint64)
    x = ((w_hi << np.uint64(32)) | w_lo) >> np.uint64(12)
    return (x.astype(np.float64) + 0.5) * 2.0 ** -52


def uniforms(sample_idx, diagram_id: int, seed: int, n_draws: int):
    """Uniform draws [len(sample_idx), n_draws] for the given samples."""
    s = np.asarray(sample_idx, dtype=np.uint64)
    lo = s & np.uint64(M32)
    hi = s >> np.uint64(32)
    k0 = np.uint64(seed & M32)
    k1 = np.uint64((seed >> 32) & M32)
    out = np.empty((s.size, n_draws), dtype=np.float64)
    for blk in range((n_draws + 1) // 2):
        w = philox_np(lo, hi, np.full_like(lo, diagram_id), np.full_like(lo, blk), k0, k1)
        out[:, 2 * blk] = words_to_uniform(w[0], w[1])
        if 2 * blk + 1 < n_draws:
            out[:, 2 * blk + 1] = words_to_uniform(w[2], w[3])
    return out
