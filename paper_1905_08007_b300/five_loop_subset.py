"""The five-loop workload: 64 graphs drawn from the 6354 lepton-loop-free
five-loop vertex graphs (both orientations, in the enumeration order of
qed_enumerate) by a Fisher-Yates shuffle driven by Philox4x32-10 with seed 0.

    python -m paper_1905_08007_b300.five_loop_subset   # rewrites five_loop_subset.txt

Step i of the shuffle (i = 6353, 6352, ...) takes the draw of counter
(i, 0, 0, 0) and key (0, 0): words (x, y) -> u = ((x << 32 | y) >> 12) + 1/2)
* 2^-52, j = floor(u * (i + 1)), swap a[i] and a[j]; the graphs that end in
the last 64 places form the set, listed in ascending index order.
"""
from pathlib import Path

N_FIVE_LOOP = 6354
SUBSET_SIZE = 64
PATH = Path(__file__).resolve().parent / "five_loop_subset.txt"
_M = 0xFFFFFFFF


def _philox(c, k0, k1):
    """Philox4x32-10 (Salmon et al., SC'11): 10 rounds, multipliers
    0xD2511F53 / 0xCD9E8D57, key increments 0x9E3779B9 / 0xBB67AE85."""
    c0, c1, c2, c3 = c
    for _ in range(10):
        p0 = 0xD2511F53 * c0
        p1 = 0xCD9E8D57 * c2
        c0, c1, c2, c3 = ((p1 >> 32) ^ c1 ^ k0) & _M, p1 & _M, ((p0 >> 32) ^ c3 ^ k1) & _M, p0 & _M
        k0 = (k0 + 0x9E3779B9) & _M
        k1 = (k1 + 0xBB67AE85) & _M
    return c0, c1, c2, c3


def subset(n=N_FIVE_LOOP, size=SUBSET_SIZE, seed=0):
    a = list(range(n))
    for i in range(n - 1, n - 1 - size, -1):
        x, y, _, _ = _philox((i, 0, 0, 0), seed & _M, seed >> 32)
        u = ((((x << 32) | y) >> 12) + 0.5) * 2.0 ** -52
        j = int(u * (i + 1))
        a[i], a[j] = a[j], a[i]
    return sorted(a[n - size:])


def read():
    return [int(t) for t in PATH.read_text().split()]


if __name__ == "__main__":
    PATH.write_text(" ".join(str(i) for i in subset()) + "\n")
    print(PATH, read())
