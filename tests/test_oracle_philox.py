"""Oracle pins: Philox4x32-10 known answers and the uniform map."""
from pathlib import Path

import numpy as np

from oracle.philox import philox4x32_10, philox_np, uniforms, words_to_uniform

GOLD = Path(__file__).parent / "golden"


def _kat():
    for line in (GOLD / "philox4x32_10_kat.txt").read_text().splitlines():
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        yield v[0:4], v[4:6], v[6:10]


def test_known_answers_scalar_and_vector():
    for ctr, key, out in _kat():
        assert list(philox4x32_10(ctr, key)) == out
        w = philox_np(*[np.array([c]) for c in ctr], key[0], key[1])
        assert [int(x[0]) for x in w] == out


def test_uniform_map_open_interval_and_resolution():
    u = words_to_uniform(np.array([0, 0xFFFFFFFF], dtype=np.uint64), np.array([0, 0xFFFFFFFF], dtype=np.uint64))
    assert u[0] == 0.5 * 2.0 ** -52
    assert u[1] == 1.0 - 0.5 * 2.0 ** -52
    assert np.all((u > 0) & (u < 1))


def test_stream_layout_and_moments():
    u = uniforms(np.arange(20000), 3, 12345, 7)
    assert u.shape == (20000, 7)
    assert abs(u.mean() - 0.5) < 0.01
    assert abs(u.var() - 1 / 12) < 0.002
    # draws 2b, 2b+1 come from Philox block b
    w = philox_np(np.array([5]), np.array([0]), np.array([3]), np.array([1]), 12345, 0)
    assert u[5, 2] == words_to_uniform(w[0], w[1])[0]
    assert u[5, 3] == words_to_uniform(w[2], w[3])[0]
