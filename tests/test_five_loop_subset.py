"""The five-loop workload's graph list: its Philox4x32-10 matches the
published known-answer vectors, and the committed list is the Fisher-Yates
selection it defines (64 distinct graphs of the 6354)."""
from pathlib import Path

from paper_1905_08007_b300 import five_loop_subset as fs

KAT = Path(__file__).resolve().parent / "golden" / "philox4x32_10_kat.txt"


def test_philox_known_answers():
    rows = [ln.split() for ln in KAT.read_text().splitlines() if ln and not ln.startswith("#")]
    assert len(rows) >= 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert fs._philox(tuple(v[0:4]), v[4], v[5]) == tuple(v[6:10])


def test_committed_subset_is_the_shuffle():
    s = fs.read()
    assert s == fs.subset()
    assert len(s) == 64 and len(set(s)) == 64 and 0 <= min(s) and max(s) < 6354
