"""The no-allocation entry point (qed_integrate_range_noalloc), called through
the C ABI, against the regular entry point (qed_integrate_range) on the same
samples.

It exists for callers that must not allocate device memory once running
(an application whose pool allocator owns all device memory, or a
latency-critical loop that cannot afford an allocation's implicit device
synchronisation): its scratch is a static device array shared by all calls.
Two calls in a row must both match, which also checks that each call clears
the shared scratch it reuses.  This file is collected last so that a run
stopping at the first failure has already run every other test; it also
passes on its own in a fresh process.
"""
import ctypes as C

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1905_08007_b300 as q                     # noqa: E402
from paper_1905_08007_b300._lib import _Result, _check, load_library   # noqa: E402


def _noalloc(d, begin, n, seed):
    L = load_library()
    f = L.qed_integrate_range_noalloc
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_uint64, C.c_uint64, C.c_uint64, C.POINTER(_Result)]
    r = _Result()
    _check(f(d._h, begin, n, seed, C.byref(r)))
    return q.Result._from_c(r)


@pytest.mark.parametrize("n,gi,count", [(1, 0, 1_000_003), (2, 4, 3_000_017)])
def test_noalloc_matches_regular_entry_point_twice(n, gi, count):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    ctx = q.Context(0)
    d = ctx.load(q.enumerate_graphs(n)[gi])
    ref = d.integrate(count, seed=13, begin=5)
    for _ in range(2):
        r = _noalloc(d, 5, count, 13)
        assert r.n == ref.n
        assert r.n_flagged == ref.n_flagged
        assert r.n_unstable == ref.n_unstable
        assert r.value == pytest.approx(ref.value, rel=1e-12)
        assert r.variance == pytest.approx(ref.variance, rel=1e-12)


def test_noalloc_rejects_too_many_blocks():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    ctx = q.Context(0, threads=128, blocks=4096)
    d = ctx.load(q.enumerate_graphs(1)[0])
    with pytest.raises(q.QedError) as e:
        _noalloc(d, 0, 1000, 0)
    assert e.value.code == -1


def test_noalloc_matches_regular_entry_point_when_the_queue_overflows():
    """Threshold 1e-15 on a self-energy graph flags most points, so both
    entry points overflow their flagged queues (65536 here, 2^22 in the
    context) and re-scan the chunk in the double-double kernel, which alone
    decides which points are flagged: the two agree point for point."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    ctx = q.Context(0, threshold=1e-15)
    d = ctx.load(q.enumerate_graphs(2)[4])
    count = 6_000_011
    ref = d.integrate(count, seed=17, begin=3)
    assert ref.n_flagged > (1 << 22)
    for _ in range(2):
        r = _noalloc(d, 3, count, 17)
        assert (r.n, r.n_flagged, r.n_unstable) == (ref.n, ref.n_flagged, ref.n_unstable)
        assert r.unstable_abs_w == pytest.approx(ref.unstable_abs_w, rel=1e-12, abs=0)
        assert r.value == pytest.approx(ref.value, rel=1e-12)
        assert r.variance == pytest.approx(ref.variance, rel=1e-12)
        assert r.kernel_seconds > 0.0
