"""GPU tests of the batched persistent integrator (all graphs of an order in
one launch per round, variance-driven allocation, CUDA-graph replay): each
graph's batch result must equal the per-graph integration of the same counter
range (the same samples, summed in another order), for both allocation
policies, with and without graph replay, and with flagged lists forced to
overflow."""
import math

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1905_08007_b300 as q   # noqa: E402


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    ctx = q.Context(0)
    ds = [ctx.load(g) for g in q.enumerate_graphs(2)]
    return ctx, ds


@pytest.mark.parametrize("policy,use_graph,list_div", [("variance", True, 16), ("equal", False, 16),
                                                       ("variance", True, 100000)])
def test_batch_equals_per_graph_on_same_counters(setup, policy, use_graph, list_div):
    ctx, ds = setup
    res = ctx.integrate_batch(ds, 24 * (1 << 18), seed=4, policy=policy, rounds=3, chunk=1 << 18,
                              use_graph=use_graph, list_div=list_div)
    assert sum(r.n for r in res) >= 24 * (1 << 18)
    for d, r in zip(ds, res):
        ref = d.integrate(r.n, seed=4, begin=0)
        assert r.n == ref.n
        assert r.value == pytest.approx(ref.value, rel=1e-11, abs=1e-15)
        assert r.variance == pytest.approx(ref.variance, rel=1e-9)
        assert r.n_flagged == ref.n_flagged
        assert r.n_unstable == ref.n_unstable


def test_batch_variance_policy_moves_samples_to_noisy_graphs(setup):
    ctx, ds = setup
    res = ctx.integrate_batch(ds, 512 * (1 << 15), seed=5, policy="variance", rounds=4, chunk=1 << 15)
    per_sample_sigma = [math.sqrt(r.variance * r.n) for r in res]
    # the noisiest graph gets more samples than the quietest one
    hi = max(range(6), key=lambda i: per_sample_sigma[i])
    lo = min(range(6), key=lambda i: per_sample_sigma[i])
    assert res[hi].n > res[lo].n
    assert len({r.n for r in res}) > 1


def test_batch_is_deterministic(setup):
    ctx, ds = setup
    a = ctx.integrate_batch(ds, 12 * (1 << 18), seed=6, rounds=2)
    b = ctx.integrate_batch(ds, 12 * (1 << 18), seed=6, rounds=2)
    assert [r.sum_w for r in a] == [r.sum_w for r in b]


def test_autotuner_picks_a_measured_shape(setup):
    from paper_1905_08007_b300.autotune import tune_batch_chunk, tune_launch
    ctx, ds = setup
    best, table = tune_launch(ctx, ds[0], samples=1 << 22, threads=(128, 256), blocks_per_sm=(2, 4))
    assert best["samples_per_s"] == max(t["samples_per_s"] for t in table)
    ctx.set_launch(256, 0)
    bc, tb = tune_batch_chunk(ctx, ds, samples=1 << 24, chunks=(1 << 16, 1 << 18))
    assert bc["samples_per_s"] == max(t["samples_per_s"] for t in tb)


def test_batch_times_its_kernel_and_leaves_no_cuda_error(setup):
    """The persistent kernel's time is reported, and a torch kernel launched
    right after a batched call (graph replay) sees no stale CUDA error."""
    ctx, ds = setup
    res = ctx.integrate_batch(ds, 12 * (1 << 18), seed=8, rounds=2)
    assert 0.0 < res[0].kernel_seconds <= res[0].seconds
    x = torch.zeros(1 << 20, device="cuda")
    x.add_(1.0)
    torch.cuda.synchronize()
    assert float(x.sum()) == float(1 << 20)
