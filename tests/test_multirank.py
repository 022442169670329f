"""Multi-rank path on the CPU (gloo, world size 2): every rank takes its own
disjoint block of Philox counters (weak scaling, no data-path collective), the
per-graph moments are gathered once and merged in a fixed order with the
library's qed_result_merge (double-double sums); the merged estimate must
equal one process covering the whole range.  The per-sample weights come from
the oracle here because the ranks have no GPU; on GPUs the same merge follows
qed_integrate_range on each rank (bench.py)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import paper_1905_08007_b300 as q

N_PER_RANK = 3000


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _moments(rank, begin, n):
    from oracle.estimator import neumaier_sum, weights
    from oracle.graphs import enumerate_graphs
    from oracle.integrand import Integrand
    g = enumerate_graphs(1)[0]
    w = weights(Integrand(g), g, 0, 3, begin, n)
    return neumaier_sum(w), neumaier_sum(w * w), n


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sw, sw2, n = _moments(rank, rank * N_PER_RANK, N_PER_RANK)
    got = [None] * world
    dist.all_gather_object(got, (sw, sw2, n))
    if rank == 0:
        m = None
        for (a, b, c) in got:
            r = q.Result(0.0, 0.0, (a, 0.0), (b, 0.0), c, 0, 0, 0.0)
            m = r if m is None else q.merge_results(m, r)
        out.put((m.value, m.variance, m.n))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_merge_equals_single_run():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    value, variance, n = out.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sw, sw2, n1 = _moments(0, 0, 2 * N_PER_RANK)
    mean = sw / n1
    var = (sw2 / n1 - mean * mean) / (n1 - 1)
    assert n == n1
    assert value == pytest.approx(mean, rel=1e-13)
    assert variance == pytest.approx(var, rel=1e-10)
