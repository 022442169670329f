"""Launch-shape autotuner for the integration kernels.

Times short integrations on fresh counters and keeps the fastest shape:
* per-graph kernels: threads per block x blocks (as multiples of the SM
  count), set on the context with qed_ctx_set_launch;
* interpreter kernels: threads per block x points per thread of the FP64
  interpreter, set with qed_ctx_set_vm (bench.py runs this at set-up);
* batched kernel: the work-item size (samples per item), which trades the
  device queue's load balance against per-item overhead (bench.py too).
The register budget is fixed at build time by __launch_bounds__(256); it
does not bind the interpreter kernels, whose resident warps are set by the
shared-memory frame of the programs' registers.
Results are throughput only: the estimate itself does not depend on the
shape beyond summation order.
"""
from __future__ import annotations

import itertools


def tune_launch(ctx, diag, samples=1 << 24, threads=(64, 128, 256), blocks_per_sm=(2, 4, 8), sms=148):
    best = None
    table = []
    for t, b in itertools.product(threads, blocks_per_sm):
        ctx.set_launch(t, b * sms)
        diag.integrate(samples // 4, seed=99, begin=1 << 50)          # warm-up
        r = diag.integrate(samples, seed=99, begin=(1 << 50) + samples)
        rate = samples / r.kernel_seconds
        table.append({"threads": t, "blocks": b * sms, "samples_per_s": rate})
        if best is None or rate > best["samples_per_s"]:
            best = table[-1]
    ctx.set_launch(best["threads"], best["blocks"])
    return best, table


def tune_batch_chunk(ctx, diags, samples=1 << 27, chunks=(1 << 16, 1 << 17, 1 << 18, 1 << 19)):
    best = None
    table = []
    for c in chunks:
        ctx.integrate_batch(diags, samples // 4, seed=98, rounds=1, chunk=c, counter_base=1 << 52)
        res = ctx.integrate_batch(diags, samples, seed=98, rounds=2, chunk=c, counter_base=(1 << 52) + samples)
        n = sum(r.n for r in res)
        rate = n / res[0].seconds
        table.append({"chunk": c, "samples_per_s": rate})
        if best is None or rate > best["samples_per_s"]:
            best = table[-1]
    return best, table


def tune_vm(ctx, diags, samples=1 << 20, threads=(64, 128, 256), points=(1, 2), chunk=1 << 11):
    """Interpreter kernels (bytecode integrands): threads per block and points
    per thread of the FP64 interpreter (qed_ctx_set_vm), timed on the FP64
    batched kernel's device time over a short batch of the given graphs.
    The shape whose shared-memory frame does not fit is halved by the library
    itself; the double-double kernels pick their own block size by occupancy.
    Leaves the fastest shape set on the context."""
    best = None
    table = []
    for t, p in itertools.product(threads, points):
        ctx.set_vm(t, p)
        ctx.integrate_batch(diags, samples // 4, seed=97, rounds=1, chunk=chunk, counter_base=1 << 53)
        res = ctx.integrate_batch(diags, samples, seed=97, rounds=1, chunk=chunk, counter_base=(1 << 53) + samples)
        n = sum(r.n for r in res)
        rate = n / res[0].kernel_seconds
        table.append({"threads": t, "points": p, "samples_per_s": rate})
        if best is None or rate > best["samples_per_s"]:
            best = table[-1]
    ctx.set_vm(best["threads"], best["points"])
    return best, table
