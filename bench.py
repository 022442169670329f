"""Benchmark: Monte Carlo samples/s on the two-loop lepton-loop-free vertex set.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

A step is one pass of the whole hot path over one batch: the six two-loop
graphs integrated together with 6 x `--samples` fresh Philox counters
(default 6e8 samples per step) in the persistent batched kernel, samples
shared by running variance, from Deg-calibrated and gradient-tuned densities
(set up once before the warm-up, time reported), with the forest-subtracted
FP64 integrand, double-double re-evaluation of flagged points and compensated
reductions.  There is no input stream: points are generated from counters on
the device, so the L2 flush between steps only keeps the timing honest for
the tables.  The plain per-graph path (untuned densities, equal samples) is
reported beside it.

Multi-GPU (torchrun, one rank per GPU): every rank integrates its own disjoint
counter blocks (weak scaling); the only exchange is the final merge of the
per-graph moments (48 bytes per graph).

--impl reference times the CPU oracle on the same workload and metric, on a
bounded sample, on rank 0.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "MC samples/s and time-to-target-sigma per loop-order diagram set; FP64-pipe % of peak"
ZETA3 = 1.2020569031595942
TWO_LOOP_TARGET = (197 / 144 + math.pi ** 2 / 12 - math.pi ** 2 * math.log(2) / 2 + 3 * ZETA3 / 4) \
    - (119 / 36 - math.pi ** 2 / 3)
SIGMA_TARGET = 1e-5
# time-to-sigma target per loop order (four loops: sigma_total = 5e-3)
SIGMA_TARGETS = {1: 1e-5, 2: 1e-5, 3: 1e-4, 4: 5e-3, 5: 0.1}
# samples per graph per step: 6e8 per step on the two-loop set, 1e9 on the
# three-loop set (BASELINE's config 3 budget)
DEFAULT_SAMPLES = {1: 1e8, 2: 1e8, 3: 2e7, 4: 2 ** 16, 5: 2 ** 12}
# work-item size of the batched kernel per order (a four-loop sample is ~1e5
# FP64 operations, a five-loop one ~1e6): at four loops 2048 samples give
# about 15 items per persistent block and round, so the blocks finish together
CHUNK = {1: 1 << 18, 2: 1 << 18, 3: 1 << 18, 4: 1 << 11, 5: 1 << 11}
CLOSED_FORM = {1: 0.5, 2: TWO_LOOP_TARGET}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in Path(self.path).read_text().splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) < 8:
                continue
            try:
                rows.append((float(p[0]), float(p[1]), p[4:8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def _peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        return json.loads(p.read_text())
    return {}


def mirror_weights(graphs):
    """2 - [self-mirror] per graph of a mirror-reduced set (Sec. 3 counts each
    mirror pair once; the set total is the weighted sum)."""
    w = []
    for g in graphs:
        m = 2 * g.n - 1
        mp = tuple(sorted((min(m - s, m - t), max(m - s, m - t)) for s, t in g.pairs))
        w.append(1.0 if (mp, 2 * g.n - g.e) == (tuple(g.pairs), g.e) else 2.0)
    return w


def graph_set(q, order):
    """The benchmarked set: every graph up to three loops (mirror pairs both
    present), one per mirror pair at four loops (bytecode integrands), the
    64-graph five-loop workload (five_loop_subset.txt) at five."""
    if order == 5:
        from paper_1905_08007_b300.five_loop_subset import read
        every = q.enumerate_graphs(5)
        gs = [every[i] for i in read()]
        return gs, [1.0] * len(gs)
    if order == 4:
        gs = q.enumerate_graphs(order, reduced=True)
        return gs, mirror_weights(gs)
    gs = q.enumerate_graphs(order)
    return gs, [1.0] * len(gs)


def cpu_baseline(n_per_graph=None, seed=0, order=2):
    """The oracle as it stands on this host's cores (numpy, one thread of work),
    on a bounded sample of the same graph set (about 10-20 s)."""
    from oracle.estimator import weights
    from oracle.graphs import enumerate_graphs
    from oracle.integrand import Integrand
    graphs = enumerate_graphs(order)
    if order == 3:
        graphs = graphs[::10]
    if order == 4:
        graphs = graphs[85:86]
    n_per_graph = n_per_graph or {1: 3000, 2: 300, 3: 20, 4: 2}[order]
    t0 = time.perf_counter()
    tot = 0
    for g in graphs:
        sid = enumerate_graphs(order).index(g)
        w = weights(Integrand(g), g, sid, seed, 10**12, n_per_graph)
        tot += w.size
    dt = time.perf_counter() - t0
    return {"value": tot / dt, "unit": "samples/s", "cores": 1, "kind": "oracle",
            "sample": f"{n_per_graph} samples of each of {len(graphs)} {order}-loop graphs "
                      f"(Philox counters 1e12.., seed {seed}), {dt:.1f} s"}


def compare_plain(diags, graphs, ctx, S, seed, t_step, sigma_step, q):
    """The plain per-graph path on the same budget: untuned Eq. (1) densities
    (the Deg rule), equal samples per graph, one launch per graph; time to
    the target sigma against the batched, calibrated, tuned step."""
    plain = [ctx.load(g) for g in graphs]
    res = [d.integrate(S, seed=seed + 1, begin=1 << 41) for d in plain]
    t = sum(r.seconds for r in res)
    mw = mirror_weights(graphs) if graphs[0].n >= 4 else [1.0] * len(graphs)
    sig = math.sqrt(sum(w * w * r.variance for w, r in zip(mw, res)))
    st = SIGMA_TARGETS[graphs[0].n]
    tts_plain = t * (sig / st) ** 2
    tts_batch = t_step * (sigma_step / st) ** 2
    return {"seconds": t, "samples_per_s": S * len(graphs) / t, "sigma": sig,
            "total": sum(w * r.value for w, r in zip(mw, res)), "time_to_sigma": tts_plain,
            "kernel_seconds": sum(r.kernel_seconds for r in res),
            "speedup_time_to_sigma_batched_tuned_vs_plain": tts_plain / tts_batch,
            "note": "the plain densities give heavy-tailed weights on the self-energy graphs, so "
                    "this sigma is itself an underestimate"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    n = args.ref_samples
    from oracle.estimator import weights
    from oracle.graphs import enumerate_graphs
    from oracle.integrand import Integrand
    graphs = enumerate_graphs(args.order)
    if args.order >= 4:
        # bounded sample: a four-loop point costs the oracle seconds
        graphs = graphs[85::108]
        n = 1
    fs = [Integrand(g) for g in graphs]

    def step(s):
        tot = 0
        for sid, (g, f) in enumerate(zip(graphs, fs)):
            w = weights(f, g, sid, args.seed, s * n, n)
            tot += w.size
        return tot
    for s in range(args.warmup):
        step(s)
    t0 = time.perf_counter()
    tot = sum(step(args.warmup + s) for s in range(args.steps))
    dt = time.perf_counter() - t0
    v = tot / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "samples/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (Philox counters)",
        "config": {"workload": f"{args.order}-loop lepton-loop-free vertex set: {len(graphs)} graphs, "
                               "Eq. (1) density, forest-subtracted integrand, FP64 (the CPU oracle)",
                   "loops": args.order, "graphs": len(graphs),
                   "samples_per_graph_per_step": n, "seed": args.seed},
        "cpu_baseline": {"value": v, "unit": "samples/s", "cores": 1, "kind": "oracle",
                         "sample": f"{n} samples per graph per step, {args.steps} steps"},
        "e2e": {"value": v, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_native(args):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import paper_1905_08007_b300 as q
    from paper_1905_08007_b300.tune import tune
    ctx = q.Context(local)
    stream = torch.cuda.current_stream()
    ctx.set_stream(stream)
    graphs, mw = graph_set(q, args.order)
    S = int(args.samples if args.samples else DEFAULT_SAMPLES[args.order])
    total = S * len(graphs)
    fp64_peak = q.fp64_peak(local, 50.0)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    # set-up (not timed): Deg calibrated on the integrand, densities tuned
    t0 = time.perf_counter()
    diags = [ctx.load(g) for g in graphs]
    # one and two loops: Deg calibrated on the integrand, then tuned; from
    # three loops on the calibration (too few base points for 9 or 12 lines)
    # sends samples into corners where even double-double fails (three
    # loops, calibrated + tuned: 51 % of the samples flagged, 15 % unstable),
    # so only the gradient tuning runs; at five loops the Deg rule is used as
    # it is
    ts, tn = {1: (10, 1 << 21), 2: (10, 1 << 21), 3: (10, 1 << 21), 4: (4, 1 << 15), 5: (0, 0)}[args.order]
    for d in diags:
        if args.order <= 2:
            d.calibrate_deg(n_base=8, seed=args.seed + 5)
        if ts:
            tune(d, steps=ts, n=tn, lr=0.08, seed=args.seed + 7)
    setup_s = time.perf_counter() - t0
    flops = [d.flops_per_sample() for d in diags]
    rounds, chunk = 4, int(args.chunk or CHUNK[args.order])

    def step(s):
        base = (s * ws + rank) * total + (1 << 40)      # fresh counters every step and rank
        return ctx.integrate_batch(diags, total, seed=args.seed, policy="variance", rounds=rounds,
                                   chunk=chunk, counter_base=base)

    for s in range(args.warmup):
        flush.zero_()
        step(s)
    acc = [None] * len(diags)
    clocks = Clocks(local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    launches, ksec, alg, nsamp = 0, 0.0, 0.0, 0
    wall0 = time.perf_counter()
    ev0.record(stream)
    for s in range(args.steps):
        flush.zero_()
        res = step(args.warmup + s)
        launches += res[0].launches
        ksec += res[0].kernel_seconds
        for i, r in enumerate(res):
            alg += flops[i] * r.n
            nsamp += r.n
            acc[i] = r if acc[i] is None else q.merge_results(acc[i], r)
    ev1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    t = ev0.elapsed_time(ev1) * 1e-3
    tmax, wmax = t, wall
    results = acc
    if ws > 1:
        import torch.distributed as dist
        tt = torch.tensor([t, wall], device="cuda", dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        tmax, wmax = float(tt[0]), float(tt[1])
        gathered = [None] * ws
        dist.all_gather_object(gathered, [(r.sum_w, r.sum_w2, r.n, r.n_flagged, r.n_unstable) for r in acc])
        results = []
        for i in range(len(diags)):
            m = None
            for rk in range(ws):
                sw, sw2, n, nf, nu = gathered[rk][i]
                r = q.Result(0.0, 0.0, tuple(sw), tuple(sw2), n, nf, nu, 0.0)
                m = r if m is None else q.merge_results(m, r)
            results.append(m)
    if rank != 0:
        return 0
    total_samples = ws * nsamp
    value = total_samples / tmax
    tot = sum(w * r.value for w, r in zip(mw, results))
    sigma = math.sqrt(sum(w * w * r.variance for w, r in zip(mw, results)))
    achieved = alg / ksec / 1e12
    peak = fp64_peak / 1e12
    n_items = max(len(diags), (total // rounds + chunk - 1) // chunk)
    flagged = sum(r.n_flagged for r in results)
    line = {
        "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tmax / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (Philox counters)",
        "config": {"workload": f"{args.order}-loop lepton-loop-free vertex set: {len(graphs)} graphs"
                               + {4: " (one per mirror pair, bytecode integrands)",
                                  5: " (the 64-graph workload, bytecode integrands)"}.get(args.order, "") + ", "
                               f"{total:.0e} Philox samples per step shared by running variance, "
                               + {3: "gradient-tuned Deg-rule densities", 4: "gradient-tuned Deg-rule densities",
                                  5: "Deg-rule densities"}.get(
                                   args.order, "Deg-calibrated + gradient-tuned densities")
                               + ", forest-subtracted FP64 integrand, double-double re-evaluation, "
                               "persistent batched kernel (4 CUDA-graph rounds per step)",
                   "loops": args.order, "graphs": len(graphs), "samples_per_step": total, "seed": args.seed, "l2_flush": True,
                   "launch": {"threads": 256, "items_per_round": n_items, "chunk": chunk},
                   "setup_seconds_calibrate_and_tune": setup_s},
        "set_total": {"loops": args.order, "value": tot, "sigma": sigma,
                           "closed_form": CLOSED_FORM.get(args.order),
                           "pull": ((tot - CLOSED_FORM[args.order]) / sigma
                                    if sigma > 0 and args.order in CLOSED_FORM else None),
                           "flagged_fraction": flagged / total_samples,
                           "unstable": sum(r.n_unstable for r in results),
                           "samples_per_graph": [r.n for r in results]},
        "time_to_sigma": {"target_sigma": SIGMA_TARGETS[args.order],
                          "seconds": tmax * (sigma / SIGMA_TARGETS[args.order]) ** 2,
                          "sigma_reached": sigma, "seconds_run": tmax},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": ("k_batch_fp64 (persistent FP64 integration kernel)" if args.order <= 3 else
                                f"k_batch_vm_fp64<{3 * args.order}> (persistent FP64 interpreter kernel, "
                                "bytecode integrands)"),
                     "peak_source": "measured FP64 FMA throughput (qed_fp64_peak), of measured",
                     "flops_per_sample": {str(i): f for i, f in enumerate(flops)}},
        "gpu_launches": launches,
        "e2e": {"value": total_samples / wmax, "unit": "samples/s",
                "h2d_bytes_per_step": rounds * n_items * 16,
                "d2h_bytes_per_step": rounds * n_items * 96},
        "clocks": clk,
    }
    if ws == 1 and args.compare and args.order in (2, 4):
        line["plain_per_graph"] = compare_plain(diags, graphs, ctx, S, args.seed, tmax / args.steps, sigma, q)
    if ws == 1 and not args.no_cpu_baseline and args.order <= 4:
        line["cpu_baseline"] = cpu_baseline(order=args.order)
    print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--samples", type=float, default=None, help="samples per graph per step")
    ap.add_argument("--order", type=int, default=2, choices=[1, 2, 3, 4, 5], help="loop order of the graph set")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--chunk", type=int, default=None, help="samples per work item of the batched kernel")
    ap.add_argument("--ref-samples", type=int, default=60)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", dest="compare", action="store_false",
                    help="skip the plain vs batched-tuned time-to-sigma comparison")
    a = ap.parse_args(argv)
    if a.warmup < 3:
        a.warmup = 3
    if a.impl == "reference":
        return run_reference(a)
    return run_native(a)


if __name__ == "__main__":
    sys.exit(main())
