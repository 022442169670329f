"""Benchmark: Monte Carlo samples/s, time to a target sigma and FP64 fraction
on a loop-order set of lepton-loop-free vertex graphs (default: four loops).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
                    [--order 2|3|4|5]

A step is one pass of the whole hot path over one batch: every graph of the
set (four loops: the 269 mirror-reduced graphs, bytecode integrands)
integrated together with `--samples` fresh Philox counters per graph
(default 2^16 at four loops, 1.76e7 per step) in the persistent batched
kernels, samples shared by running variance, from Deg-calibrated and
gradient-tuned densities (set up once before the warm-up, time reported),
with the forest-subtracted FP64 integrand, double-double re-evaluation of
flagged points and compensated reductions.  There is no input stream:
points are generated from counters on the device, so the L2 flush between
steps only keeps the timing honest for the tables and programs.  The plain
per-graph path (Deg-rule densities, equal samples, one launch pair per graph)
is timed beside it on the same budget for the time-to-sigma comparison, and
a short two-loop run reports its pull against the two-loop closed form.

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
# samples per graph per step: 6e8 per step on the two-loop set, 1.2e8 on the
# 28 mirror-reduced three-loop graphs, 8.8e6 on the 269 four-loop graphs
# (about 5 s of device time), 2^16 per graph of the five-loop workload
DEFAULT_SAMPLES = {1: 1e8, 2: 1e8, 3: 2 ** 22, 4: 2 ** 15, 5: 2 ** 16}
# work-item size of the batched kernel per order (a four-loop sample is ~1e5
# FP64 operations, a five-loop one ~1e6): at four loops 2048 samples give
# about 15 items per persistent block and round, so the blocks finish together
CHUNK = {1: 1 << 18, 2: 1 << 18, 3: 1 << 14, 4: 1 << 11, 5: 1 << 8}
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
    """The benchmarked set: every graph at one and two loops (mirror pairs
    both present, compiled integrands), one per mirror pair at three and
    four loops (bytecode integrands, mirror weights), the 64-graph five-loop
    workload (five_loop_subset.txt) at five.  At three loops the compiled
    integrands' double-double versions spill registers and ran the flagged
    points at 0.004 of the FP64 peak (59 of 63 s of a 1e8-sample step with 2 %
    flagged), while the interpreter's compacted double-double pass runs
    them at about 0.4."""
    if order == 5:
        from paper_1905_08007_b300.five_loop_subset import read
        every = q.enumerate_graphs(5)
        gs = [every[i] for i in read()]
        return gs, [1.0] * len(gs)
    if order in (3, 4):
        gs = q.enumerate_graphs(order, reduced=True)
        return gs, mirror_weights(gs)
    gs = q.enumerate_graphs(order)
    return gs, [1.0] * len(gs)


def _cpu_model():
    try:
        for ln in Path("/proc/cpuinfo").read_text().splitlines():
            if ln.startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def _oracle_job(job):
    """Oracle weights (numpy FP64, as it stands) for samples [begin, begin + n)
    of graph gi of the given order; returns the sample count."""
    order, gi, begin, n, seed = job
    from oracle.estimator import weights
    from oracle.graphs import enumerate_graphs
    from oracle.integrand import Integrand
    g = enumerate_graphs(order)[gi]
    if n == 0:
        return 0
    return int(weights(Integrand(g), g, gi, seed, begin, n).size)


# bounded oracle samples per order: (graph indices in the full enumeration,
# samples per graph).  Four loops: graph 85 (one forest term, the cheapest of
# the set; a typical four-loop graph costs the oracle many times more).
CPU_SAMPLE = {1: ([0], 3000), 2: (list(range(6)), 300), 3: (list(range(0, 50, 10)), 20), 4: ([85], 1)}


def cpu_baseline(order=4, seed=0):
    """The oracle as it stands on this host's cores, on a bounded sample of the
    same graph set: on one core in this process, then on every core (one
    spawned process per core, each on its own counters, the pool started and
    its imports done before the clock starts)."""
    import multiprocessing as mp
    if order not in CPU_SAMPLE:
        return None
    gis, n = CPU_SAMPLE[order]
    jobs = [(order, gi, 10**12, n, seed) for gi in gis]
    _oracle_job((order, gis[0], 0, 0, seed))
    t0 = time.perf_counter()
    tot = sum(_oracle_job(j) for j in jobs)
    dt1 = time.perf_counter() - t0
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_job, [(order, gis[0], 0, 0, seed)] * cores)
        jobs_all = [(order, gi, 10**12 + (k + 1) * 10**6, n, seed) for k in range(cores) for gi in gis]
        t0 = time.perf_counter()
        tot_all = sum(pool.map(_oracle_job, jobs_all, chunksize=1))
        dtn = time.perf_counter() - t0
    what = (f"{n} sample(s) of each of {len(gis)} {order}-loop graph(s) "
            f"{gis if len(gis) <= 6 else ''} (Philox counters from 1e12, seed {seed})")
    return {"value": tot_all / dtn, "unit": "samples/s", "cores": cores, "kind": "oracle",
            "cpu_model": _cpu_model(),
            "sample": f"{what}, once per core in parallel: {tot_all} samples in {dtn:.1f} s",
            "one_core": {"value": tot / dt1, "unit": "samples/s", "cores": 1,
                         "sample": f"{what}: {tot} samples in {dt1:.1f} s"},
            "note": "numpy FP64 oracle as it stands; a reported baseline, not a target"}


def compare_plain(diags, graphs, mw, ctx, S, seed, t_step, sigma_step, q):
    """The plain per-graph path on the same budget: untuned Eq. (1) densities
    (the Deg rule), equal samples per graph, one launch per graph; time to
    the target sigma against the batched, calibrated, tuned step."""
    plain = [ctx.load(g) for g in graphs]
    res = [d.integrate(S, seed=seed + 1, begin=1 << 41) for d in plain]
    t = sum(r.seconds for r in res)
    sig = math.sqrt(sum(w * w * r.variance for w, r in zip(mw, res)))
    st = SIGMA_TARGETS[graphs[0].n]
    tts_plain = t * (sig / st) ** 2
    tts_batch = t_step * (sigma_step / st) ** 2
    return {"seconds": t, "samples_per_s": S * len(graphs) / t, "sigma": sig,
            "total": sum(w * r.value for w, r in zip(mw, res)), "time_to_sigma": tts_plain,
            "kernel_seconds": sum(r.kernel_seconds for r in res),
            "speedup_time_to_sigma_batched_tuned_vs_plain": tts_plain / tts_batch,
            "note": ("a sigma is a reliable error bar where sigma sqrt(N) stays constant over a decade "
                     "of samples: at two loops on both paths; at three loops on the calibrated, tuned "
                     "path, not on the plain Deg-rule path (its weights are heavy-tailed); at four loops "
                     "on neither")}


def run_reference(args):
    """The CPU oracle as it stands on the same workload and metric: each step a
    bounded sample of the graph set (CPU_SAMPLE), fresh counters every step,
    on rank 0 only."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    if args.order not in CPU_SAMPLE:
        print(json.dumps({"impl": "reference", "unavailable": "the oracle needs hours per five-loop point"}))
        return 0
    gis, n = CPU_SAMPLE[args.order]

    def step(s):
        return sum(_oracle_job((args.order, gi, 10**12 + s * n, n, args.seed)) for gi in gis)
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
        "config": {"workload": f"{args.order}-loop lepton-loop-free vertex set, bounded sample: "
                               f"{n} sample(s) per step of each of graphs {gis}, Eq. (1) density, "
                               "forest-subtracted integrand, FP64 (the CPU oracle)",
                   "loops": args.order, "graphs": len(gis), "samples_per_graph_per_step": n, "seed": args.seed},
        "cpu_baseline": {"value": v, "unit": "samples/s", "cores": 1, "kind": "oracle", "cpu_model": _cpu_model(),
                         "sample": f"{n} sample(s) of each of graphs {gis} per step, {args.steps} steps"},
        "e2e": {"value": v, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def two_loop_pull(q, ctx, seed, samples=6e8, threshold=1e-6):
    """The six two-loop graphs, Deg-calibrated and tuned, 6e8 samples in the
    batched kernel: the set total against the two-loop closed form (on a
    context of its own: all six with their compiled integrands, whatever the
    benchmarked set's context prefers)."""
    from paper_1905_08007_b300.tune import tune
    ctx = q.Context(ctx.device, threshold=threshold)
    ds = [ctx.load(g) for g in q.enumerate_graphs(2)]
    for d in ds:
        d.calibrate_deg(n_base=8, seed=seed + 5)
        tune(d, steps=10, n=1 << 21, lr=0.08, seed=seed + 7)
    res = ctx.integrate_batch(ds, int(samples), seed=seed + 11, policy="variance", rounds=4, chunk=1 << 18,
                              counter_base=1 << 42)
    tot = sum(r.value for r in res)
    sig = math.sqrt(sum(r.variance for r in res))
    return {"value": tot, "sigma": sig, "closed_form": TWO_LOOP_TARGET, "pull": (tot - TWO_LOOP_TARGET) / sig,
            "samples": sum(r.n for r in res), "seconds": res[0].seconds}


def _traffic(kernel, order, seconds, launches):
    """DRAM bytes per launch of `kernel` from the committed ncu summary for this
    workload (profiles/<kernel>_<order>_loop_traffic.md), or None when there is
    none or the kernel's source has changed since it was taken."""
    import hashlib
    path = ROOT / "profiles" / f"{kernel}_{order}_loop_traffic.md"
    if not path.exists():
        return None
    vals = {}
    for ln in path.read_text().splitlines():
        if ":" in ln and ln.startswith("- "):
            k, v = ln[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    src = ROOT / "paper_1905_08007_b300" / "csrc" / vals.get("source", "")
    if not src.is_file() or hashlib.sha256(src.read_bytes()).hexdigest()[:16] != vals.get("source_sha256_16"):
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def run_native(args):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import paper_1905_08007_b300 as q
    from paper_1905_08007_b300.tune import tune
    # three loops: the bytecode programs (see graph_set)
    ctx = q.Context(local, threshold=args.threshold, rng=args.rng, prefer_programs=args.order == 3)
    stream = torch.cuda.current_stream()
    ctx.set_stream(stream)
    graphs, mw = graph_set(q, args.order)
    if args.graph_stride > 1:
        # a smaller case of the same workload (every k-th graph), for profiling
        graphs, mw = graphs[::args.graph_stride], mw[::args.graph_stride]
    if args.order == 5:
        # the five-loop programs are generated on request and may cover part
        # of the 64-graph workload: integrate the graphs that have one
        have = []
        for g, w in zip(graphs, mw):
            try:
                ctx.load(g).close()
                have.append((g, w))
            except q.QedError as e:
                if e.code != -6:
                    raise
        if not have:
            raise SystemExit("no five-loop programs built (python -m paper_1905_08007_b300.build --programs 2 3 4 5)")
        graphs, mw = [g for g, _ in have], [w for _, w in have]
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
        if args.calibrate and args.order <= 4:
            d.calibrate_deg(n_base=8, seed=args.seed + 5)
        if ts:
            tune(d, steps=ts, n=tn, lr=0.08, seed=args.seed + 7)
    autotuned = None
    # the autotuner's short batches are a few seconds at four loops; at five
    # loops (1e6 FP64 operations a sample, most points flagged) the default
    # shape and items of 256 samples are used
    if args.autotune and args.order == 4:
        from paper_1905_08007_b300.autotune import tune_batch_chunk, tune_vm
        small = max(1 << 19, 4 * len(diags) * CHUNK[args.order])
        best_vm, tab_vm = tune_vm(ctx, diags, samples=small, chunk=CHUNK[args.order])
        best_ch, tab_ch = tune_batch_chunk(ctx, diags, samples=small,
                                           chunks=(1 << 10, 1 << 11, 1 << 12))
        if args.chunk is None:
            args.chunk = best_ch["chunk"]
        autotuned = {"vm": best_vm, "chunk": best_ch, "vm_table": tab_vm, "chunk_table": tab_ch}
    setup_s = time.perf_counter() - t0
    flops = [d.flops_per_sample() for d in diags]
    ddflops = []
    for d in diags:
        try:
            ddflops.append(d.flops_per_dd_sample())
        except q.QedError:
            ddflops.append(None)
    # allocation rounds per step: round 0 equal, the others by running
    # variance; every round ends with the tail of its double-double pass,
    # so fewer, larger rounds waste less (three at four loops)
    rounds, chunk = args.rounds, int(args.chunk or CHUNK[args.order])

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
    launches, ksec, dsec, alg, algdd, nsamp = 0, 0.0, 0.0, 0.0, 0.0, 0
    wall0 = time.perf_counter()
    ev0.record(stream)
    for s in range(args.steps):
        flush.zero_()
        res = step(args.warmup + s)
        launches += res[0].launches
        ksec += res[0].kernel_seconds
        dsec += res[0].dd_seconds
        for i, r in enumerate(res):
            alg += flops[i] * r.n
            algdd += (ddflops[i] or 0.0) * r.n_flagged
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
        dist.all_gather_object(gathered, [(r.sum_w, r.sum_w2, r.n, r.n_flagged, r.n_unstable, r.unstable_abs_w)
                                          for r in acc])
        results = []
        for i in range(len(diags)):
            m = None
            for rk in range(ws):
                sw, sw2, n, nf, nu, uw = gathered[rk][i]
                r = q.Result(0.0, 0.0, tuple(sw), tuple(sw2), n, nf, nu, 0.0, unstable_abs_w=uw)
                m = r if m is None else q.merge_results(m, r)
            results.append(m)
    if rank != 0:
        return 0
    total_samples = ws * nsamp
    value = total_samples / tmax
    tot = sum(w * r.value for w, r in zip(mw, results))
    sigma = math.sqrt(sum(w * w * r.variance for w, r in zip(mw, results)))
    peak = fp64_peak / 1e12
    k64 = {"name": ("k_batch_fp64 (persistent FP64 integration kernel)" if args.order <= 2 else
                    f"k_batch_vm_fp64<{3 * args.order}> (persistent FP64 interpreter kernel, bytecode integrands)"),
           "seconds": ksec, "achieved": alg / ksec / 1e12, "frac": alg / ksec / 1e12 / peak,
           "flops": alg}
    kdd = {"name": ("k_batch_dd (double-double pass)" if args.order <= 2 else
                    f"k_batch_vm_dd<{3 * args.order}> (double-double interpreter pass)"),
           "seconds": dsec, "achieved": algdd / dsec / 1e12 if dsec > 0 else None,
           "frac": algdd / dsec / 1e12 / peak if dsec > 0 else None, "flops": algdd,
           "flops_counted": all(x is not None for x in ddflops)}
    dom = k64 if ksec >= dsec else kdd
    traffic = _traffic(dom["name"].split(" ")[0].split("<")[0], args.order, ksec if dom is k64 else dsec,
                       args.steps * rounds)
    n_items = max(len(diags), (total // rounds + chunk - 1) // chunk)
    flagged = sum(r.n_flagged for r in results)
    line = {
        "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tmax / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (Philox counters)",
        "config": {"workload": f"{args.order}-loop lepton-loop-free vertex set: {len(graphs)} graphs"
                               + {3: " (one per mirror pair, bytecode integrands)",
                                  4: " (one per mirror pair, bytecode integrands)",
                                  5: " of the 64-graph workload (those with generated programs, bytecode "
                                     "integrands)"}.get(args.order, "") + ", "
                               f"{total:.0e} Philox samples per step shared by running variance, "
                               + ("Deg-rule densities" if args.order == 5 else
                                  ("Deg-calibrated + gradient-tuned densities" if args.calibrate
                                   else "gradient-tuned Deg-rule densities"))
                               + f", forest-subtracted FP64 integrand, double-double re-evaluation above "
                               f"{args.threshold:g}, "
                               f"persistent batched kernel ({rounds} CUDA-graph rounds per step)",
                   "loops": args.order, "graphs": len(graphs), "samples_per_step": total, "seed": args.seed, "l2_flush": True,
                   "flag_threshold": args.threshold, "deg": "calibrated" if args.calibrate else "rule",
                   "rng": {"philox": "Philox4x32-10 (Calc 2)", "mrg32k3a": "MRG32k3a (Calc 1)"}[args.rng],
                   "launch": {"items_per_round": n_items, "chunk": chunk,
                              **({"vm_threads": ctx.vm_shape[0], "vm_points": ctx.vm_shape[1]} if args.order >= 3
                                 else {"threads": 256})},
                   "setup_seconds_calibrate_and_tune": setup_s, "autotune": autotuned},
        "set_total": {"loops": args.order, "value": tot, "sigma": sigma,
                           "closed_form": CLOSED_FORM.get(args.order),
                           "pull": ((tot - CLOSED_FORM[args.order]) / sigma
                                    if sigma > 0 and args.order in CLOSED_FORM else None),
                           "flagged_fraction": flagged / total_samples,
                           "unstable": sum(r.n_unstable for r in results),
                           # w := 0 at the unstable points; this is the most
                           # that can have shifted the set total
                           "unstable_abs_w_bound": sum(w * r.unstable_abs_w / r.n for w, r in zip(mw, results) if r.n),
                           "samples_per_graph": [r.n for r in results]},
        "time_to_sigma": {"target_sigma": SIGMA_TARGETS[args.order],
                          "seconds": tmax * (sigma / SIGMA_TARGETS[args.order]) ** 2,
                          "sigma_reached": sigma, "seconds_run": tmax},
        "roofline": {"bound": "alu", "achieved": dom["achieved"], "peak": peak, "unit": "TFLOP/s",
                     "frac": dom["frac"], "traffic": traffic,
                     "kernel": dom["name"],
                     "peak_source": "measured FP64 FMA throughput (qed_fp64_peak), of measured",
                     "kernels": {"fp64": k64, "dd": kdd},
                     "step": {"flops": alg + algdd, "seconds": tmax,
                              "achieved": (alg + algdd) / tmax / 1e12,
                              "frac": (alg + algdd) / tmax / 1e12 / peak,
                              "note": "whole step: both passes' algorithmic FP64 work (qed_diagram_flops "
                                      "per sample, qed_diagram_flops_dd per flagged sample) over the "
                                      "step's device time"},
                     "flops_per_sample_mean": sum(flops) / len(flops)},
        "gpu_launches": launches,
        "e2e": {"value": total_samples / wmax, "unit": "samples/s",
                "h2d_bytes_per_step": rounds * n_items * 16,
                "d2h_bytes_per_step": rounds * n_items * 96},
        "clocks": clk,
    }
    if args.order >= 4:
        # Table 1's columns per gauge-invariant class (k, m, n): value, N_diag
        # (mirror-reduced graphs), sum |a_j|, max |a_j|
        from paper_1905_08007_b300.classes import class_table
        line["set_total"]["classes"] = class_table(graphs, results, mw)
        line["set_total"]["max_abs_a_j"] = max(abs(w * r.value) for w, r in zip(mw, results))
        if args.order == 5:
            line["set_total"]["table1_max_abs_a_j"] = 85.8
    if ws == 1 and args.compare and args.order in (2, 3, 4):
        line["plain_per_graph"] = compare_plain(diags, graphs, mw, ctx, S, args.seed, tmax / args.steps, sigma, q)
    if ws == 1 and args.order != 2 and args.order <= 4:
        line["two_loop_total"] = two_loop_pull(q, ctx, args.seed, threshold=args.threshold)
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
    ap.add_argument("--order", type=int, default=4, choices=[1, 2, 3, 4, 5], help="loop order of the graph set")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--chunk", type=int, default=None, help="samples per work item of the batched kernel")
    ap.add_argument("--rounds", type=int, default=None,
                    help="allocation rounds per step (default 3 at four loops, else 4)")
    ap.add_argument("--threshold", type=float, default=1e-6,
                    help="relative rounding-error threshold above which a point is re-evaluated in "
                         "double-double: at four loops every accepted point was measured within 0.21 x the "
                         "threshold of its double-double value, far below any run's statistical error")
    ap.add_argument("--rng", default="philox", choices=["philox", "mrg32k3a"],
                    help="generator of the sample points (Sec. 3: Calc 2 used Philox4x32-10, Calc 1 MRG32k3a)")
    ap.add_argument("--graph-stride", type=int, default=1,
                    help="every k-th graph of the set only (a small case for ncu captures)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="keep the default interpreter launch shape and work-item size")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--calibrate", dest="calibrate", action="store_true", default=None,
                    help="cap Deg by the integrand's measured exponents (default up to three loops)")
    ap.add_argument("--no-calibrate", dest="calibrate", action="store_false",
                    help="the Deg rule without the calibration (default from four loops on: there "
                         "the calibrated densities were measured to have heavier tails than the rule)")
    ap.add_argument("--no-compare", dest="compare", action="store_false",
                    help="skip the plain vs batched-tuned time-to-sigma comparison")
    a = ap.parse_args(argv)
    if a.warmup < 3:
        a.warmup = 3
    if a.calibrate is None:
        a.calibrate = a.order <= 3
    if a.rounds is None:
        a.rounds = 3 if a.order == 4 else 4
    if a.impl == "reference":
        return run_reference(a)
    return run_native(a)


if __name__ == "__main__":
    sys.exit(main())
