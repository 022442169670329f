/*
 * qedmc -- C ABI of the B300 Monte Carlo integrator for the lepton-loop-free
 * QED vertex graphs of arXiv:1905.08007 (Volkov, 5-loop electron AMM).
 *
 * The paper states the problem as: each vertex graph G of order n contributes
 * one Feynman-parametric integral a_G of a pointwise-subtracted integrand, and
 * A_1^(2n) = sum_G a_G (Sec. 2, items 3-4); a_G is estimated by nonadaptive
 * Monte Carlo with the per-graph density of Eq. (1) (Sec. 2) on GPUs (Sec. 3).
 * This header exposes exactly that: load a graph (with its generated
 * integrand and its Deg-based density), then integrate it.
 *
 * Conventions shared by every call:
 *  - Return value: 0 = QED_OK, negative = error code below.  No call throws.
 *    qed_last_error() returns a thread-local message for the last failure.
 *  - Graph: n photons; photon a joins photon vertices pairs[2a] < pairs[2a+1]
 *    (vertices 0..2n-1 along the electron flow); the external photon vertex
 *    sits after the first e photon vertices.  Lines: electron lines 0..2n-1
 *    along the flow, then photons 2n..3n-1.
 *  - Random numbers: Philox4x32-10 (Sec. 3, Calc 2; MRG32k3a, Calc 1, with
 *    qed_ctx_set_rng), counter = (sample lo32,
 *    sample hi32, graph stream id, block), key = (seed lo32, seed hi32).
 *    Sample s uses draws 0..N-2 for the Hepp-sector walk and N-1..2N-3 for
 *    the radial variables, two draws per Philox block; draw = words (hi, lo)
 *    -> ((((hi << 32) | lo) >> 12) + 0.5) * 2^-52, strictly inside (0,1).  Results depend only
 *    on (seed, stream id, sample range, launch shape).
 *  - All pointers are owned by the caller unless stated otherwise; the
 *    library copies what it keeps.  Device pointers must be on the context's
 *    device.  Calls on one context are not thread-safe.
 */
#ifndef QEDMC_H
#define QEDMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QED_OK 0
#define QED_EINVAL (-1)            /* bad argument or unsupported graph */
#define QED_ENOMEM (-2)            /* device or host allocation failed */
#define QED_ECUDA (-3)             /* a CUDA runtime call failed */
#define QED_ETIMEOUT (-4)          /* reserved (no call waits on the device without bound) */
#define QED_EUNSTABLE_LIMIT (-5)   /* reserved */
#define QED_ENOTFOUND (-6)         /* no generated integrand for this graph */

#define QED_MAX_LOOPS 5

typedef struct qed_ctx qed_ctx;
typedef struct qed_diag qed_diag;

/* A vertex graph with no closed lepton loop, the set Sec. 3 computes (mirror
 * images are distinct graphs here).  stream_id is the third Philox counter
 * word used for this graph's samples. */
typedef struct {
  int n;                          /* loops = internal photons, 1..QED_MAX_LOOPS */
  int pairs[2 * QED_MAX_LOOPS];   /* photon a: vertices pairs[2a] < pairs[2a+1] */
  int e;                          /* external vertex after e photon vertices */
  uint32_t stream_id;
} qed_graph;

/* Density of Eq. (1).  If deg != NULL it holds Deg(s) for every subset s of
 * the N = 3n lines as a bitmask-indexed array of 2^N doubles (entries 0 and
 * 2^N-1 unused); all used entries must be > 0 (else QED_EINVAL).  If deg is
 * NULL the library builds Deg(s) = -omega(I-closure(s)) / 2 when positive,
 * else c_div, floored at d_min (Sec. 2: Deg from omega of I-closures,
 * sometimes fractional and below 1; omega counts momentum powers, and a
 * Feynman parameter scales like the inverse square of its line's momentum,
 * so the integrand's exponent in the parameters is half of it). */
typedef struct {
  const double *deg;
  double c_div;                   /* default 0.5 when <= 0 */
  double d_min;                   /* default 0.05 when <= 0 */
} qed_pdf;

/* Per-graph Monte Carlo result in units of (alpha/pi)^n (Sec. 3). */
typedef struct {
  double value;                   /* mean of f/p */
  double variance;                /* variance of the mean */
  double sum_w[2];                /* sum of w = f/p as a double-double (hi, lo) */
  double sum_w2[2];               /* sum of w^2 as a double-double */
  uint64_t n;                     /* samples */
  uint64_t n_flagged;             /* points re-evaluated in double-double */
  uint64_t n_unstable;            /* points unstable in double-double: w := 0
                                     (see unstable_abs_w) */
  double seconds;                 /* device time of the call (all kernels) */
  double kernel_seconds;          /* device time of the FP64 integration kernel */
  uint32_t launches;              /* kernels launched by the call */
  double dd_seconds;              /* device time of the double-double kernels */
  double unstable_abs_w;          /* sum of |w| over the unstable points (their
                                     double-double value where finite): what
                                     setting them to 0 can have removed from
                                     sum_w, for context */
} qed_result;

/* ---- context ------------------------------------------------------------ */
/* Context flag: graphs loaded on this context use a registered bytecode
 * program (qed_programs_load) even where a compiled integrand exists (used to
 * compare the two paths on the same graph). */
#define QED_CTX_PREFER_PROGRAMS 1u
/* Create a context on CUDA device `device`.  flags: 0 or
 * QED_CTX_PREFER_PROGRAMS (other bits: QED_EINVAL).  The context owns every
 * device buffer it allocates. */
int qed_ctx_create(int device, uint64_t flags, qed_ctx **out);
int qed_ctx_destroy(qed_ctx *ctx);
/* Launch subsequent work on this cudaStream_t (0 = legacy default stream). */
int qed_ctx_set_stream(qed_ctx *ctx, uintptr_t stream);
/* Launch shape of the integration kernels: threads per block (multiple of 32,
 * 32..256) and blocks (0 = 4 x the SM count).  Results depend on it through
 * the summation order only. */
int qed_ctx_set_launch(qed_ctx *ctx, int threads_per_block, int blocks);
/* Launch shape of the interpreter kernels (bytecode integrands): threads per
 * block of the FP64 kernels (multiple of 32, 32..256; halved while the
 * shared-memory frame does not fit) and points evaluated per thread by one
 * instruction stream (1 or 2).  Defaults 128 and 1.  Results depend on it
 * through the summation order only. */
int qed_ctx_set_vm(qed_ctx *ctx, int threads_per_block, int points_per_thread);
/* Relative rounding-error threshold above which a point is re-evaluated in
 * double-double (Sec. 3: arithmetics of different precisions).  Default 1e-8
 * (per-point errors far below the statistical error of any run); 1e-12 makes
 * every accepted FP64 value accurate to 1e-12.  The estimate is
 * 8 ulp x (sum of the absolute values of the integrand's monomials) / |f|; the
 * double-double result is accepted under the same rule with its own ulp. */
int qed_ctx_set_threshold(qed_ctx *ctx, double rel_err);
/* Generator of the sample points (Sec. 3 integrates with two generators of
 * the CURAND library as an independent check: MRG32k3a in Calc 1,
 * Philox4x32-10 in Calc 2).  QED_RNG_PHILOX (default): the Philox layout of
 * the conventions above.  QED_RNG_MRG32K3A: L'Ecuyer's MRG32k3a started from
 * the state with all six words 12345; sample s of a graph with stream id g
 * under seed k takes its draws 0..2N-3 from positions
 * k * 2^127 + g * 2^96 + s * 2^5 + d of that sequence (32 draws per sample,
 * jumps by matrix powers), u = z / (m1 + 1) computed as z times the double
 * nearest 1 / (m1 + 1) (32 random bits).  Applies to every later launch on
 * the context; results depend on (generator, seed, stream id, sample range,
 * launch shape) as above.  Other values: QED_EINVAL. */
#define QED_RNG_PHILOX 0
#define QED_RNG_MRG32K3A 1
int qed_ctx_set_rng(qed_ctx *ctx, int rng);
/* Which points the double-double pass re-evaluates (Sec. 3: the round-off
 * of the numerical subtraction is removed with interval arithmetic of
 * different precisions).
 * QED_FLAG_ESTIMATE (default): the FP64 value with its rounding-error
 * estimate (qed_ctx_set_threshold).
 * QED_FLAG_INTERVAL: every point is evaluated in FP64 interval arithmetic
 * (each operation rounds the lower end down and the upper end up, so the
 * interval encloses the exact value of the program's arithmetic); the
 * midpoint is accepted when both ends have one sign and
 * hi - lo <= 2 threshold min(|lo|, |hi|), a rigorous bound of its relative
 * error by the threshold; other points are re-evaluated in double-double
 * (accepted there by the estimate).  Bytecode programs only: on this rule
 * qed_integrate / qed_integrate_range of a graph with a compiled integrand,
 * qed_integrate_batch and qed_integrate_range_noalloc give QED_EINVAL (load
 * the graph on a QED_CTX_PREFER_PROGRAMS context to use its program);
 * qed_pdf_grad and qed_dump_points keep the estimate.  Other values:
 * QED_EINVAL. */
#define QED_FLAG_ESTIMATE 0
#define QED_FLAG_INTERVAL 1
int qed_ctx_set_flag_rule(qed_ctx *ctx, int rule);
const char *qed_last_error(void);

/* ---- graphs ------------------------------------------------------------- */
/* Enumerate the graphs of order n (Sec. 3, Table 1 counts): all of them
 * (reduced = 0) or one per mirror pair (reduced = 1, the lexicographically
 * smaller key).  Writes min(count, cap) graphs to out (may be NULL when
 * cap = 0) and the total to *count.  stream_id = index in the list. */
int qed_enumerate(int n, int reduced, qed_graph *out, int cap, int *count);
/* Gauge-invariant class (k, m, n) of Table 1: photons spanning X, photons on
 * the larger and on the smaller side of X. */
int qed_gauge_class(const qed_graph *g, int kmn[3]);

/* Register bytecode integrands with the context.  Sec. 2 makes every graph's
 * contribution one parametric integral of a generated, forest-subtracted
 * integrand; Sec. 3 notes that the generated code for the 5-loop set reaches
 * 500 GB.  From four loops on, the generator therefore writes each
 * integrand as a program for the library's interpreter kernels instead of
 * source to compile.  data/bytes: the contents of a program file written by
 * the generator (vm_n<n>.bin: "QEDVM004", count, then per program its graph
 * name, line count, register count, 64-bit instructions and constants), in
 * host memory, owned by the caller and copied to the device.  Every
 * instruction is checked against its program's register and constant counts
 * (QED_EINVAL on any violation, nothing registered); *count (may be NULL)
 * receives the number of programs added. */
int qed_programs_load(qed_ctx *ctx, const void *data, size_t bytes, int *count);

/* Load a graph: validate it (lepton-loop free, one-particle irreducible, no
 * self-energy on an external leg), select its integrand -- the compiled one,
 * else a registered bytecode program of the same graph (always the program
 * on a QED_CTX_PREFER_PROGRAMS context) -- and build and upload the Eq. (1)
 * tables.  QED_ENOTFOUND if neither exists for this graph. */
int qed_diagram_load(qed_ctx *ctx, const qed_graph *g, const qed_pdf *pdf, qed_diag **out);
int qed_diagram_free(qed_diag *d);
/* N = 3n lines, integrand id (compiled: 0..count-1; bytecode program:
 * count + its registration index), log of the Eq. (1) normaliser F(E). */
int qed_diagram_info(const qed_diag *d, int *n_lines, int *integrand_id, double *log_norm);

/* ---- integration (Sec. 2 nonadaptive MC, Sec. 3) ------------------------- */
/* Estimate a_G from samples [0, n_samples). */
int qed_integrate(qed_diag *d, uint64_t n_samples, uint64_t seed, qed_result *out);
/* Same over samples [begin, begin + n): disjoint ranges give independent
 * replicas whose moments merge exactly (resume, multi-process). */
int qed_integrate_range(qed_diag *d, uint64_t begin, uint64_t n, uint64_t seed, qed_result *out);

/* Parity mode: for samples [begin, begin + n) write, into caller-owned DEVICE
 * buffers, the point z (n x N doubles, row-major, largest component 1), the
 * integrand f (FP64 path), log p(z) of Eq. (1) and a flag byte (bit 0: the
 * rounding-error estimate exceeded the threshold; bit 1: non-finite). */
int qed_dump_points(qed_diag *d, uint64_t begin, uint64_t n, uint64_t seed,
                    double *z_dev, double *f_dev, double *logp_dev, uint8_t *flag_dev);
/* Evaluate the integrand at caller-supplied DEVICE points z (n x N) in FP64
 * (prec = 0) or double-double (prec = 1, result rounded to double). */
int qed_eval_points(qed_diag *d, const double *z_dev, uint64_t n, int prec, double *f_dev);

/* FP64 interval arithmetic at caller-supplied DEVICE points z (n x N):
 * lo_dev[i] <= (exact value of the program's arithmetic at z_i) <= hi_dev[i]
 * (Sec. 3, interval arithmetic; see QED_FLAG_INTERVAL).  The program's
 * constants are the FP64 roundings of the generated coefficients, so the
 * exact integrand can differ from the enclosed value by that rounding (a
 * few ulp of the sum of the absolute values of the monomials).  An interval
 * that lost every digit comes back as [-inf, inf] or with NaN ends.
 * lo_dev, hi_dev: n doubles each, caller-owned device buffers (may be NULL
 * when n = 0).  Runs on the context's stream and returns after it
 * completed.  Bytecode programs only (QED_EINVAL for a compiled integrand). */
int qed_eval_interval(qed_diag *d, const double *z_dev, uint64_t n, double *lo_dev, double *hi_dev);

/* ---- tunable density and the adjoint of the second moment --------------- */
/* Set the density's parameters theta (Sec. 2 builds the density from Deg;
 * the paper's version is nonadaptive, these parameters only reshape it):
 * Deg_theta(S) = max(d_min, Deg(S) + sum_{l in S} alpha[l]) and the first
 * walk step weighted by exp(beta[j]).  alpha, beta: N doubles each (NULL =
 * zeros).  The estimator stays unbiased for any finite theta. */
int qed_diagram_set_pdf_params(qed_diag *d, const double *alpha, const double *beta);
/* Adjoint of M2 = E_p[(f/p)^2], the second moment that sets the variance,
 * over samples [begin, begin + n) recomputed from their Philox counters:
 * *m2 = estimate of M2, grad[0..N-1] = dM2/dalpha, grad[N..2N-1] =
 * dM2/dbeta (score-function form -E_p[w^2 d log p / d theta]; d log Z /
 * d theta from a reverse pass over the F recursion on the host).  The
 * weights follow the estimator's rule: a point whose FP64 rounding-error
 * estimate exceeds the context threshold enters with its double-double
 * value, and with w = 0 if it fails there too.  Launches cover at most
 * 2^22 samples each (the flagged queue's capacity); allocates one small
 * device buffer for the duration of the call. */
int qed_pdf_grad(qed_diag *d, uint64_t begin, uint64_t n, uint64_t seed, double *m2, double *grad);

/* Calibrate Deg on the integrand itself (Sec. 2 gives the Deg rule as a
 * heuristic without a complete proof, lowered for infrared limits).  For
 * every proper subset s the growth exponent a_s of the integrand under
 * z_s -> eps z_s is measured on the GPU in double-double at n_base random
 * points (eps = 1e-6 and 1e-8, past the bumps of nearby scales) and Deg(s)
 * is capped at |s| - a_s (a_s: |f| grows like eps^-a_s), where w = f/p stays
 * bounded in that limit and the variance finite:
 * Deg(s) = max(d_min, min(Deg(s), |s| - a_s)).
 * Allocates two small device buffers for the duration of the call. */
int qed_diagram_calibrate_deg(qed_diag *d, int n_base, uint64_t seed);
/* The current Deg table (2^N doubles, bitmask-indexed). */
int qed_diagram_get_deg(const qed_diag *d, double *deg_out);

/* ---- batched integration of a graph set --------------------------------- */
/* Options of qed_integrate_batch.  Zero-initialised fields take defaults. */
typedef struct {
  int policy;          /* 0 = variance-driven (Neyman: N_g ~ sigma_g / sqrt(cost_g)), 1 = equal */
  int rounds;          /* allocation rounds (default 4); round 0 is equal */
  uint64_t chunk;      /* samples per work item (default 262144, <= 2^31) */
  int use_graph;       /* 0 = default: capture one round as a CUDA graph and replay it; -1 = plain launches */
  int list_div;        /* flagged-list capacity per item = chunk / list_div (default 16) */
  uint64_t counter_base; /* first Philox counter of every graph's samples (default 0) */
} qed_batch_opts;

/* Integrate the k graphs d[0..k-1] (all loaded on the same context; all
 * with compiled integrands, or all with bytecode programs of one loop order,
 * else QED_EINVAL) with
 * total_samples samples in all, in one persistent launch per round: blocks
 * take (graph, counter-block) work items from a device queue, so graphs of
 * different cost share the GPU; the queue holds the items of the costliest
 * graphs first, so the blocks finish a round close together (the order
 * changes neither a graph's samples nor the order its items are folded
 * in).  After round r the samples of round r+1 are
 * split by the running per-sample variance and the cost model (FP64 ops per
 * sample, qed_diagram_flops, weighted by the flagged fraction).  Every graph's
 * samples are consecutive counters from 0, so a result depends only on
 * (seed, graphs, total, options).  out_k[g] receives graph g's result
 * (seconds and launches of the whole call on every entry). */
int qed_integrate_batch(qed_ctx *ctx, qed_diag *const *d, int k, uint64_t total_samples, uint64_t seed,
                        const qed_batch_opts *opts, qed_result *out_k);

/* Merge replica results over disjoint sample ranges: the raw moments add in
 * double-double, so the merge is exact and order-fixed: out = a (+) b. */
int qed_result_merge(const qed_result *a, const qed_result *b, qed_result *out);

/* ---- measurement -------------------------------------------------------- */
/* FP64 arithmetic operations (add, sub, mul, div; transcendental functions
 * counted once each) per sample of this graph's hot path: sampler, integrand
 * and accumulation.  Used as the algorithmic work of the roofline. */
int qed_diagram_flops(const qed_diag *d, double *flops_per_sample);
/* FP64 operations (an FMA counts 2) per sample re-evaluated in double-double:
 * the sampler as above plus the integrand in the interpreter's
 * double-double arithmetic, counted instruction by instruction over the
 * graph's bytecode program (for a graph with a compiled integrand, the
 * program of the same graph; QED_ENOTFOUND if none is registered).  With
 * qed_diagram_flops it gives the algorithmic FP64 work of a whole step, both
 * passes included. */
int qed_diagram_flops_dd(const qed_diag *d, double *flops_per_sample);
/* Measured FP64 fused-multiply-add throughput of the device (FLOP/s, 2 per
 * FMA): every SM runs independent FMA chains for about `ms` milliseconds. */
int qed_fp64_peak(int device, double ms, double *flops_per_s);

/* ---- integration without allocation -------------------------------------
 * No counterpart in the paper.  Same estimate as qed_integrate_range (equal
 * within rounding: the block partials are folded on the device), for callers
 * that must not allocate device memory once they are running -- an
 * application whose own pool allocator owns all device memory and forbids
 * further cudaMalloc, or a latency-critical loop where an allocation, which
 * can synchronise the device, is not acceptable.  The call allocates nothing
 * on the device or the host: its scratch is one file-scope device array of
 * 753,736 bytes (about 736 KiB) per GPU.  The GPU takes that memory when the
 * library's device code is loaded on it: under CUDA's default lazy module
 * loading that is the first use of the library's device code on that
 * device (this call's address lookup, or any other call that launches a
 * kernel), so make one such call, or run with CUDA_MODULE_LOADING=EAGER,
 * before handing the remaining device memory to a pool.  The memory is held
 * until the process exits.  The first call on a device looks up the array's
 * device address (with the device current) and keeps it for the process:
 * make that first call before any stream capture, and do not use the
 * library on a device after cudaDeviceReset in the same process.
 * Limits: at most 2048 blocks in the context's launch shape (QED_EINVAL
 * otherwise); when more than 65536 points of a chunk of 2^30 samples are
 * flagged, the double-double kernel re-scans the whole chunk and that pass
 * replaces the first (each point is flagged or accepted by one decision).
 * All calls in the process share the array, so calls that overlap on the
 * GPU (other threads, other streams) race: serialise them.  Each call clears
 * the counters it needs before use.  kernel_seconds is the FP64 integration
 * kernel's device time, as for qed_integrate_range.  Compiled integrands
 * only: a graph that uses a bytecode program gives QED_EINVAL. */
int qed_integrate_range_noalloc(qed_diag *d, uint64_t begin, uint64_t n, uint64_t seed, qed_result *out);

#ifdef __cplusplus
}
#endif
#endif /* QEDMC_H */
