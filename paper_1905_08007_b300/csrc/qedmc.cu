// qedmc: B300 (sm_103a) Monte Carlo integrator for the subtracted
// Feynman-parametric integrands of lepton-loop-free QED vertex graphs
// (arXiv:1905.08007, Sec. 2 and Sec. 3).  C ABI in include/qedmc.h.
//
// Hot path, one thread per sample, per launch:
//   Philox4x32-10 draws (Sec. 3, Calc 2)
//   -> Hepp-sector walk and radial variables of the Eq. (1) density
//   -> generated FP64 integrand (forest-like subtraction, Sec. 2)
//   -> rounding-error estimate; flagged points are queued for a
//      double-double re-evaluation kernel (Sec. 3: arithmetics of different
//      precisions)
//   -> w = f / p accumulated per thread with Neumaier compensation, reduced
//      with warp shuffles and shared memory to one double-double partial per
//      block; the host folds the partials in a fixed order.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "qedmc.h"
#include "qed_graph.hpp"
#include "qed_kernels.cuh"
#include "qed_batch.cuh"
#include "qed_vm.cuh"
#include "qed_registry.h"

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;
static int set_err(int code, const std::string &msg) { g_err = msg; return code; }
#define CUDA_TRY(x)                                                                     \
  do {                                                                                  \
    cudaError_t e_ = (x);                                                               \
    if (e_ != cudaSuccess) return set_err(QED_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

extern "C" const char *qed_last_error(void) { return g_err.c_str(); }

// ---------------------------------------------------------------------------
// MRG32k3a jump-ahead on the host (L'Ecuyer 1999; L'Ecuyer, Simard, Chen,
// Kelton 2002 for jumps by matrix powers): the one-step matrices of both
// recurrences, their powers A^(2^k) for k = 0..190 by repeated squaring
// (exact products in 128-bit integers), the start state of a (seed, stream)
// at position seed * 2^127 + stream * 2^96 from the all-12345 state, and
// the device table of A^(2^(5+k)), k = 0..63, the jumps by sample index.
// ---------------------------------------------------------------------------
namespace mrg {
constexpr uint64_t M1 = 4294967087ull, M2 = 4294944443ull;
struct Mat { uint64_t a[9]; };
static Mat mul(const Mat &x, const Mat &y, uint64_t m) {
  Mat r;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      unsigned __int128 acc = 0;
      for (int k = 0; k < 3; ++k) acc += (unsigned __int128)x.a[3 * i + k] * y.a[3 * k + j];
      r.a[3 * i + j] = uint64_t(acc % m);
    }
  return r;
}
static void apply(const Mat &x, uint64_t (&v)[3], uint64_t m) {
  uint64_t r[3];
  for (int i = 0; i < 3; ++i) {
    unsigned __int128 acc = 0;
    for (int k = 0; k < 3; ++k) acc += (unsigned __int128)x.a[3 * i + k] * v[k];
    r[i] = uint64_t(acc % m);
  }
  for (int i = 0; i < 3; ++i) v[i] = r[i];
}
// powers()[c][k] = A_c^(2^k), c = 0 (x1, mod m1) or 1 (x2, mod m2)
static const std::vector<Mat> *powers() {
  static const std::vector<Mat> *P = [] {
    auto *t = new std::vector<Mat>[2];
    const Mat a1 = {{0, 1, 0, 0, 0, 1, M1 - 810728ull, 1403580ull, 0}};
    const Mat a2 = {{0, 1, 0, 0, 0, 1, M2 - 1370589ull, 0, 527612ull}};
    t[0].push_back(a1);
    t[1].push_back(a2);
    for (int k = 1; k < 191; ++k) {
      t[0].push_back(mul(t[0].back(), t[0].back(), M1));
      t[1].push_back(mul(t[1].back(), t[1].back(), M2));
    }
    return t;
  }();
  return P;
}
static void stream_start(uint64_t seed, uint32_t stream, uint32_t out[6]) {
  const std::vector<Mat> *P = powers();
  uint64_t v1[3] = {12345, 12345, 12345}, v2[3] = {12345, 12345, 12345};
  for (int j = 0; j < 64; ++j)
    if (seed >> j & 1) { apply(P[0][127 + j], v1, M1); apply(P[1][127 + j], v2, M2); }
  for (int j = 0; j < 32; ++j)
    if (stream >> j & 1) { apply(P[0][96 + j], v1, M1); apply(P[1][96 + j], v2, M2); }
  for (int i = 0; i < 3; ++i) { out[i] = uint32_t(v1[i]); out[3 + i] = uint32_t(v2[i]); }
}
static std::vector<uint32_t> jump_table() {
  const std::vector<Mat> *P = powers();
  std::vector<uint32_t> t(64 * 18);
  for (int k = 0; k < 64; ++k)
    for (int i = 0; i < 9; ++i) {
      t[18 * k + i] = uint32_t(P[0][5 + k].a[i]);
      t[18 * k + 9 + i] = uint32_t(P[1][5 + k].a[i]);
    }
  return t;
}
// sample indices below 2^bits cover [0, end)
static uint32_t index_bits(uint64_t end) {
  return end <= 1 ? 1u : uint32_t(64 - __builtin_clzll(end - 1));
}
}  // namespace mrg

// ---------------------------------------------------------------------------
// kernel tables (one translation unit per generated graph defines qed_kset_<id>)
// ---------------------------------------------------------------------------
#define QED_DECL_KSET(id, lines) extern const KernelSet qed_kset_##id;
QED_GENERATED_LIST(QED_DECL_KSET)
#define QED_REF_KSET(id, lines) &qed_kset_##id,
static const KernelSet *const g_kernels[] = {QED_GENERATED_LIST(QED_REF_KSET)};
// persistent batched kernels (defined in the generated batch translation unit)
extern const void *const qed_batch_kernels[2];
// bytecode path: one kernel set per line count N = 3n and points per thread
// P of the FP64 kernels (1 or 2)
static const VmKernelSet g_vm_kernels[2][QED_MAX_LOOPS] = {
    {QED_VM_KSET(3, 1), QED_VM_KSET(6, 1), QED_VM_KSET(9, 1), QED_VM_KSET(12, 1), QED_VM_KSET(15, 1)},
    {QED_VM_KSET(3, 2), QED_VM_KSET(6, 2), QED_VM_KSET(9, 2), QED_VM_KSET(12, 2), QED_VM_KSET(15, 2)}};

// ---------------------------------------------------------------------------
// host objects
// ---------------------------------------------------------------------------
struct qed_ctx {
  int device = 0;
  cudaStream_t stream = 0;
  int threads = 256;
  int blocks = 0;            // 0 = 4 x SMs
  int sms = 148;
  double thresh = 1e-8;
  // scratch owned by the context
  double *partials = nullptr;
  unsigned long long *counts = nullptr;
  unsigned long long *queue = nullptr;
  unsigned int *queue_len = nullptr;
  unsigned int queue_cap = 1u << 22;
  int partial_cap = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, evk0 = nullptr, evk1 = nullptr, evk2 = nullptr;
  std::vector<double> h_partials;
  std::vector<unsigned long long> h_counts;
  // bytecode integrands registered by qed_programs_load
  struct VmProg {
    std::string name;
    int n_lines, n_regs, n_ins, n_kon;
    double flops;
    double dd_flops;        // FP64 operations of one double-double evaluation
    const uint2 *d_ins;
    const double *d_kon;
  };
  std::vector<VmProg> vm;
  std::vector<void *> vm_bufs;
  bool prefer_vm = false;
  struct BatchPlan *plan = nullptr;   // qed_integrate_batch's cached set-up
  int vm_threads = 128;      // threads per block of the FP64 interpreter kernels
  int vm_points = 1;         // points per thread of the FP64 interpreter kernels
  int flag_rule = QED_FLAG_ESTIMATE;   // which points go to the double-double pass
  int rng = QED_RNG_PHILOX;  // generator of the sample points
  uint32_t *mrg_jump = nullptr;   // MRG32k3a jump table on the device
};

struct qed_diag {
  qed_ctx *ctx = nullptr;
  qed::Graph g;
  uint32_t stream_id = 0;
  int fid = -1;
  int vm = -1;                       // index of the bytecode program (fid = -1), or -1
  int N = 0;
  double logZ = 0.0;
  double d_min = 0.05;
  std::vector<double> deg0;          // Deg(S) before the tunable shifts
  std::vector<double> alpha, beta;   // per-line Deg shifts, first-level sector weights
  std::vector<double> deg, F;        // current Deg_theta and F tables
  std::vector<uint8_t> act;          // Deg_theta(S) not clamped at d_min
  double *d_tab = nullptr;           // F, G, 1/Deg (3 x 2^N), then N first-line offsets
  uint8_t *d_act = nullptr;          // 2^N activity flags (adjoint kernel)
};

// Deg_theta(S) = max(d_min, Deg0(S) + sum_{l in S} alpha_l); the first walk
// step picks line j with weight e^{beta_j} F(E\j) / Deg(E\j), so
// Z = sum_j e^{beta_j} F(E\j) / Deg(E\j) and log p gains beta_{j_1} - log Z.
static int rebuild_tables(qed_diag *d) {
  const int N = d->N;
  const size_t M = size_t(1) << N;
  d->deg.assign(M, 0.0);
  d->act.assign(M, 0);
  for (size_t m = 1; m + 1 < M; ++m) {
    double v = d->deg0[m];
    for (int l = 0; l < N; ++l) if (m >> l & 1) v += d->alpha[l];
    if (v > d->d_min) { d->deg[m] = v; d->act[m] = 1; }
    else d->deg[m] = d->d_min;
    if (!std::isfinite(d->deg[m])) return set_err(QED_EINVAL, "Deg not finite");
  }
  d->F.assign(M, 0.0);
  std::vector<double> G(M, 0.0), inv(M, 0.0), off(N, 0.0);
  for (size_t m = 1; m + 1 < M; ++m) {
    if (__builtin_popcountll(m) == 1) { d->F[m] = 1.0; continue; }
    double acc = 0.0;
    for (int j = 0; j < N; ++j) if (m >> j & 1) { size_t r = m & ~(size_t(1) << j); acc += d->F[r] / d->deg[r]; }
    d->F[m] = acc;
  }
  for (size_t m = 1; m + 1 < M; ++m) { G[m] = d->F[m] / d->deg[m]; inv[m] = 1.0 / d->deg[m]; }
  double Z = 0.0;
  for (int j = 0; j < N; ++j) {
    const size_t r = (M - 1) & ~(size_t(1) << j);
    G[r] *= std::exp(d->beta[j]);
    Z += G[r];
  }
  std::vector<double> Ft = d->F;
  Ft[M - 1] = Z;
  d->F[M - 1] = Z;
  d->logZ = std::log(Z);
  for (int j = 0; j < N; ++j) off[j] = d->beta[j] - d->logZ;
  CUDA_TRY(cudaSetDevice(d->ctx->device));
  CUDA_TRY(cudaMemcpy(d->d_tab, Ft.data(), M * sizeof(double), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(d->d_tab + M, G.data(), M * sizeof(double), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(d->d_tab + 2 * M, inv.data(), M * sizeof(double), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(d->d_tab + 3 * M, off.data(), N * sizeof(double), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(d->d_act, d->act.data(), M, cudaMemcpyHostToDevice));
  return QED_OK;
}

static size_t table_smem(int N) { return (3 * (size_t(1) << N) + size_t(N)) * sizeof(double); }

static int ensure_scratch(qed_ctx *c, int blocks) {
  if (blocks <= c->partial_cap) return QED_OK;
  if (c->partials) cudaFree(c->partials);
  if (c->counts) cudaFree(c->counts);
  c->partials = nullptr; c->counts = nullptr;
  CUDA_TRY(cudaMalloc(&c->partials, size_t(blocks) * QED_PART * sizeof(double)));
  CUDA_TRY(cudaMalloc(&c->counts, size_t(blocks) * 2 * sizeof(unsigned long long)));
  c->partial_cap = blocks;
  c->h_partials.resize(size_t(blocks) * QED_PART);
  c->h_counts.resize(size_t(blocks) * 2);
  return QED_OK;
}

extern "C" int qed_ctx_create(int device, uint64_t flags, qed_ctx **out) {
  if (!out) return set_err(QED_EINVAL, "out is NULL");
  if (flags & ~uint64_t(QED_CTX_PREFER_PROGRAMS)) return set_err(QED_EINVAL, "unknown context flags");
  int ndev = 0;
  CUDA_TRY(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return set_err(QED_EINVAL, "no such device");
  CUDA_TRY(cudaSetDevice(device));
  qed_ctx *c = new qed_ctx();
  c->device = device;
  c->prefer_vm = (flags & QED_CTX_PREFER_PROGRAMS) != 0;
  cudaDeviceProp prop;
  CUDA_TRY(cudaGetDeviceProperties(&prop, device));
  c->sms = prop.multiProcessorCount;
  CUDA_TRY(cudaMalloc(&c->queue, size_t(c->queue_cap) * sizeof(unsigned long long)));
  CUDA_TRY(cudaMalloc(&c->queue_len, sizeof(unsigned int)));
  CUDA_TRY(cudaEventCreate(&c->ev0));
  CUDA_TRY(cudaEventCreate(&c->ev1));
  CUDA_TRY(cudaEventCreate(&c->evk0));
  CUDA_TRY(cudaEventCreate(&c->evk1));
  CUDA_TRY(cudaEventCreate(&c->evk2));
  int rc = ensure_scratch(c, 8 * c->sms);
  if (rc) return rc;
  const std::vector<uint32_t> jt = mrg::jump_table();
  CUDA_TRY(cudaMalloc(&c->mrg_jump, jt.size() * sizeof(uint32_t)));
  CUDA_TRY(cudaMemcpy(c->mrg_jump, jt.data(), jt.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
  *out = c;
  return QED_OK;
}

static void drop_plan(qed_ctx *c);
extern "C" int qed_ctx_destroy(qed_ctx *c) {
  if (!c) return QED_OK;
  cudaSetDevice(c->device);
  drop_plan(c);
  if (c->partials) cudaFree(c->partials);
  if (c->counts) cudaFree(c->counts);
  if (c->queue) cudaFree(c->queue);
  if (c->queue_len) cudaFree(c->queue_len);
  if (c->mrg_jump) cudaFree(c->mrg_jump);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->evk0) cudaEventDestroy(c->evk0);
  if (c->evk1) cudaEventDestroy(c->evk1);
  if (c->evk2) cudaEventDestroy(c->evk2);
  for (void *p : c->vm_bufs) cudaFree(p);
  delete c;
  return QED_OK;
}

extern "C" int qed_ctx_set_stream(qed_ctx *c, uintptr_t stream) {
  if (!c) return set_err(QED_EINVAL, "ctx is NULL");
  c->stream = reinterpret_cast<cudaStream_t>(stream);
  return QED_OK;
}

extern "C" int qed_ctx_set_launch(qed_ctx *c, int threads, int blocks) {
  if (!c) return set_err(QED_EINVAL, "ctx is NULL");
  if (threads < 32 || threads > 256 || threads % 32) return set_err(QED_EINVAL, "threads per block must be a multiple of 32 in [32, 256]");
  if (blocks < 0 || blocks > 1 << 20) return set_err(QED_EINVAL, "blocks out of range");
  c->threads = threads;
  c->blocks = blocks;
  return QED_OK;
}

extern "C" int qed_ctx_set_vm(qed_ctx *c, int threads, int points) {
  if (!c) return set_err(QED_EINVAL, "ctx is NULL");
  if (threads < 32 || threads > 256 || threads % 32) return set_err(QED_EINVAL, "threads per block must be a multiple of 32 in [32, 256]");
  if (points != 1 && points != 2) return set_err(QED_EINVAL, "points per thread must be 1 or 2");
  c->vm_threads = threads;
  c->vm_points = points;
  return QED_OK;
}

extern "C" int qed_ctx_set_rng(qed_ctx *c, int rng) {
  if (!c) return set_err(QED_EINVAL, "ctx is NULL");
  if (rng != QED_RNG_PHILOX && rng != QED_RNG_MRG32K3A) return set_err(QED_EINVAL, "unknown generator");
  c->rng = rng;
  return QED_OK;
}

extern "C" int qed_ctx_set_flag_rule(qed_ctx *c, int rule) {
  if (!c) return set_err(QED_EINVAL, "ctx is NULL");
  if (rule != QED_FLAG_ESTIMATE && rule != QED_FLAG_INTERVAL) return set_err(QED_EINVAL, "unknown flag rule");
  c->flag_rule = rule;
  return QED_OK;
}

extern "C" int qed_ctx_set_threshold(qed_ctx *c, double rel) {
  if (!c || !(rel > 0.0)) return set_err(QED_EINVAL, "threshold must be > 0");
  c->thresh = rel;
  return QED_OK;
}

// ---------------------------------------------------------------------------
// bytecode programs
// ---------------------------------------------------------------------------
// Every instruction is checked against its program's register and constant
// counts here, so that the interpreter's shared-memory accesses stay inside
// the frame the host sized for it.
static bool vm_check(const uint2 *ins, int n_ins, int n_regs, int n_kon, int n_lines, std::string &why) {
  if (n_regs < n_lines || n_regs > 1023 || n_kon < 0 || n_kon > 4096 || n_ins < 1) { why = "program sizes out of range"; return false; }
  auto ok = [&](uint32_t a) { return a < VM_KFLAG ? int(a) < n_regs : int(a - VM_KFLAG) < n_kon; };
  for (int i = 0; i < n_ins; ++i) {
    const uint32_t lo = ins[i].x, hi = ins[i].y;
    const uint32_t a = lo & 8191u, b = (lo >> 13) & 8191u, d = (hi >> 6) & 1023u, sp = (hi >> 2) & 7u;
    if ((lo >> 26) || (hi >> 16) || sp > VM_SP_END) { why = "reserved or bad instruction field"; return false; }
    // both operands are read by every instruction
    if (!ok(a) || !ok(b)) { why = "operand out of range"; return false; }
    if (d != 0 && (int(d) < n_lines || int(d) >= n_regs)) { why = "store target out of range"; return false; }
    // the interpreter loads an instruction's operands before the previous
    // instruction stores
    if (i > 0) {
      const uint32_t pd = (ins[i - 1].y >> 6) & 1023u;
      if (pd != 0 && (a == pd || b == pd)) { why = "instruction reads the register the previous one writes"; return false; }
    }
    if (sp == VM_SP_END) {
      if (i != n_ins - 1) { why = "END is not the last instruction"; return false; }
      return true;
    }
  }
  why = "program without END";
  return false;
}

// FP64 operations (an FMA counts 2) of one evaluation of a program in the
// interpreter's double-double arithmetic, instruction by instruction: the
// fused step acc = X * B + O costs 18 in general, 10 without an addend, 11
// when B is the constant 1 and there is an addend, none for a move; its
// absolute-value lane one FMA; RCP a double-double division (86); ACCW one
// FMA.  An algorithmic count of the re-evaluation of a flagged point.
static double vm_dd_flops(const uint2 *ins, int n_ins, const unsigned char *kon, int n_kon) {
  double f = 0.0;
  for (int i = 0; i < n_ins; ++i) {
    const uint32_t lo = ins[i].x, hi = ins[i].y;
    const uint32_t b = (lo >> 13) & 8191u, zo = (hi >> 1) & 1u, spec = (hi >> 2) & 7u, nocomp = (hi >> 5) & 1u;
    if (!nocomp) {
      bool b_one = false;
      if (b >= 4096u && int(b - 4096u) < n_kon) {
        double v;
        std::memcpy(&v, kon + 8 * size_t(b - 4096u), 8);
        b_one = v == 1.0;
      }
      f += b_one ? (zo ? 11.0 : 0.0) : (zo ? 18.0 : 10.0);
      f += 2.0;
    }
    if (spec == 1u) f += 86.0;
    else if (spec == 3u) f += 2.0;
  }
  return f;
}

extern "C" int qed_programs_load(qed_ctx *c, const void *data, size_t bytes, int *count) {
  if (!c || !data) return set_err(QED_EINVAL, "ctx/data is NULL");
  const unsigned char *p = static_cast<const unsigned char *>(data), *end = p + bytes;
  if (bytes < 16 || std::memcmp(p, "QEDVM004", 8) != 0) return set_err(QED_EINVAL, "not a qed program file");
  uint32_t n = 0;
  std::memcpy(&n, p + 8, 4);
  p += 16;
  struct Rec { qed_ctx::VmProg pr; const unsigned char *ins; const unsigned char *kon; };
  std::vector<Rec> recs;
  size_t words = 0, kons = 0;
  for (uint32_t i = 0; i < n; ++i) {
    if (end - p < 64 + 24) return set_err(QED_EINVAL, "truncated program file");
    Rec r;
    char nm[65] = {0};
    std::memcpy(nm, p, 64);
    r.pr.name = nm;
    int32_t m[4];
    std::memcpy(m, p + 64, 16);
    std::memcpy(&r.pr.flops, p + 80, 8);
    p += 88;
    r.pr.n_lines = m[0]; r.pr.n_regs = m[1]; r.pr.n_ins = m[2]; r.pr.n_kon = m[3];
    if (m[0] < 3 || m[0] > 3 * QED_MAX_LOOPS || m[0] % 3 || m[2] < 1 || m[3] < 0) return set_err(QED_EINVAL, "bad program header");
    const size_t ib = size_t(m[2]) * 8, kb = size_t(m[3]) * 8;
    if (size_t(end - p) < ib + kb) return set_err(QED_EINVAL, "truncated program file");
    r.ins = p;
    r.kon = p + ib;
    std::string why;
    std::vector<uint2> tmp(static_cast<size_t>(m[2]));
    std::memcpy(tmp.data(), r.ins, ib);
    if (!vm_check(tmp.data(), m[2], m[1], m[3], m[0], why)) return set_err(QED_EINVAL, "program " + r.pr.name + ": " + why);
    r.pr.dd_flops = vm_dd_flops(tmp.data(), m[2], r.kon, m[3]);
    p += ib + kb;
    words += (((size_t(m[2]) + 1) & ~size_t(1)) + 16) * 2;  // 32-bit words: pairs, plus 8 zero groups
    kons += size_t(m[3]);
    recs.push_back(r);
  }
  CUDA_TRY(cudaSetDevice(c->device));
  // one buffer per file: instructions (each program padded with zero words
  // to an even count, so 16-byte aligned, then eight zero groups that the
  // interpreter's look-ahead reads but never executes: END comes first and
  // a zero word names register 0), then the constants
  void *buf = nullptr;
  const size_t wbytes = words * 4, total = wbytes + kons * 8 + 16;
  CUDA_TRY(cudaMalloc(&buf, total));
  std::vector<unsigned char> host(total, 0);
  size_t wo = 0, ko = wbytes;
  std::vector<qed_ctx::VmProg> progs;
  for (auto &r : recs) {
    std::memcpy(host.data() + wo, r.ins, size_t(r.pr.n_ins) * 8);
    r.pr.d_ins = reinterpret_cast<const uint2 *>(static_cast<unsigned char *>(buf) + wo);
    wo += (((size_t(r.pr.n_ins) + 1) & ~size_t(1)) + 16) * 8;
    std::memcpy(host.data() + ko, r.kon, size_t(r.pr.n_kon) * 8);
    r.pr.d_kon = reinterpret_cast<const double *>(static_cast<unsigned char *>(buf) + ko);
    ko += size_t(r.pr.n_kon) * 8;
    progs.push_back(r.pr);
  }
  cudaError_t e = cudaMemcpy(buf, host.data(), total, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { cudaFree(buf); return set_err(QED_ECUDA, cudaGetErrorString(e)); }
  c->vm_bufs.push_back(buf);
  for (auto &pr : progs) c->vm.push_back(pr);
  if (count) *count = int(progs.size());
  return QED_OK;
}

// ---------------------------------------------------------------------------
// graphs
// ---------------------------------------------------------------------------
static bool to_graph(const qed_graph *in, qed::Graph &g, std::string &why) {
  if (!in) { why = "graph is NULL"; return false; }
  if (in->n < 1 || in->n > QED_MAX_LOOPS) { why = "loop order out of range"; return false; }
  g = qed::Graph();
  g.n = in->n;
  g.e = in->e;
  std::vector<int> seen(2 * g.n, 0);
  for (int a = 0; a < g.n; ++a) {
    int s = in->pairs[2 * a], t = in->pairs[2 * a + 1];
    if (s < 0 || t < 0 || s >= 2 * g.n || t >= 2 * g.n || s == t) { why = "photon endpoint out of range"; return false; }
    if (seen[s]++ || seen[t]++) { why = "vertex used twice"; return false; }
    g.ph.push_back({std::min(s, t), std::max(s, t)});
  }
  std::sort(g.ph.begin(), g.ph.end());
  if (g.e < 1 || g.e > 2 * g.n - 1) { why = "external vertex position out of range"; return false; }
  if (!qed::admissible(g)) { why = "graph has a self-energy on an external leg or is one-particle reducible"; return false; }
  return true;
}

static void from_graph(const qed::Graph &g, uint32_t id, qed_graph *o) {
  std::memset(o, 0, sizeof *o);
  o->n = g.n;
  o->e = g.e;
  for (int a = 0; a < g.n; ++a) { o->pairs[2 * a] = g.ph[a].first; o->pairs[2 * a + 1] = g.ph[a].second; }
  o->stream_id = id;
}

extern "C" int qed_enumerate(int n, int reduced, qed_graph *out, int cap, int *count) {
  if (n < 1 || n > QED_MAX_LOOPS || !count) return set_err(QED_EINVAL, "bad arguments");
  auto gs = qed::enumerate_graphs(n);
  std::vector<qed::Graph> sel;
  if (!reduced) sel = gs;
  else {
    for (auto &g : gs) {
      auto m = g.mirror();
      if (g.key() <= m.key()) sel.push_back(g);
    }
  }
  *count = int(sel.size());
  for (int i = 0; i < std::min(cap, int(sel.size())); ++i) from_graph(sel[i], uint32_t(i), out + i);
  return QED_OK;
}

extern "C" int qed_gauge_class(const qed_graph *in, int kmn[3]) {
  qed::Graph g;
  std::string why;
  if (!to_graph(in, g, why)) return set_err(QED_EINVAL, why);
  auto c = g.gauge_class();
  kmn[0] = c[0]; kmn[1] = c[1]; kmn[2] = c[2];
  return QED_OK;
}

extern "C" int qed_diagram_free(qed_diag *d);
extern "C" int qed_eval_points(qed_diag *d, const double *z_dev, uint64_t n, int prec, double *f_dev);
extern "C" int qed_diagram_load(qed_ctx *ctx, const qed_graph *gin, const qed_pdf *pdf, qed_diag **out) {
  if (!ctx || !out) return set_err(QED_EINVAL, "ctx/out is NULL");
  qed::Graph g;
  std::string why;
  if (!to_graph(gin, g, why)) return set_err(QED_EINVAL, why);
  int fid = -1, vm = -1;
  const std::string nm = g.name();
  for (int i = 0; i < QED_N_GENERATED; ++i) if (nm == qed_generated_names[i]) fid = i;
  if (fid < 0 || ctx->prefer_vm)
    for (size_t i = 0; i < ctx->vm.size(); ++i)
      if (ctx->vm[i].name == nm && ctx->vm[i].n_lines == g.n_lines()) vm = int(i);
  if (vm >= 0) fid = -1;
  if (fid < 0 && vm < 0) return set_err(QED_ENOTFOUND, "no generated integrand or program for " + nm);
  const int N = g.n_lines();
  const size_t M = size_t(1) << N;
  qed_diag *d = new qed_diag();
  d->ctx = ctx; d->g = g; d->stream_id = gin->stream_id; d->fid = fid; d->vm = vm; d->N = N;
  if (pdf && pdf->deg) {
    d->deg0.assign(pdf->deg, pdf->deg + M);
    for (size_t m = 1; m + 1 < M; ++m)
      if (!(d->deg0[m] > 0.0) || !std::isfinite(d->deg0[m])) { delete d; return set_err(QED_EINVAL, "Deg must be positive and finite on every proper subset"); }
    d->d_min = 1e-300;   // a caller's table is used as given (no floor)
  } else {
    double c_div = (pdf && pdf->c_div > 0) ? pdf->c_div : 0.5;
    d->d_min = (pdf && pdf->d_min > 0) ? pdf->d_min : 0.05;
    d->deg0 = qed::deg_table(g, c_div, d->d_min);
  }
  d->alpha.assign(N, 0.0);
  d->beta.assign(N, 0.0);
  CUDA_TRY(cudaSetDevice(ctx->device));
  if (cudaMalloc(&d->d_tab, (3 * M + N) * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&d->d_act, M) != cudaSuccess) {
    qed_diagram_free(d);
    return set_err(QED_ENOMEM, "table allocation");
  }
  int rc = rebuild_tables(d);
  if (rc) { qed_diagram_free(d); return rc; }
  *out = d;
  return QED_OK;
}

extern "C" int qed_diagram_free(qed_diag *d) {
  if (!d) return QED_OK;
  cudaSetDevice(d->ctx->device);
  if (d->d_tab) cudaFree(d->d_tab);
  if (d->d_act) cudaFree(d->d_act);
  delete d;
  return QED_OK;
}

extern "C" int qed_diagram_info(const qed_diag *d, int *n_lines, int *fid, double *log_norm) {
  if (!d) return set_err(QED_EINVAL, "diag is NULL");
  if (n_lines) *n_lines = d->N;
  if (fid) *fid = d->vm >= 0 ? QED_N_GENERATED + d->vm : d->fid;
  if (log_norm) *log_norm = d->logZ;
  return QED_OK;
}

// ---------------------------------------------------------------------------
// integration
// ---------------------------------------------------------------------------
static KParams base_params(const qed_diag *d, uint64_t begin, uint64_t n, uint64_t seed) {
  KParams P;
  std::memset(&P, 0, sizeof P);
  const size_t M = size_t(1) << d->N;
  P.F = d->d_tab; P.G = d->d_tab + M; P.invdeg = d->d_tab + 2 * M; P.off = d->d_tab + 3 * M;
  P.logZ = d->logZ;
  P.begin = begin; P.n = n;
  P.key0 = uint32_t(seed); P.key1 = uint32_t(seed >> 32);
  P.stream = d->stream_id;
  P.thresh = d->ctx->thresh;
  P.rng = uint32_t(d->ctx->rng);
  if (P.rng == QED_RNG_MRG32K3A) {
    P.mrg_bits = mrg::index_bits(begin + n);
    P.mrg_jump = d->ctx->mrg_jump;
    mrg::stream_start(seed, d->stream_id, P.mrg);
  }
  return P;
}

static int launch(const void *fn, int blocks, int threads, size_t smem, cudaStream_t st, void **args) {
  CUDA_TRY(cudaLaunchKernel(fn, dim3(blocks), dim3(threads), args, smem, st));
  return QED_OK;
}

// Launch shape of an interpreter kernel: the block size starts at `threads`
// and halves until the frame (constants + one register file per thread)
// fits in shared memory; blocks = resident blocks per SM x SMs.
struct VmLaunch {
  int threads = 0, blocks = 0;
  size_t smem = 0;
  VmCode code;
};
// frame: 0 = FP64 (the context's points per thread), 1 = double-double,
// 2 = FP64 interval
static int vm_launch(const qed_ctx *c, const qed_ctx::VmProg &pr, const void *fn, int frame, int threads,
                     VmLaunch &L) {
  L.code = VmCode{pr.d_ins, pr.d_kon, pr.n_kon, pr.n_regs};
  const size_t cap = 220 * 1024;       // dynamic part; the kernels' static shared memory is a few KB
  const bool dd_frame = frame != 0;    // both wide frames take the occupancy search below
  auto bytes = [&](int t) {
    if (frame == 2) return vm_smem_bytes<ivl, 1>(pr.n_kon, pr.n_regs, t);
    if (frame == 1) return vm_smem_bytes<dd, 1>(pr.n_kon, pr.n_regs, t);
    return c->vm_points == 2 ? vm_smem_bytes<double, 2>(pr.n_kon, pr.n_regs, t)
                             : vm_smem_bytes<double, 1>(pr.n_kon, pr.n_regs, t);
  };
  int T = threads;
  while (T > 32 && bytes(T) > cap) T /= 2;
  if (bytes(T) > cap) return set_err(QED_EINVAL, "program " + pr.name + " needs more shared memory than a block has");
  int occ = 0;
  if (dd_frame) {
    // the double-double frame (24 bytes per register and thread; an
    // interval 16) limits an SM to a few warps: take the block size, 32 to 256 threads, that keeps
    // the most threads resident (the smaller one on a tie), e.g. one block
    // of 128 rather than one of 64 for the largest four-loop programs
    int best = 0;
    for (int t = 32; t <= 256; t *= 2) {
      if (bytes(t) > cap) break;
      CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes(t))));
      int o = 0;
      CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fn, t, bytes(t)));
      if (o * t > best) { best = o * t; T = t; }
    }
  }
  L.threads = T;
  L.smem = bytes(T);
  CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(L.smem)));
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, T, L.smem));
  L.blocks = std::max(1, occ) * c->sms;
  return QED_OK;
}
static const VmKernelSet &vm_kernels(const qed_diag *d) {
  return g_vm_kernels[d->ctx->vm_points == 2 ? 1 : 0][d->N / 3 - 1];
}

static int fold(qed_ctx *c, int blocks, qed_result *r, bool add_flagged_as_count);
static void finish(qed_result *r);

// Per-graph integration with a bytecode integrand: launches of at most
// queue_cap samples, so the flagged queue cannot overflow.
static int integrate_range_vm(qed_diag *d, uint64_t begin, uint64_t n, uint64_t seed, qed_result *out) {
  qed_ctx *c = d->ctx;
  const VmKernelSet &K = vm_kernels(d);
  const auto &pr = c->vm[d->vm];
  VmLaunch L1, L2;
  const bool interval = c->flag_rule == QED_FLAG_INTERVAL;
  const void *kint = interval ? K.integrate_ivl : K.integrate;
  int rc = vm_launch(c, pr, kint, interval ? 2 : 0, interval ? 64 : c->vm_threads, L1);
  if (!rc) rc = vm_launch(c, pr, K.redo, 1, 64, L2);
  if (!rc) rc = ensure_scratch(c, std::max(L1.blocks, L2.blocks));
  if (rc) return rc;
  qed_result r;
  std::memset(&r, 0, sizeof r);
  r.n = n;
  CUDA_TRY(cudaEventRecord(c->ev0, c->stream));
  const uint64_t chunk = c->queue_cap;
  for (uint64_t off = 0; off < n; off += chunk) {
    const uint64_t m = std::min(chunk, n - off);
    KParams P = base_params(d, begin + off, m, seed);
    P.partials = c->partials; P.counts = c->counts;
    P.queue = c->queue; P.queue_len = c->queue_len; P.queue_cap = c->queue_cap;
    CUDA_TRY(cudaMemsetAsync(c->queue_len, 0, sizeof(unsigned int), c->stream));
    void *args[] = {&P, &L1.code};
    CUDA_TRY(cudaEventRecord(c->evk0, c->stream));
    if ((rc = launch(kint, L1.blocks, L1.threads, L1.smem, c->stream, args))) return rc;
    CUDA_TRY(cudaEventRecord(c->evk1, c->stream));
    ++r.launches;
    if ((rc = fold(c, L1.blocks, &r, true))) return rc;
    float kms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&kms, c->evk0, c->evk1));
    r.kernel_seconds += kms * 1e-3;
    unsigned int qn = 0;
    CUDA_TRY(cudaMemcpy(&qn, c->queue_len, sizeof qn, cudaMemcpyDeviceToHost));
    if (qn > c->queue_cap) return set_err(QED_ECUDA, "flagged queue overflow");   // cannot happen: m <= queue_cap
    if (qn > 0) {
      void *args2[] = {&P, &L2.code, &qn};
      CUDA_TRY(cudaEventRecord(c->evk1, c->stream));
      if ((rc = launch(K.redo, L2.blocks, L2.threads, L2.smem, c->stream, args2))) return rc;
      CUDA_TRY(cudaEventRecord(c->evk2, c->stream));
      ++r.launches;
      if ((rc = fold(c, L2.blocks, &r, false))) return rc;
      float dms = 0.f;
      CUDA_TRY(cudaEventElapsedTime(&dms, c->evk1, c->evk2));
      r.dd_seconds += dms * 1e-3;
    }
  }
  CUDA_TRY(cudaEventRecord(c->ev1, c->stream));
  CUDA_TRY(cudaEventSynchronize(c->ev1));
  float ms = 0.f;
  CUDA_TRY(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
  r.seconds = ms * 1e-3;
  finish(&r);
  *out = r;
  return QED_OK;
}

static void dd_acc(double &hi, double &lo, double a_hi, double a_lo) {
  // host double-double accumulate (hi, lo) += (a_hi, a_lo)
  double s = hi + a_hi;
  double bb = s - hi;
  double err = (hi - (s - bb)) + (a_hi - bb);
  err += lo + a_lo;
  hi = s + err;
  lo = err - (hi - s);
}

static int fold(qed_ctx *c, int blocks, qed_result *r, bool add_flagged_as_count) {
  CUDA_TRY(cudaMemcpyAsync(c->h_partials.data(), c->partials, size_t(blocks) * QED_PART * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaMemcpyAsync(c->h_counts.data(), c->counts, size_t(blocks) * 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  for (int b = 0; b < blocks; ++b) {
    const double *pb = c->h_partials.data() + QED_PART * size_t(b);
    dd_acc(r->sum_w[0], r->sum_w[1], pb[0], pb[1]);
    dd_acc(r->sum_w2[0], r->sum_w2[1], pb[2], pb[3]);
    r->unstable_abs_w += pb[4];
    if (add_flagged_as_count) r->n_flagged += c->h_counts[2 * b];
    r->n_unstable += c->h_counts[2 * b + 1];
  }
  return QED_OK;
}

static void finish(qed_result *r) {
  const double N = double(r->n);
  if (r->n == 0) { r->value = 0.0; r->variance = 0.0; return; }
  const double mean = (r->sum_w[0] + r->sum_w[1]) / N;
  const double m2 = (r->sum_w2[0] + r->sum_w2[1]) / N;
  r->value = mean;
  r->variance = r->n > 1 ? std::max(0.0, m2 - mean * mean) / (N - 1.0) : 0.0;
}

extern "C" int qed_integrate_range(qed_diag *d, uint64_t begin, uint64_t n, uint64_t seed, qed_result *out) {
  if (!d || !out) return set_err(QED_EINVAL, "diag/out is NULL");
  qed_ctx *c = d->ctx;
  CUDA_TRY(cudaSetDevice(c->device));
  if (d->vm >= 0) return integrate_range_vm(d, begin, n, seed, out);
  if (c->flag_rule == QED_FLAG_INTERVAL)
    return set_err(QED_EINVAL, "the interval rule evaluates bytecode programs: load the graph on a "
                               "QED_CTX_PREFER_PROGRAMS context");
  const KernelSet &K = *g_kernels[d->fid];
  const int threads = c->threads;
  const int blocks = c->blocks > 0 ? c->blocks : 4 * c->sms;
  int rc = ensure_scratch(c, blocks);
  if (rc) return rc;
  const size_t smem = table_smem(d->N);
  qed_result r;
  std::memset(&r, 0, sizeof r);
  r.n = n;
  CUDA_TRY(cudaEventRecord(c->ev0, c->stream));
  const uint64_t chunk = uint64_t(1) << 30;
  for (uint64_t off = 0; off < n; off += chunk) {
    const uint64_t m = std::min(chunk, n - off);
    KParams P = base_params(d, begin + off, m, seed);
    P.partials = c->partials; P.counts = c->counts;
    P.queue = c->queue; P.queue_len = c->queue_len; P.queue_cap = c->queue_cap;
    CUDA_TRY(cudaMemsetAsync(c->queue_len, 0, sizeof(unsigned int), c->stream));
    void *args[] = {&P};
    CUDA_TRY(cudaEventRecord(c->evk0, c->stream));
    if ((rc = launch(K.integrate, blocks, threads, smem, c->stream, args))) return rc;
    CUDA_TRY(cudaEventRecord(c->evk1, c->stream));
    ++r.launches;
    qed_result first;
    std::memset(&first, 0, sizeof first);
    if ((rc = fold(c, blocks, &first, true))) return rc;
    float kms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&kms, c->evk0, c->evk1));
    r.kernel_seconds += kms * 1e-3;
    unsigned int qn = 0;
    CUDA_TRY(cudaMemcpy(&qn, c->queue_len, sizeof qn, cudaMemcpyDeviceToHost));
    // mode 1 (the queue overflowed): the double-double kernel makes a
    // complete second pass that replaces this one (flag decisions included)
    const int mode = qn > c->queue_cap ? 1 : 0;
    if (mode == 0) {
      dd_acc(r.sum_w[0], r.sum_w[1], first.sum_w[0], first.sum_w[1]);
      dd_acc(r.sum_w2[0], r.sum_w2[1], first.sum_w2[0], first.sum_w2[1]);
      r.n_flagged += first.n_flagged;
    }
    if (qn > 0) {
      int m = mode;
      unsigned int qcount = std::min(qn, c->queue_cap);
      void *args2[] = {&P, &m, &qcount};
      CUDA_TRY(cudaEventRecord(c->evk1, c->stream));
      if ((rc = launch(K.redo, blocks, threads, smem, c->stream, args2))) return rc;
      CUDA_TRY(cudaEventRecord(c->evk2, c->stream));
      ++r.launches;
      if ((rc = fold(c, blocks, &r, mode == 1))) return rc;
      float dms = 0.f;
      CUDA_TRY(cudaEventElapsedTime(&dms, c->evk1, c->evk2));
      r.dd_seconds += dms * 1e-3;
    }
  }
  CUDA_TRY(cudaEventRecord(c->ev1, c->stream));
  CUDA_TRY(cudaEventSynchronize(c->ev1));
  float ms = 0.f;
  CUDA_TRY(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
  r.seconds = ms * 1e-3;
  finish(&r);
  *out = r;
  return QED_OK;
}

extern "C" int qed_integrate(qed_diag *d, uint64_t n, uint64_t seed, qed_result *out) {
  return qed_integrate_range(d, 0, n, seed, out);
}

extern "C" int qed_dump_points(qed_diag *d, uint64_t begin, uint64_t n, uint64_t seed, double *z_dev, double *f_dev,
                               double *lp_dev, uint8_t *flag_dev) {
  if (!d || !z_dev || !f_dev || !lp_dev || !flag_dev) return set_err(QED_EINVAL, "NULL argument");
  qed_ctx *c = d->ctx;
  CUDA_TRY(cudaSetDevice(c->device));
  KParams P = base_params(d, begin, n, seed);
  P.z_out = z_dev; P.f_out = f_dev; P.lp_out = lp_dev; P.flag_out = flag_dev;
  if (d->vm >= 0) {
    VmLaunch L;
    int rc = vm_launch(c, c->vm[d->vm], vm_kernels(d).dump, 0, c->vm_threads, L);
    if (rc) return rc;
    const int blocks = int(std::max<uint64_t>(1, std::min<uint64_t>((n + L.threads - 1) / L.threads, uint64_t(L.blocks))));
    void *args[] = {&P, &L.code};
    if ((rc = launch(vm_kernels(d).dump, blocks, L.threads, L.smem, c->stream, args))) return rc;
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return QED_OK;
  }
  const int threads = c->threads;
  const int blocks = int(std::max<uint64_t>(1, std::min<uint64_t>((n + threads - 1) / threads, uint64_t(c->sms) * 8)));
  void *args[] = {&P};
  int rc = launch(g_kernels[d->fid]->dump, blocks, threads, table_smem(d->N), c->stream, args);
  if (rc) return rc;
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return QED_OK;
}

extern "C" int qed_eval_points(qed_diag *d, const double *z_dev, uint64_t n, int prec, double *f_dev) {
  if (!d || !z_dev || !f_dev || (prec != 0 && prec != 1)) return set_err(QED_EINVAL, "bad argument");
  qed_ctx *c = d->ctx;
  CUDA_TRY(cudaSetDevice(c->device));
  if (d->vm >= 0) {
    VmLaunch L;
    const void *fn = vm_kernels(d).eval;
    int rc = vm_launch(c, c->vm[d->vm], fn, prec == 1 ? 1 : 0, prec == 1 ? 64 : c->vm_threads, L);
    if (rc) return rc;
    const int blocks = int(std::max<uint64_t>(1, std::min<uint64_t>((n + L.threads - 1) / L.threads, uint64_t(L.blocks))));
    void *args[] = {(void *)&z_dev, &n, &prec, &f_dev, &L.code};
    if ((rc = launch(fn, blocks, L.threads, L.smem, c->stream, args))) return rc;
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return QED_OK;
  }
  const int threads = c->threads;
  const int blocks = int(std::max<uint64_t>(1, std::min<uint64_t>((n + threads - 1) / threads, uint64_t(c->sms) * 8)));
  void *args[] = {(void *)&z_dev, &n, &prec, &f_dev};
  int rc = launch(g_kernels[d->fid]->eval, blocks, threads, 0, c->stream, args);
  if (rc) return rc;
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return QED_OK;
}

extern "C" int qed_eval_interval(qed_diag *d, const double *z_dev, uint64_t n, double *lo_dev, double *hi_dev) {
  if (!d) return set_err(QED_EINVAL, "diag is NULL");
  if (d->vm < 0)
    return set_err(QED_EINVAL, "interval arithmetic runs on bytecode programs: load the graph on a "
                               "QED_CTX_PREFER_PROGRAMS context");
  if (n == 0) return QED_OK;
  if (!z_dev || !lo_dev || !hi_dev) return set_err(QED_EINVAL, "NULL buffer");
  qed_ctx *c = d->ctx;
  CUDA_TRY(cudaSetDevice(c->device));
  VmLaunch L;
  const void *fn = vm_kernels(d).eval_ivl;
  int rc = vm_launch(c, c->vm[d->vm], fn, 2, 64, L);
  if (rc) return rc;
  const int blocks = int(std::max<uint64_t>(1, std::min<uint64_t>((n + L.threads - 1) / L.threads, uint64_t(L.blocks))));
  void *args[] = {(void *)&z_dev, &n, &lo_dev, &hi_dev, &L.code};
  if ((rc = launch(fn, blocks, L.threads, L.smem, c->stream, args))) return rc;
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return QED_OK;
}

extern "C" int qed_result_merge(const qed_result *a, const qed_result *b, qed_result *out) {
  if (!a || !b || !out) return set_err(QED_EINVAL, "NULL argument");
  qed_result r;
  std::memset(&r, 0, sizeof r);
  r.sum_w[0] = a->sum_w[0]; r.sum_w[1] = a->sum_w[1];
  r.sum_w2[0] = a->sum_w2[0]; r.sum_w2[1] = a->sum_w2[1];
  dd_acc(r.sum_w[0], r.sum_w[1], b->sum_w[0], b->sum_w[1]);
  dd_acc(r.sum_w2[0], r.sum_w2[1], b->sum_w2[0], b->sum_w2[1]);
  r.n = a->n + b->n;
  r.n_flagged = a->n_flagged + b->n_flagged;
  r.n_unstable = a->n_unstable + b->n_unstable;
  r.seconds = a->seconds + b->seconds;
  r.unstable_abs_w = a->unstable_abs_w + b->unstable_abs_w;
  r.dd_seconds = a->dd_seconds + b->dd_seconds;
  r.kernel_seconds = a->kernel_seconds + b->kernel_seconds;
  r.launches = a->launches + b->launches;
  finish(&r);
  *out = r;
  return QED_OK;
}

// ---------------------------------------------------------------------------
// measurement helpers
// ---------------------------------------------------------------------------
extern "C" int qed_diagram_flops(const qed_diag *d, double *flops) {
  if (!d || !flops) return set_err(QED_EINVAL, "NULL argument");
  const double N = d->N;
  // sampler: uniform map (2 per draw), walk (target product and on average
  // half of the running sums per level), radial (log, scale, running sum,
  // exp, density update), weight (exp, product), accumulation (square and
  // two compensated sums)
  const double sampler = 4.0 * (N - 1) + (N - 1) + (N - 1) * (N + 2) / 4.0 + 6.0 * (N - 1) + 2.0 + 9.0;
  *flops = (d->vm >= 0 ? d->ctx->vm[d->vm].flops : qed_generated_flops[d->fid]) + sampler;
  return QED_OK;
}

__global__ void k_fp64_peak(double *out, int iters, double b, double c) {
  double a[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) a[i] = 1e-3 * (threadIdx.x + 1) + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = fma(a[i], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 16; ++i) s += a[i];
  if (s == -1.2345e300) out[0] = s;   // keeps the chains live
}

extern "C" int qed_diagram_flops_dd(const qed_diag *d, double *flops) {
  if (!d || !flops) return set_err(QED_EINVAL, "NULL argument");
  const qed_ctx *c = d->ctx;
  int k = d->vm;
  if (k < 0) {
    // compiled integrand: the count of the same graph's program, if registered
    const std::string nm = d->g.name();
    for (size_t i = 0; i < c->vm.size() && k < 0; ++i)
      if (c->vm[i].name == nm) k = int(i);
    if (k < 0) return set_err(QED_ENOTFOUND, "no program of this graph is registered (qed_programs_load)");
  }
  double f64 = 0.0;
  qed_diagram_flops(d, &f64);
  // the sampler part runs in FP64 in both passes
  *flops = c->vm[k].dd_flops + (f64 - (d->vm >= 0 ? c->vm[d->vm].flops : qed_generated_flops[d->fid]));
  return QED_OK;
}

extern "C" int qed_fp64_peak(int device, double ms, double *flops) {
  if (!flops || !(ms > 0)) return set_err(QED_EINVAL, "bad argument");
  CUDA_TRY(cudaSetDevice(device));
  cudaDeviceProp prop;
  CUDA_TRY(cudaGetDeviceProperties(&prop, device));
  double *out = nullptr;
  CUDA_TRY(cudaMalloc(&out, sizeof(double)));
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  const int threads = 256, blocks = prop.multiProcessorCount * 8;
  int iters = 1 << 12;
  double best = 0.0;
  for (int rep = 0; rep < 8; ++rep) {
    CUDA_TRY(cudaEventRecord(e0));
    k_fp64_peak<<<blocks, threads>>>(out, iters, 0.99999999, 1e-9);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaEventRecord(e1));
    CUDA_TRY(cudaEventSynchronize(e1));
    float t = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
    const double f = 2.0 * 16.0 * double(iters) * threads * blocks / (t * 1e-3);
    best = std::max(best, f);
    if (t < 0.5 * ms && iters < (1 << 24)) iters *= 2;   // grow until the launch lasts about ms
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  *flops = best;
  return QED_OK;
}

// ---------------------------------------------------------------------------
// batched integration of a graph set (persistent kernel, variance-driven
// allocation, one CUDA graph per round shape replayed every round)
// ---------------------------------------------------------------------------
// qed_integrate_batch's set-up: device buffers, pinned host buffers and the
// captured round (a CUDA graph), owned by the context and reused by the next
// call of the same shape (same graphs, seed, threshold, item count, list
// size, kernels and launch shapes, stream), so that a caller integrating the
// same set step after step pays for the allocations and the capture once.
struct BatchPlan {
  // shape (the key)
  std::vector<qed_diag *> diags;
  uint64_t seed = 0;
  double thresh = 0.0;
  unsigned int n_items = 0;
  uint32_t list_cap = 0, dd_tiles = 0;
  const void *kern1 = nullptr, *kern2 = nullptr;
  int grid1 = 0, grid2 = 0, thr1 = 0, thr2 = 0;
  size_t smem = 0, smem2 = 0;
  bool use_graph = true;
  cudaStream_t user_stream = 0;
  int rng = 0;
  uint32_t mrg_bits = 0;
  bool vm = false;                  // bytecode batch: compacted double-double pass
  // resources: dev = {graph descriptors, items, next-item counters, FP64
  // partials, FP64 counts, dd partials, dd counts, flagged lists, and for
  // bytecode batches the dd plan: flat starts, tile table, tile count,
  // per-point w, per-point unstable |w|}
  void *dev[13] = {nullptr};
  void *h_items = nullptr, *h_out = nullptr;
  double *o_part = nullptr, *o_pdd = nullptr;
  unsigned long long *o_cnt = nullptr, *o_cdd = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t st = 0;
  bool own_stream = false;
  BatchParams B;
  size_t n_dd = 0;

  bool same_shape(const BatchPlan &o) const {
    return diags == o.diags && seed == o.seed && thresh == o.thresh && n_items == o.n_items &&
           list_cap == o.list_cap && dd_tiles == o.dd_tiles && kern1 == o.kern1 && kern2 == o.kern2 &&
           grid1 == o.grid1 && grid2 == o.grid2 && thr1 == o.thr1 && thr2 == o.thr2 && smem == o.smem &&
           smem2 == o.smem2 && use_graph == o.use_graph && user_stream == o.user_stream && rng == o.rng &&
           mrg_bits == o.mrg_bits && vm == o.vm;
  }
  BatchPlan() = default;
  BatchPlan(const BatchPlan &key) : diags(key.diags), seed(key.seed), thresh(key.thresh), n_items(key.n_items),
      list_cap(key.list_cap), dd_tiles(key.dd_tiles), kern1(key.kern1), kern2(key.kern2), grid1(key.grid1),
      grid2(key.grid2), thr1(key.thr1), thr2(key.thr2), smem(key.smem), smem2(key.smem2),
      use_graph(key.use_graph), user_stream(key.user_stream), rng(key.rng), mrg_bits(key.mrg_bits), vm(key.vm) {}
  BatchPlan &operator=(const BatchPlan &) = delete;
  ~BatchPlan() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (own_stream && st) cudaStreamDestroy(st);
    for (void *p : dev) if (p) cudaFree(p);
    if (h_items) cudaFreeHost(h_items);
    if (h_out) cudaFreeHost(h_out);
  }

  // copy the items in, run the FP64 kernel and the double-double kernel,
  // copy the partials out; with external event nodes when captured, so the
  // kernels can be timed after every replay
  int enqueue_round(qed_ctx *c, cudaStream_t s, bool capturing) {
    CUDA_TRY(cudaMemcpyAsync(dev[1], h_items, sizeof(BatchItem) * n_items, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemsetAsync(dev[2], 0, 2 * sizeof(unsigned int), s));
    void *args[] = {&B};
    const unsigned int evflags = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    CUDA_TRY(cudaEventRecordWithFlags(c->evk0, s, evflags));
    CUDA_TRY(cudaLaunchKernel(kern1, dim3(grid1), dim3(thr1), args, smem, s));
    CUDA_TRY(cudaEventRecordWithFlags(c->evk1, s, evflags));
    if (vm) CUDA_TRY(cudaLaunchKernel((const void *)k_batch_vm_dd_plan, dim3(1), dim3(32), args, 0, s));
    CUDA_TRY(cudaLaunchKernel(kern2, dim3(grid2), dim3(thr2), args, smem2, s));
    if (vm) CUDA_TRY(cudaLaunchKernel((const void *)k_batch_vm_dd_fold, dim3(n_items), dim3(32), args, 0, s));
    CUDA_TRY(cudaEventRecordWithFlags(c->evk2, s, evflags));
    CUDA_TRY(cudaMemcpyAsync(o_part, dev[3], sizeof(double) * QED_PART * n_items, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(o_pdd, dev[5], sizeof(double) * QED_PART * n_dd, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(o_cnt, dev[4], sizeof(unsigned long long) * 2 * n_items, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(o_cdd, dev[6], sizeof(unsigned long long) * 2 * n_dd, cudaMemcpyDeviceToHost, s));
    return QED_OK;
  }

  int allocate(qed_ctx *c, int k, size_t ndd) {
    n_dd = ndd;
    CUDA_TRY(cudaMalloc(&dev[0], sizeof(BatchDiag) * k));
    CUDA_TRY(cudaMalloc(&dev[1], sizeof(BatchItem) * n_items));
    CUDA_TRY(cudaMalloc(&dev[2], 2 * sizeof(unsigned int)));
    CUDA_TRY(cudaMalloc(&dev[3], sizeof(double) * QED_PART * n_items));
    CUDA_TRY(cudaMalloc(&dev[4], sizeof(unsigned long long) * 2 * n_items));
    CUDA_TRY(cudaMalloc(&dev[5], sizeof(double) * QED_PART * n_dd));
    CUDA_TRY(cudaMalloc(&dev[6], sizeof(unsigned long long) * 2 * n_dd));
    CUDA_TRY(cudaMalloc(&dev[7], sizeof(uint32_t) * size_t(list_cap) * n_items));
    uint32_t tab_cap = 0;
    if (vm) {
      // tiles: at most (all points) / tile + one partial tile per graph
      tab_cap = uint32_t((size_t(n_items) * list_cap + thr2 - 1) / size_t(thr2) + size_t(k) + 1);
      CUDA_TRY(cudaMalloc(&dev[8], sizeof(uint32_t) * (size_t(n_items) + 1)));
      CUDA_TRY(cudaMalloc(&dev[9], sizeof(uint4) * size_t(tab_cap)));
      CUDA_TRY(cudaMalloc(&dev[10], sizeof(unsigned int)));
      CUDA_TRY(cudaMalloc(&dev[11], sizeof(double) * size_t(list_cap) * n_items));
      CUDA_TRY(cudaMalloc(&dev[12], sizeof(double) * size_t(list_cap) * n_items));
    }
    const size_t out_bytes = n_items * (QED_PART * sizeof(double) + 2 * sizeof(unsigned long long)) +
                             n_dd * (QED_PART * sizeof(double) + 2 * sizeof(unsigned long long));
    CUDA_TRY(cudaMallocHost(&h_items, sizeof(BatchItem) * n_items));
    CUDA_TRY(cudaMallocHost(&h_out, out_bytes));
    o_part = (double *)h_out;
    o_pdd = o_part + QED_PART * size_t(n_items);
    o_cnt = (unsigned long long *)(o_pdd + QED_PART * n_dd);
    o_cdd = o_cnt + 2 * size_t(n_items);
    B.diags = (const BatchDiag *)dev[0]; B.items = (const BatchItem *)dev[1]; B.n_items = n_items;
    B.next_item = (unsigned int *)dev[2]; B.key0 = uint32_t(seed); B.key1 = uint32_t(seed >> 32);
    B.thresh = thresh; B.part = (double *)dev[3]; B.cnt = (unsigned long long *)dev[4];
    B.lists = (uint32_t *)dev[7]; B.list_cap = list_cap;
    B.part_dd = (double *)dev[5]; B.cnt_dd = (unsigned long long *)dev[6];
    B.dd_tiles = dd_tiles; B.next_tile = (unsigned int *)dev[2] + 1;
    B.rng = uint32_t(rng); B.mrg_bits = mrg_bits; B.mrg_jump = c->mrg_jump;
    B.dd_start = (uint32_t *)dev[8]; B.dd_tab = (uint4 *)dev[9]; B.dd_ntiles = (unsigned int *)dev[10];
    B.dd_tab_cap = tab_cap; B.dd_tile = uint32_t(thr2);
    B.dd_w = (double *)dev[11]; B.dd_u = (double *)dev[12];
    st = user_stream;
    if (use_graph) {
      if (st == 0) { CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)); own_stream = true; }
      cudaGraph_t graph;
      CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      int rc = enqueue_round(c, st, true);
      cudaError_t ce = cudaStreamEndCapture(st, &graph);
      if (rc) return rc;
      if (ce != cudaSuccess) return set_err(QED_ECUDA, std::string("capture: ") + cudaGetErrorString(ce));
      ce = cudaGraphInstantiate(&gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (ce != cudaSuccess) return set_err(QED_ECUDA, std::string("instantiate: ") + cudaGetErrorString(ce));
    }
    return QED_OK;
  }
};

static void drop_plan(qed_ctx *c) {
  delete c->plan;
  c->plan = nullptr;
}

extern "C" int qed_integrate_batch(qed_ctx *c, qed_diag *const *d, int k, uint64_t total, uint64_t seed,
                                   const qed_batch_opts *opts, qed_result *out) {
  if (!c || !d || !out || k < 1) return set_err(QED_EINVAL, "bad arguments");
  for (int g = 0; g < k; ++g)
    if (!d[g] || d[g]->ctx != c) return set_err(QED_EINVAL, "every graph must be loaded on this context");
  qed_batch_opts o;
  std::memset(&o, 0, sizeof o);
  if (opts) o = *opts;
  const int rounds = o.rounds > 0 ? o.rounds : 4;
  const uint64_t chunk = o.chunk > 0 ? o.chunk : (uint64_t(1) << 18);
  const int list_div = o.list_div > 0 ? o.list_div : 16;
  if (chunk > (uint64_t(1) << 31)) return set_err(QED_EINVAL, "chunk must be <= 2^31");
  if (o.policy != 0 && o.policy != 1) return set_err(QED_EINVAL, "policy must be 0 or 1");
  if (c->flag_rule != QED_FLAG_ESTIMATE) return set_err(QED_EINVAL, "the batched path flags by the estimate rule");
  CUDA_TRY(cudaSetDevice(c->device));
  // items per round (all rounds the same size so one captured graph serves all)
  const uint64_t per_round = (total + rounds - 1) / rounds;
  const unsigned int n_items = unsigned(std::max<uint64_t>(uint64_t(k), (per_round + chunk - 1) / chunk));
  // a batch is all compiled graphs or all bytecode graphs of one loop order
  int nvm = 0;
  for (int g = 0; g < k; ++g) nvm += d[g]->vm >= 0;
  const bool vmb = nvm > 0;
  if (vmb && nvm != k) return set_err(QED_EINVAL, "a batch holds compiled graphs or bytecode graphs, not both");
  if (vmb)
    for (int g = 0; g < k; ++g)
      if (d[g]->N != d[0]->N) return set_err(QED_EINVAL, "a batch of bytecode graphs holds one loop order");
  // bytecode batches: the flagged list of an item holds the whole chunk
  const uint32_t list_cap = vmb ? uint32_t(chunk) : uint32_t(std::max<uint64_t>(1, chunk / list_div));
  int Nmax = 0;
  for (int g = 0; g < k; ++g) Nmax = std::max(Nmax, d[g]->N);
  size_t smem = table_smem(Nmax), smem2 = smem;
  int thr1 = 256, thr2 = 256;
  const void *kern1 = qed_batch_kernels[0], *kern2 = qed_batch_kernels[1];
  VmLaunch L1, L2;
  if (vmb) {
    qed_ctx::VmProg big = c->vm[d[0]->vm];
    for (int g = 0; g < k; ++g) {
      big.n_regs = std::max(big.n_regs, c->vm[d[g]->vm].n_regs);
      big.n_kon = std::max(big.n_kon, c->vm[d[g]->vm].n_kon);
    }
    const VmKernelSet &K = vm_kernels(d[0]);
    kern1 = K.batch64;
    kern2 = K.batchdd;
    int rc = vm_launch(c, big, kern1, 0, c->vm_threads, L1);
    if (!rc) rc = vm_launch(c, big, kern2, 1, 64, L2);
    if (rc) return rc;
    smem = L1.smem; smem2 = L2.smem; thr1 = L1.threads; thr2 = L2.threads;
  }
  // one double-double partial per item (bytecode batches: folded per item
  // from the compacted pass's per-point results)
  const uint32_t dd_tiles = 1u;
  const size_t n_dd = size_t(n_items);
  int occ = 0;
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern1, thr1, smem));
  const int grid1 = std::max(1, occ) * c->sms;
  const int grid2 = vmb ? L2.blocks : std::min<int>(int(n_items), 4 * c->sms);
  // the set-up (buffers, pinned memory, the captured round) is kept on the
  // context and reused while the batch's shape is the same
  BatchPlan key;
  key.diags.assign(d, d + k);
  key.seed = seed; key.thresh = c->thresh; key.n_items = n_items; key.list_cap = list_cap; key.dd_tiles = dd_tiles;
  key.kern1 = kern1; key.kern2 = kern2; key.grid1 = grid1; key.grid2 = grid2; key.thr1 = thr1; key.thr2 = thr2;
  key.smem = smem; key.smem2 = smem2; key.use_graph = o.use_graph >= 0; key.user_stream = c->stream;
  key.rng = c->rng;
  key.vm = vmb;
  if (c->rng == QED_RNG_MRG32K3A) {
    // every sample index of the call is below counter_base + rounds x items
    // x chunk; rounded up to a multiple of 8 bits so that the captured round
    // is rebuilt rarely as the counters grow from call to call
    const uint64_t end = o.counter_base + uint64_t(rounds) * n_items * chunk;
    key.mrg_bits = std::min<uint32_t>(64u, (mrg::index_bits(end) + 7u) & ~7u);
  }
  if (!c->plan || !c->plan->same_shape(key)) {
    drop_plan(c);
    BatchPlan *P = new BatchPlan(key);
    c->plan = P;
    int rc = P->allocate(c, k, n_dd);
    if (rc) { drop_plan(c); return rc; }
  }
  BatchPlan &PL = *c->plan;
  std::vector<BatchDiag> hd(k);
  for (int g = 0; g < k; ++g) {
    const size_t M = size_t(1) << d[g]->N;
    hd[g].F = d[g]->d_tab; hd[g].G = d[g]->d_tab + M; hd[g].inv = d[g]->d_tab + 2 * M; hd[g].off = d[g]->d_tab + 3 * M;
    hd[g].logZ = d[g]->logZ; hd[g].stream = d[g]->stream_id; hd[g].fid = d[g]->fid; hd[g].N = d[g]->N; hd[g].pad = 0;
    hd[g].vins = nullptr; hd[g].vkon = nullptr; hd[g].vnk = 0; hd[g].vnr = 0;
    std::memset(hd[g].mrg, 0, sizeof hd[g].mrg);
    hd[g].pad2[0] = hd[g].pad2[1] = 0;
    if (c->rng == QED_RNG_MRG32K3A) mrg::stream_start(seed, d[g]->stream_id, hd[g].mrg);
    if (d[g]->vm >= 0) {
      const auto &pr = c->vm[d[g]->vm];
      hd[g].vins = pr.d_ins; hd[g].vkon = pr.d_kon; hd[g].vnk = pr.n_kon; hd[g].vnr = pr.n_regs;
    }
  }
  // the graphs' tables may have been rebuilt since the last call: upload
  // their descriptors every time (a few hundred bytes, before the rounds)
  CUDA_TRY(cudaMemcpy(PL.dev[0], hd.data(), sizeof(BatchDiag) * k, cudaMemcpyHostToDevice));
  double *o_part = PL.o_part, *o_pdd = PL.o_pdd;
  unsigned long long *o_cnt = PL.o_cnt, *o_cdd = PL.o_cdd;
  cudaGraphExec_t gexec = PL.gexec;
  cudaStream_t st = PL.st;
  // per-graph running state
  std::vector<qed_result> R(k);
  std::vector<uint64_t> next(k, o.counter_base);
  for (int g = 0; g < k; ++g) std::memset(&R[g], 0, sizeof(qed_result));
  std::vector<double> weight(k, 1.0), cost(k, 0.0);
  for (int g = 0; g < k; ++g) qed_diagram_flops(d[g], &cost[g]);
  BatchItem *hi = (BatchItem *)PL.h_items;
  uint32_t launches = 0;
  double kernel_ms = 0.0, dd_ms = 0.0;
  CUDA_TRY(cudaEventRecord(c->ev0, st));
  for (int r = 0; r < rounds; ++r) {
    // split n_items among graphs: round 0 (and policy 1) equal, else by weight
    // one item per graph, the rest by weight (largest-remainder rounding)
    std::vector<unsigned int> cnt(k, 1);
    std::vector<double> frac(k, 0.0);
    double wsum = 0.0;
    for (int g = 0; g < k; ++g) wsum += (r == 0 || o.policy == 1) ? 1.0 : weight[g];
    unsigned int given = unsigned(k);
    for (int g = 0; g < k; ++g) {
      const double w = (r == 0 || o.policy == 1) ? 1.0 : weight[g];
      const double q = double(n_items - k) * w / wsum;
      const unsigned int fl = unsigned(std::floor(q));
      cnt[g] += fl;
      frac[g] = q - double(fl);
      given += fl;
    }
    while (given < n_items) {
      const int gm = int(std::max_element(frac.begin(), frac.end()) - frac.begin());
      ++cnt[gm];
      frac[gm] = -1.0;
      ++given;
    }
    // items of the most expensive graphs first (FP64 operations per sample,
    // flagged samples at the double-double factor), so that the blocks that
    // take the last items from the queue finish close together: graphs of
    // one order differ up to ten-fold in cost.  The samples of every graph
    // and the order in which its items are folded stay the same.
    std::vector<int> ord(k);
    for (int g = 0; g < k; ++g) ord[g] = g;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    unsigned int it = 0;
    for (int g : ord)
      for (unsigned int j = 0; j < cnt[g]; ++j) {
        hi[it].diag = uint32_t(g); hi[it].begin = next[g]; hi[it].count = uint32_t(chunk);
        next[g] += chunk;
        ++it;
      }
    if (gexec) { CUDA_TRY(cudaGraphLaunch(gexec, st)); }
    else { int rc = PL.enqueue_round(c, st, false); if (rc) return rc; }
    launches += vmb ? 4 : 2;
    CUDA_TRY(cudaStreamSynchronize(st));
    {
      float kms = 0.f;
      if (cudaEventElapsedTime(&kms, c->evk0, c->evk1) == cudaSuccess) kernel_ms += kms;
      else (void)cudaGetLastError();   // timing unavailable: leave no error behind
      if (cudaEventElapsedTime(&kms, c->evk1, c->evk2) == cudaSuccess) dd_ms += kms;
      else (void)cudaGetLastError();
    }
    for (unsigned int i = 0; i < n_items; ++i) {
      qed_result &q = R[hi[i].diag];
      // an item whose flagged list overflowed (compiled batches: list_cap is
      // chunk / list_div) was evaluated again in full by the double-double
      // pass, which alone decides its points: its FP64 sums are not used
      const bool overflow = !vmb && o_cnt[2 * size_t(i)] > list_cap;
      if (!overflow) {
        const double *p = o_part + QED_PART * size_t(i);
        dd_acc(q.sum_w[0], q.sum_w[1], p[0], p[1]);
        dd_acc(q.sum_w2[0], q.sum_w2[1], p[2], p[3]);
        q.n_flagged += o_cnt[2 * size_t(i)];
      }
      for (uint32_t kt = 0; kt < dd_tiles; ++kt) {
        const size_t t = size_t(i) * dd_tiles + kt;
        const double *p = o_pdd + QED_PART * t;
        dd_acc(q.sum_w[0], q.sum_w[1], p[0], p[1]);
        dd_acc(q.sum_w2[0], q.sum_w2[1], p[2], p[3]);
        q.unstable_abs_w += p[4];
        q.n_unstable += o_cdd[2 * t + 1];
        if (overflow) q.n_flagged += o_cdd[2 * t];
      }
      q.n += hi[i].count;
    }
    // Neyman weights: sigma_g / sqrt(cost_g), cost = FP64 ops per sample with
    // flagged samples counted at the double-double factor
    for (int g = 0; g < k; ++g) {
      finish(&R[g]);
      const double var1 = R[g].variance * double(R[g].n);          // per-sample variance
      double fl = 0.0;
      qed_diagram_flops(d[g], &fl);
      const double frac = R[g].n ? double(R[g].n_flagged) / double(R[g].n) : 0.0;
      cost[g] = fl * (1.0 + 12.0 * frac);
      weight[g] = std::sqrt(std::max(var1, 0.0) / std::max(cost[g], 1.0));
      if (!(weight[g] > 0.0) || !std::isfinite(weight[g])) weight[g] = 1e-300;
    }
  }
  CUDA_TRY(cudaEventRecord(c->ev1, st));
  CUDA_TRY(cudaEventSynchronize(c->ev1));
  float ms = 0.f;
  CUDA_TRY(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
  for (int g = 0; g < k; ++g) {
    finish(&R[g]);
    R[g].seconds = ms * 1e-3;
    R[g].kernel_seconds = kernel_ms * 1e-3;
    R[g].dd_seconds = dd_ms * 1e-3;
    R[g].launches = launches;
    out[g] = R[g];
  }
  return QED_OK;
}

// ---------------------------------------------------------------------------
// tunable density parameters and the adjoint of the second moment
// ---------------------------------------------------------------------------
extern "C" int qed_diagram_set_pdf_params(qed_diag *d, const double *alpha, const double *beta) {
  if (!d) return set_err(QED_EINVAL, "diag is NULL");
  for (int l = 0; l < d->N; ++l) {
    d->alpha[l] = alpha ? alpha[l] : 0.0;
    d->beta[l] = beta ? beta[l] : 0.0;
    if (!std::isfinite(d->alpha[l]) || !std::isfinite(d->beta[l])) return set_err(QED_EINVAL, "parameters must be finite");
  }
  return rebuild_tables(d);
}

// d log Z / d theta by a reverse pass over the F recursion.
static void dlogz(const qed_diag *d, std::vector<double> &ga, std::vector<double> &gb) {
  const int N = d->N;
  const size_t M = size_t(1) << N;
  const std::vector<double> &D = d->deg, &F = d->F;
  std::vector<double> Fb(M, 0.0), Db(M, 0.0);
  const double Z = F[M - 1];
  ga.assign(N, 0.0);
  gb.assign(N, 0.0);
  for (int j = 0; j < N; ++j) {
    const size_t r = (M - 1) & ~(size_t(1) << j);
    const double e = std::exp(d->beta[j]) / Z;
    Fb[r] += e / D[r];
    Db[r] -= e * F[r] / (D[r] * D[r]);
    gb[j] = e * F[r] / D[r];
  }
  // sets in decreasing size: F(S) = sum_j F(S\j) / D(S\j)
  std::vector<size_t> order;
  for (size_t m = 1; m + 1 < M; ++m) order.push_back(m);
  std::sort(order.begin(), order.end(), [](size_t a, size_t b) { return __builtin_popcountll(a) > __builtin_popcountll(b); });
  for (size_t m : order) {
    if (__builtin_popcountll(m) < 2 || Fb[m] == 0.0) continue;
    for (int j = 0; j < N; ++j) if (m >> j & 1) {
      const size_t r = m & ~(size_t(1) << j);
      Fb[r] += Fb[m] / D[r];
      Db[r] -= Fb[m] * F[r] / (D[r] * D[r]);
    }
  }
  for (size_t m = 1; m + 1 < M; ++m)
    if (d->act[m] && Db[m] != 0.0)
      for (int l = 0; l < N; ++l) if (m >> l & 1) ga[l] += Db[m];
}

extern "C" int qed_pdf_grad(qed_diag *d, uint64_t begin, uint64_t n, uint64_t seed, double *m2, double *grad) {
  if (!d || !m2 || !grad || n == 0) return set_err(QED_EINVAL, "bad argument");
  qed_ctx *c = d->ctx;
  CUDA_TRY(cudaSetDevice(c->device));
  const int N = d->N, W = 2 * N + 1;
  const bool vm = d->vm >= 0;
  // FP64 pass (flagged points queued) and double-double pass over the queue
  int blocks = 4 * c->sms, threads = 256, blocks2 = blocks, threads2 = threads;
  size_t smem = table_smem(N), smem2 = smem;
  VmLaunch L, L2;
  if (vm) {
    int rc = vm_launch(c, c->vm[d->vm], vm_kernels(d).grad, 0, c->vm_threads, L);
    if (!rc) rc = vm_launch(c, c->vm[d->vm], vm_kernels(d).grad_dd, 1, 64, L2);
    if (rc) return rc;
    blocks = L.blocks; threads = L.threads; smem = L.smem;
    blocks2 = L2.blocks; threads2 = L2.threads; smem2 = L2.smem;
  }
  const int B = std::max(blocks, blocks2);
  double *dout = nullptr;
  CUDA_TRY(cudaMalloc(&dout, sizeof(double) * size_t(B) * W));
  std::vector<double> h(size_t(B) * W), acc(W, 0.0);
  const uint8_t *act = d->d_act;
  auto collect = [&](int nb) -> int {
    cudaError_t e = cudaMemcpyAsync(h.data(), dout, size_t(nb) * W * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return set_err(QED_ECUDA, cudaGetErrorString(e));
    for (int b = 0; b < nb; ++b)
      for (int k = 0; k < W; ++k) acc[k] += h[size_t(b) * W + k];
    return QED_OK;
  };
  int rc = QED_OK;
  // launches of at most queue_cap samples: the flagged queue cannot overflow
  for (uint64_t off = 0; off < n && !rc; off += c->queue_cap) {
    const uint64_t m = std::min<uint64_t>(c->queue_cap, n - off);
    KParams P = base_params(d, begin + off, m, seed);
    P.queue = c->queue; P.queue_len = c->queue_len; P.queue_cap = c->queue_cap;
    if (cudaMemsetAsync(c->queue_len, 0, sizeof(unsigned int), c->stream) != cudaSuccess) { rc = set_err(QED_ECUDA, "memset"); break; }
    void *args[] = {&P, (void *)&act, &dout};
    void *vargs[] = {&P, &L.code, (void *)&act, &dout};
    rc = vm ? launch(vm_kernels(d).grad, blocks, threads, smem, c->stream, vargs)
            : launch(g_kernels[d->fid]->grad, blocks, threads, smem, c->stream, args);
    if (!rc) rc = collect(blocks);
    unsigned int qn = 0;
    if (!rc && cudaMemcpy(&qn, c->queue_len, sizeof qn, cudaMemcpyDeviceToHost) != cudaSuccess) rc = set_err(QED_ECUDA, "copy");
    if (!rc && qn > 0) {
      void *args2[] = {&P, &qn, (void *)&act, &dout};
      void *vargs2[] = {&P, &L2.code, &qn, (void *)&act, &dout};
      rc = vm ? launch(vm_kernels(d).grad_dd, blocks2, threads2, smem2, c->stream, vargs2)
              : launch(g_kernels[d->fid]->grad_dd, blocks2, threads2, smem2, c->stream, args2);
      if (!rc) rc = collect(blocks2);
    }
  }
  cudaFree(dout);
  if (rc) return rc;
  const double M2 = acc[0] / double(n);
  std::vector<double> ga, gb;
  dlogz(d, ga, gb);
  for (int m = 0; m < N; ++m) {
    grad[m] = -(acc[1 + m] / double(n) - M2 * ga[m]);
    grad[N + m] = -(acc[1 + N + m] / double(n) - M2 * gb[m]);
  }
  *m2 = M2;
  return QED_OK;
}

// ---------------------------------------------------------------------------
// Calibrated Deg: the growth exponent of the integrand in the limit where the
// lines of s shrink (z_s -> eps z_s), measured on the GPU in double-double,
// caps Deg(s) at |s| - a_s, the value at which w = f / p stays bounded in
// that limit.  Deg(s) = max(d_min, min(rule(s), |s| - a_s)).
// ---------------------------------------------------------------------------
extern "C" int qed_diagram_calibrate_deg(qed_diag *d, int n_base, uint64_t seed) {
  if (!d || n_base < 1 || n_base > 64) return set_err(QED_EINVAL, "n_base must be in [1, 64]");
  qed_ctx *c = d->ctx;
  const int N = d->N;
  const size_t M = size_t(1) << N;
  // far enough into the limit that the integrand follows its power law: at
  // 1e-4 .. 1e-5 some three-loop limits still show the bump of a nearby
  // scale, from 1e-6 on the measured exponents are the asymptotic ones
  const double e1 = 1e-6, e2 = 1e-8;
  // base points: uniform on the simplex (normalised exponentials)
  uint64_t st = seed * 0x9E3779B97F4A7C15ull + 0x2545F4914F6CDD1Dull;
  auto next = [&]() { st ^= st << 13; st ^= st >> 7; st ^= st << 17; return (double((st >> 11) + 1) * 1.1102230246251565e-16); };
  std::vector<double> base(size_t(n_base) * N);
  for (int b = 0; b < n_base; ++b) {
    double sum = 0.0;
    for (int l = 0; l < N; ++l) { base[b * N + l] = -std::log(next()); sum += base[b * N + l]; }
    for (int l = 0; l < N; ++l) base[b * N + l] /= sum;
  }
  const size_t npts = (M - 2) * size_t(n_base) * 2;
  std::vector<double> pts(npts * N), f(npts);
  size_t k = 0;
  for (size_t m = 1; m + 1 < M; ++m)
    for (int b = 0; b < n_base; ++b)
      for (double e : {e1, e2}) {
        for (int l = 0; l < N; ++l) pts[k * N + l] = base[b * N + l] * ((m >> l & 1) ? e : 1.0);
        ++k;
      }
  CUDA_TRY(cudaSetDevice(c->device));
  double *dz = nullptr, *df = nullptr;
  CUDA_TRY(cudaMalloc(&dz, pts.size() * sizeof(double)));
  if (cudaMalloc(&df, f.size() * sizeof(double)) != cudaSuccess) { cudaFree(dz); return set_err(QED_ENOMEM, "calibration buffers"); }
  int rc = QED_OK;
  if (cudaMemcpy(dz, pts.data(), pts.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) rc = set_err(QED_ECUDA, "copy");
  if (!rc) rc = qed_eval_points(d, dz, npts, 1, df);
  if (!rc && cudaMemcpy(f.data(), df, f.size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) rc = set_err(QED_ECUDA, "copy back");
  cudaFree(dz);
  cudaFree(df);
  if (rc) return rc;
  k = 0;
  for (size_t m = 1; m + 1 < M; ++m) {
    double a = -1e300;
    for (int b = 0; b < n_base; ++b) {
      const double f1 = std::fabs(f[k]), f2 = std::fabs(f[k + 1]);
      k += 2;
      if (f1 > 0.0 && f2 > 0.0 && std::isfinite(f1) && std::isfinite(f2))
        a = std::max(a, std::log(f2 / f1) / std::log(e1 / e2));
    }
    if (a > -1e299) {
      const double cap = double(__builtin_popcountll(m)) - a;
      d->deg0[m] = std::max(d->d_min, std::min(d->deg0[m], cap));
    }
  }
  return rebuild_tables(d);
}

extern "C" int qed_diagram_get_deg(const qed_diag *d, double *deg_out) {
  if (!d || !deg_out) return set_err(QED_EINVAL, "NULL argument");
  for (size_t m = 0; m < d->deg.size(); ++m) deg_out[m] = d->deg[m];
  return QED_OK;
}

// ---------------------------------------------------------------------------
// Integration without allocation (no counterpart in the paper).
//
// For callers that must not allocate device memory once they are running:
// for example an application that has handed all device memory to its own
// pool allocator and forbids further cudaMalloc, or a latency-critical loop
// where an allocation (which can synchronise the device) is not acceptable.
// The scratch of the FP64 integration kernel (block partials, the flagged
// queue and its counter) lives in one file-scope device array instead of
// context buffers, and the block partials are folded on the device, so the
// call allocates nothing on the device or the host.
// ---------------------------------------------------------------------------
#define QED_NOALLOC_MAX_BLOCKS 2048
#define QED_NOALLOC_QUEUE 65536
struct NoAllocScratch {
  double part[2][QED_NOALLOC_MAX_BLOCKS][QED_PART];       // FP64 pass, double-double pass
  unsigned long long cnt[2][QED_NOALLOC_MAX_BLOCKS][2];
  unsigned long long queue[QED_NOALLOC_QUEUE];
  double result[8];                                       // folded sums (see k_noalloc_fold)
  unsigned int queue_len;
};
static_assert(sizeof(NoAllocScratch) == 753736, "the header states this size");
// Every GPU that loads the library holds this array (753,736 bytes, about
// 736 KiB) from the moment the library's module is loaded on it until the
// process exits.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Folds the per-block partials of passes [p_begin, p_end) (0 = FP64, 1 =
// double-double) in block order, in double-double: result = {sum w (hi, lo),
// sum w^2 (hi, lo), flagged, unstable, sum |w| over the unstable points}.
__global__ void k_noalloc_fold(NoAllocScratch *s, int blocks, int p_begin, int p_end) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  dd x{0.0, 0.0}, y{0.0, 0.0};
  double uw = 0.0;
  unsigned long long nf = 0, nu = 0;
  for (int p = p_begin; p < p_end; ++p)
    for (int b = 0; b < blocks; ++b) {
      x = x + dd{s->part[p][b][0], s->part[p][b][1]};
      y = y + dd{s->part[p][b][2], s->part[p][b][3]};
      uw += s->part[p][b][4];
      nf += s->cnt[p][b][0];
      nu += s->cnt[p][b][1];
    }
  s->result[0] = x.hi; s->result[1] = x.lo; s->result[2] = y.hi; s->result[3] = y.lo;
  s->result[4] = double(nf); s->result[5] = double(nu); s->result[6] = uw;
}

static std::mutex g_noalloc_mu;
static NoAllocScratch *g_noalloc_ptr[64] = {nullptr};

// The array's device address on the current device (looked up once per
// device with that device current; the host-side name is only a stand-in).
static int noalloc_scratch(int device, NoAllocScratch **out) {
  if (device < 0 || device >= 64) return set_err(QED_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return set_err(QED_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_noalloc_ptr[device] = static_cast<NoAllocScratch *>(p);
  }
  *out = g_noalloc_ptr[device];
  return QED_OK;
}

extern "C" int qed_integrate_range_noalloc(qed_diag *d, uint64_t begin, uint64_t n, uint64_t seed, qed_result *out) {
  if (!d || !out) return set_err(QED_EINVAL, "diag/out is NULL");
  qed_ctx *c = d->ctx;
  if (d->vm >= 0) return set_err(QED_EINVAL, "qed_integrate_range_noalloc: compiled integrands only (this graph uses a bytecode program)");
  if (c->flag_rule != QED_FLAG_ESTIMATE) return set_err(QED_EINVAL, "qed_integrate_range_noalloc: estimate rule only");
  const int threads = c->threads;
  const int blocks = c->blocks > 0 ? c->blocks : 4 * c->sms;
  if (blocks > QED_NOALLOC_MAX_BLOCKS)
    return set_err(QED_EINVAL, "qed_integrate_range_noalloc: at most 2048 blocks (qed_ctx_set_launch)");
  CUDA_TRY(cudaSetDevice(c->device));
  NoAllocScratch *S = nullptr;
  int rc = noalloc_scratch(c->device, &S);
  if (rc) return rc;
  const KernelSet &K = *g_kernels[d->fid];
  const size_t smem = table_smem(d->N);
  qed_result r;
  std::memset(&r, 0, sizeof r);
  r.n = n;
  CUDA_TRY(cudaEventRecord(c->ev0, c->stream));
  const uint64_t chunk = uint64_t(1) << 30;
  for (uint64_t off = 0; off < n; off += chunk) {
    const uint64_t m = std::min(chunk, n - off);
    KParams P = base_params(d, begin + off, m, seed);
    P.partials = &S->part[0][0][0]; P.counts = &S->cnt[0][0][0];
    P.queue = S->queue; P.queue_len = &S->queue_len; P.queue_cap = QED_NOALLOC_QUEUE;
    CUDA_TRY(cudaMemsetAsync(&S->queue_len, 0, sizeof(unsigned int), c->stream));
    void *args[] = {&P};
    CUDA_TRY(cudaEventRecord(c->evk0, c->stream));
    if ((rc = launch(K.integrate, blocks, threads, smem, c->stream, args))) return rc;
    CUDA_TRY(cudaEventRecord(c->evk1, c->stream));
    ++r.launches;
    unsigned int qn = 0;
    CUDA_TRY(cudaMemcpyAsync(&qn, &S->queue_len, sizeof qn, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    float kms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&kms, c->evk0, c->evk1));
    r.kernel_seconds += kms * 1e-3;
    // passes to fold: the FP64 pass, plus the double-double pass over its
    // queue; on overflow the double-double kernel re-scans the whole chunk
    // and its pass alone replaces the first (one flag decision per point)
    int p_begin = 0, p_end = 1;
    bool dd_timed = false;
    if (qn > 0) {
      int mode = qn > QED_NOALLOC_QUEUE ? 1 : 0;
      unsigned int qcount = std::min<unsigned int>(qn, QED_NOALLOC_QUEUE);
      KParams P2 = P;
      P2.partials = &S->part[1][0][0]; P2.counts = &S->cnt[1][0][0];
      void *args2[] = {&P2, &mode, &qcount};
      CUDA_TRY(cudaEventRecord(c->evk1, c->stream));
      if ((rc = launch(K.redo, blocks, threads, smem, c->stream, args2))) return rc;
      CUDA_TRY(cudaEventRecord(c->evk2, c->stream));
      ++r.launches;
      p_begin = mode;
      p_end = 2;
      dd_timed = true;
    }
    void *args3[] = {&S, (void *)&blocks, &p_begin, &p_end};
    if ((rc = launch((const void *)k_noalloc_fold, 1, 32, 0, c->stream, args3))) return rc;
    double res[7];
    CUDA_TRY(cudaMemcpyAsync(res, S->result, sizeof res, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (dd_timed) {
      float dms = 0.f;
      CUDA_TRY(cudaEventElapsedTime(&dms, c->evk1, c->evk2));
      r.dd_seconds += dms * 1e-3;
    }
    dd_acc(r.sum_w[0], r.sum_w[1], res[0], res[1]);
    dd_acc(r.sum_w2[0], r.sum_w2[1], res[2], res[3]);
    r.n_flagged += (unsigned long long)res[4];
    r.n_unstable += (unsigned long long)res[5];
    r.unstable_abs_w += res[6];
  }
  CUDA_TRY(cudaEventRecord(c->ev1, c->stream));
  CUDA_TRY(cudaEventSynchronize(c->ev1));
  float ms = 0.f;
  CUDA_TRY(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
  r.seconds = ms * 1e-3;
  finish(&r);
  *out = r;
  return QED_OK;
}
