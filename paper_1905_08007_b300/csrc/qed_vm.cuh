// Device side of the bytecode integrands: an accumulator-machine interpreter
// and the kernels that use it in place of a compiled integrand (graphs of four
// loops and up; the same programs exist for lower orders, for tests).
//
// Why an interpreter: the subtracted integrand of one 4-loop graph is ~1e5
// FP64 operations and the 5-loop set needs thousands of them (Sec. 3 of the
// paper: 500 GB of generated code).  On B300 the FP64 pipe retires about two
// lanes per clock per SM, while the SM issues four warp-instructions per
// clock; decoding one instruction word, reading its operands from shared
// memory and dispatching costs integer, load and branch issue slots that sit
// in the shadow of the FP64 operation each instruction carries.  One generic
// kernel per line count N then serves every graph, and a program is data
// (a few hundred KB in HBM/L2, read through the read-only cache as a
// warp-uniform stream).
//
// Machine (the generator's qed_vm_gen.hpp writes the programs):
//   per thread: accumulator (v, e), register file R[r] = (v, e) in shared
//   memory, laid out R[r * T + thread] so that a warp's access is
//   conflict-free; R[0..N) = z; a double W collecting the absolute sum.
//   v is double (FP64 path) or dd (double-double re-evaluation); e, the
//   absolute-value lane of the rounding-error estimate, is float on the FP64
//   path (the FP32 pipe is idle there) and double on the dd path.
//   Constants live in shared memory (value and |value|).
#pragma once
#include "qed_kernels.cuh"
#include "qed_batch.cuh"

// Instruction (64 bits, written by the generator's fuse step):
//   lo = A | B << 13,  hi = XA | ZO << 1 | SPEC << 2 | NOCOMP << 5 | D << 6
//   1. unless NOCOMP:  X = XA ? A : acc,  O = XA ? acc : A,
//                      acc = X * B + (ZO ? O : 0)          (e lane alike)
//   2. SPEC 1: acc = 1 / acc, e = |acc|;  2: e = |acc|;  3: W += |A.v| * B.e;
//      4: end
//   3. store acc in R[D] (D = 0: in the spare register)
// Operands A, B: a register index, or 4096 + a constant index.  Every
// instruction reads both operands (the generator names the constants 0 or 1
// where one is unused), so the common path has no branch on the operation.
#define VM_KFLAG 4096u
#define VM_SP_RCP 1u
#define VM_SP_ABS 2u
#define VM_SP_ACCW 3u
#define VM_SP_END 4u
#define VM_NOCOMP 32u

struct VmCode {
  const uint2 *ins;       // instructions (lo, hi), END-padded to an even count
  const double *kon;      // constants
  int n_kon, n_regs;
};

// Smallest magnitude of a forest term's block value that the FP32 e lane
// represents with margin: below it, parts of the absolute sum may have
// underflowed, and the point is handed to the double-double pass (whose e
// lane is double).
#define VM_E_FLOOR 1e-30f

// Interval of the FP64 interval pass (Sec. 3 controls the round-off of the
// numerical subtraction with interval arithmetic): every operation rounds
// its lower end down and its upper end up, so [lo, hi] encloses the exact
// value of the program's arithmetic at the point (with the program's FP64
// constants), whatever the cancellation between forest terms.
struct __align__(16) ivl {
  double lo, hi;
  __host__ __device__ ivl() : lo(0.0), hi(0.0) {}
  __host__ __device__ explicit ivl(double x) : lo(x), hi(x) {}
  __host__ __device__ ivl(double l, double h) : lo(l), hi(h) {}
};

template <class R> struct VmE;
template <> struct VmE<double> { typedef float T; };
template <> struct VmE<dd> { typedef double T; };
template <> struct VmE<ivl> { typedef float T; };   // not stored: an interval bounds its own error
template <class R> struct VmHasE { static constexpr bool value = true; };
template <> struct VmHasE<ivl> { static constexpr bool value = false; };

__device__ __forceinline__ double vm_mag(double x) { return fabs(x); }
__device__ __forceinline__ double vm_mag(dd x) { return fabs(x.hi + x.lo); }
__device__ __forceinline__ double vm_fma(double a, double b, double c) { return fma(a, b, c); }
// a * b + c in double-double, the one arithmetic step of the interpreter.
// General case: the exact product of the high parts (two-product), the
// cross terms a.hi b.lo + a.lo b.hi added to its low part (a.lo b.lo, below
// 2^-106 |a b|, dropped), one two-sum of the high parts, every low part
// folded into the sum's error term, one renormalisation: 15 FP64 operations
// instead of the 27 of a double-double product followed by a full
// double-double sum.  Its error is a few 2^-106 (|a b| + |c|), bounded by
// the operands' magnitudes rather than the result's -- the form the
// absolute-value lane sums up for the rounding-error estimate, so that
// estimate stays a bound under cancellation between forest terms.
// Two operand patterns skip work (tested on bit patterns, with integer
// compares; both are warp-uniform when the operand is a constant or the
// instruction has no addend, and give the same value as the general case
// would up to its rounding): c = 0 (loads and products, about 40 % of the
// instructions of a four-loop program) leaves the product alone, 7
// operations; b = 1 (moves and sums, about 20 %) leaves the sum alone, 11
// operations, or none for a move.
__device__ __forceinline__ bool vm_bits_zero(dd x) {
  return ((__double_as_longlong(x.hi) | __double_as_longlong(x.lo)) << 1) == 0;
}
__device__ __forceinline__ dd vm_fma(dd a, dd b, dd c) {
  if (__double_as_longlong(b.hi) == 0x3ff0000000000000ll && __double_as_longlong(b.lo) == 0) {
    if (vm_bits_zero(c)) return a;
    const dd s = two_sum(a.hi, c.hi);
    return quick_two_sum(s.hi, __dadd_rn(__dadd_rn(s.lo, a.lo), c.lo));
  }
  const double p = __dmul_rn(a.hi, b.hi);
  double pl = __fma_rn(a.hi, b.hi, -p);
  pl = __fma_rn(a.hi, b.lo, pl);
  pl = __fma_rn(a.lo, b.hi, pl);
  if (vm_bits_zero(c)) return quick_two_sum(p, pl);
  const dd s = two_sum(p, c.hi);
  return quick_two_sum(s.hi, __dadd_rn(__dadd_rn(s.lo, pl), c.lo));
}
// a * b + c in interval arithmetic: the bounds of the product are the
// products of the ends picked by the signs of a and b (all four candidates
// only where both straddle zero), each fused with the matching end of c and
// rounded outward (down for lo, up for hi) by the directed-rounding FMA.
// A NaN end (a product of zero and an infinite end) fails every sign test
// and propagates, and the point is flagged.
__device__ __forceinline__ double vm_mag(ivl x) { return fmax(fabs(x.lo), fabs(x.hi)); }
__device__ __forceinline__ ivl vm_fma(ivl a, ivl b, ivl c) {
  double l, h;
  if (b.lo >= 0.0) {
    if (a.lo >= 0.0)      { l = __fma_rd(a.lo, b.lo, c.lo); h = __fma_ru(a.hi, b.hi, c.hi); }
    else if (a.hi <= 0.0) { l = __fma_rd(a.lo, b.hi, c.lo); h = __fma_ru(a.hi, b.lo, c.hi); }
    else                  { l = __fma_rd(a.lo, b.hi, c.lo); h = __fma_ru(a.hi, b.hi, c.hi); }
  } else if (b.hi <= 0.0) {
    if (a.lo >= 0.0)      { l = __fma_rd(a.hi, b.lo, c.lo); h = __fma_ru(a.lo, b.hi, c.hi); }
    else if (a.hi <= 0.0) { l = __fma_rd(a.hi, b.hi, c.lo); h = __fma_ru(a.lo, b.lo, c.hi); }
    else                  { l = __fma_rd(a.hi, b.lo, c.lo); h = __fma_ru(a.lo, b.lo, c.hi); }
  } else if (b.lo < 0.0 && b.hi > 0.0) {
    if (a.lo >= 0.0)      { l = __fma_rd(a.hi, b.lo, c.lo); h = __fma_ru(a.hi, b.hi, c.hi); }
    else if (a.hi <= 0.0) { l = __fma_rd(a.lo, b.hi, c.lo); h = __fma_ru(a.lo, b.lo, c.hi); }
    else {
      l = fmin(__fma_rd(a.lo, b.hi, c.lo), __fma_rd(a.hi, b.lo, c.lo));
      h = fmax(__fma_ru(a.lo, b.lo, c.hi), __fma_ru(a.hi, b.hi, c.hi));
    }
  } else {
    l = h = __longlong_as_double(0x7ff8000000000000ll);   // b has a NaN end
  }
  if (!(a.lo <= a.hi)) l = h = __longlong_as_double(0x7ff8000000000000ll);
  return ivl(l, h);
}
__device__ __forceinline__ double vm_rcp(double a) { return 1.0 / a; }
__device__ __forceinline__ dd vm_rcp(dd a) { return dd(1.0) / a; }
// 1 / [lo, hi] = [1/hi, 1/lo] (rounded outward) when the interval excludes
// zero, else everything
__device__ __forceinline__ ivl vm_rcp(ivl a) {
  if (a.lo > 0.0 || a.hi < 0.0) return ivl(__drcp_rd(a.hi), __drcp_ru(a.lo));
  return ivl(-__longlong_as_double(0x7ff0000000000000ll), __longlong_as_double(0x7ff0000000000000ll));
}
template <class E> __device__ __forceinline__ E vm_abs_e(double m);
template <> __device__ __forceinline__ float vm_abs_e<float>(double m) { return float(m); }
template <> __device__ __forceinline__ double vm_abs_e<double>(double m) { return m; }

// P consecutive values at a shared-memory byte offset (vector loads where
// the layout makes them 8- or 16-byte aligned)
template <class T, int P> struct VmVec {
  __device__ static __forceinline__ void ld(const unsigned char *p, T (&v)[P]) {
#pragma unroll
    for (int i = 0; i < P; ++i) v[i] = reinterpret_cast<const T *>(p)[i];
  }
  __device__ static __forceinline__ void st(unsigned char *p, const T (&v)[P]) {
#pragma unroll
    for (int i = 0; i < P; ++i) reinterpret_cast<T *>(p)[i] = v[i];
  }
};
template <> struct VmVec<double, 2> {
  __device__ static __forceinline__ void ld(const unsigned char *p, double (&v)[2]) {
    const double2 x = *reinterpret_cast<const double2 *>(p);
    v[0] = x.x; v[1] = x.y;
  }
  __device__ static __forceinline__ void st(unsigned char *p, const double (&v)[2]) {
    *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
  }
};
template <> struct VmVec<float, 2> {
  __device__ static __forceinline__ void ld(const unsigned char *p, float (&v)[2]) {
    const float2 x = *reinterpret_cast<const float2 *>(p);
    v[0] = x.x; v[1] = x.y;
  }
  __device__ static __forceinline__ void st(unsigned char *p, const float (&v)[2]) {
    *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
  }
};

// Shared-memory frame of a block: a value region (the constants, each
// repeated P times, then the register files of n_regs + 1 registers, the
// last taking the stores of instructions without a target; register r of
// point p of thread t at ((r * T) + t) * P + p), then an e region laid out
// the same way at half the size (e is half as wide as the value in both
// frames), so that an e address is X + (value address) / 2.
template <class R, int P>
__host__ __device__ __forceinline__ size_t vm_value_bytes(int n_kon, int n_regs, int T) {
  return (size_t(n_kon) * P * sizeof(R) + size_t(n_regs + 1) * T * P * sizeof(R) + 15) & ~size_t(15);
}
template <class R, int P>
__host__ __device__ __forceinline__ size_t vm_smem_bytes(int n_kon, int n_regs, int T) {
  static_assert(!VmHasE<R>::value || 2 * sizeof(typename VmE<R>::T) == sizeof(R),
                "e lane is half the value width");
  const size_t v = vm_value_bytes<R, P>(n_kon, n_regs, T);
  return VmHasE<R>::value ? v + v / 2 : v;
}

template <class R, int P>
struct VmFrame {
  typedef typename VmE<R>::T E;
  unsigned char *sm;
  uint32_t ex;              // start of the e region
  uint32_t vt;              // this thread's register 0 (value lane)
  uint32_t vs;              // bytes from one register to the next
  uint32_t spare;
  __device__ __forceinline__ void setup(const VmCode &C, unsigned char *smem) {
    sm = smem;
    const int T = blockDim.x;
    ex = uint32_t(vm_value_bytes<R, P>(C.n_kon, C.n_regs, T));
    R *k = reinterpret_cast<R *>(smem);
    E *kabs = reinterpret_cast<E *>(smem + ex);
    for (int i = threadIdx.x; i < C.n_kon * P; i += blockDim.x) {
      const double c = C.kon[i / P];
      k[i] = R(c);
      if (VmHasE<R>::value) kabs[i] = E(fabs(c));
    }
    const uint32_t v0 = uint32_t(C.n_kon) * P * sizeof(R);
    vs = uint32_t(T) * P * sizeof(R);
    vt = v0 + threadIdx.x * P * sizeof(R);
    spare = uint32_t(C.n_regs);
    __syncthreads();
  }
  __device__ __forceinline__ void put(uint32_t r, const R (&v)[P], const E (&e)[P]) {
    const uint32_t vo = vt + r * vs;
    VmVec<R, P>::st(sm + vo, v);
    if (VmHasE<R>::value) VmVec<E, P>::st(sm + ex + (vo >> 1), e);
  }
  __device__ __forceinline__ void get(uint32_t a, R (&v)[P], E (&e)[P]) const {
    const uint32_t i = a & (VM_KFLAG - 1u);
    const uint32_t vo = a >= VM_KFLAG ? i * uint32_t(P * sizeof(R)) : vt + a * vs;
    VmVec<R, P>::ld(sm + vo, v);
    if (VmHasE<R>::value) VmVec<E, P>::ld(sm + ex + (vo >> 1), e);
    else {
#pragma unroll
      for (int p = 0; p < P; ++p) e[p] = E(0);
    }
  }

  // One instruction whose operands are already loaded: compute, special,
  // store.  Returns true at END.
  __device__ __forceinline__ bool step(uint32_t lo, uint32_t hi, const R (&va)[P], const E (&ea)[P],
                                       const R (&vb)[P], const E (&eb)[P], R (&acc)[P], E (&ae)[P],
                                       double (&W)[P]) {
    if (!(hi & (VM_NOCOMP | (7u << 2)))) {        // the common case: compute and store
      const bool xa = hi & 1u, zo = (hi >> 1) & 1u;
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const R X = xa ? va[p] : acc[p], O = xa ? acc[p] : va[p];
        const E eX = xa ? ea[p] : ae[p], eO = xa ? ae[p] : ea[p];
        acc[p] = vm_fma(X, vb[p], zo ? O : R(0.0));
        if (VmHasE<R>::value) ae[p] = eX * eb[p] + (zo ? eO : E(0));
      }
      const uint32_t d = hi >> 6;
      // three quarters of the instructions of a four-loop program keep
      // their result in the accumulator only: the FP64 frame skips their
      // store (a predicated store, measured 4 % faster than storing to the
      // spare register; the wider frames store unconditionally)
      if (sizeof(R) != sizeof(double) || d) put(d ? d : spare, acc, ae);
      return false;
    }
    return step_slow(lo, hi, va, ea, vb, eb, acc, ae, W);
  }
  __device__ __forceinline__ bool step_slow(uint32_t lo, uint32_t hi, const R (&va)[P], const E (&ea)[P],
                                         const R (&vb)[P], const E (&eb)[P], R (&acc)[P], E (&ae)[P],
                                         double (&W)[P]) {
    if (!(hi & VM_NOCOMP)) {
      const bool xa = hi & 1u, zo = (hi >> 1) & 1u;
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const R X = xa ? va[p] : acc[p], O = xa ? acc[p] : va[p];
        const E eX = xa ? ea[p] : ae[p], eO = xa ? ae[p] : ea[p];
        acc[p] = vm_fma(X, vb[p], zo ? O : R(0.0));
        if (VmHasE<R>::value) ae[p] = eX * eb[p] + (zo ? eO : E(0));
      }
    }
    const uint32_t sp = (hi >> 2) & 7u;
    if (sp) {
      if (sp == VM_SP_END) return true;
#pragma unroll
      for (int p = 0; p < P; ++p) {
        if (sp == VM_SP_RCP) { acc[p] = vm_rcp(acc[p]); ae[p] = vm_abs_e<E>(vm_mag(acc[p])); }
        else if (!VmHasE<R>::value) {
        }
        else if (sp == VM_SP_ABS) ae[p] = vm_abs_e<E>(vm_mag(acc[p]));
        else if (sp == VM_SP_ACCW) {
          // range guard of the FP32 lane: a block value whose absolute sum
          // is (near) underflow or overflow cannot bound the error
          if (sizeof(E) == 4 && (!(double(eb[p]) < 3.0e38) ||
                                 (double(eb[p]) < double(VM_E_FLOOR) && vm_mag(vb[p]) != 0.0)))
            W[p] = __longlong_as_double(0x7ff0000000000000ll);
          else
            W[p] = fma(vm_mag(va[p]), double(eb[p]), W[p]);
        }
      }
    }
    const uint32_t d = hi >> 6;
    put(d ? d : spare, acc, ae);
    return false;
  }

  // Evaluate the program at the P points z[p][0..N): returns f[p] and the
  // monomial absolute sums absum[p] (+inf where the FP32 lane lost range,
  // which flags the point).  Software pipelined: the operands of the next
  // instruction are loaded before this one computes and stores (the
  // generator never lets an instruction read the register the previous one
  // writes), so shared-memory latency is off the chain through acc; the
  // instruction stream is loaded in blocks of four 16-byte groups (eight
  // instructions), one block ahead.  The host pads every program with zero
  // words to an even count plus eight zero groups, so every look-ahead
  // stays inside the program.
  template <int N>
  __device__ __forceinline__ void eval(const VmCode &C, const R (&z)[P][N], R (&f)[P], double (&absum)[P]) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      R v[P];
      E e[P];
#pragma unroll
      for (int p = 0; p < P; ++p) { v[p] = z[p][i]; e[p] = E(vm_mag(z[p][i])); }
      put(uint32_t(i), v, e);
    }
    R acc[P];
    E ae[P];
    double W[P];
#pragma unroll
    for (int p = 0; p < P; ++p) { acc[p] = R(0.0); ae[p] = E(0); W[p] = 0.0; }
    const uint4 *ip = reinterpret_cast<const uint4 *>(C.ins);
    uint4 g[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) g[j] = __ldg(ip + j);
    R va[P], vb[P], na[P], nb[P];
    E ea[P], eb[P], nea[P], neb[P];
    get(g[0].x & 8191u, va, ea);
    get((g[0].x >> 13) & 8191u, vb, eb);
    for (;; ip += 4) {
      uint4 h[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) h[j] = __ldg(ip + 4 + j);
      bool done = false;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        // slot 2j: (g[j].x, g[j].y), next operands (g[j].z)
        get(g[j].z & 8191u, na, nea);
        get((g[j].z >> 13) & 8191u, nb, neb);
        if (step(g[j].x, g[j].y, va, ea, vb, eb, acc, ae, W)) { done = true; break; }
        // slot 2j+1: (g[j].z, g[j].w), next operands: the following group's x
        const uint32_t nx = j < 3 ? g[j + 1].x : h[0].x;
        get(nx & 8191u, va, ea);
        get((nx >> 13) & 8191u, vb, eb);
        if (step(g[j].z, g[j].w, na, nea, nb, neb, acc, ae, W)) { done = true; break; }
      }
      if (done) break;
#pragma unroll
      for (int j = 0; j < 4; ++j) g[j] = h[j];
    }
#pragma unroll
    for (int p = 0; p < P; ++p) { f[p] = acc[p]; absum[p] = W[p]; }
  }
};

// ---------------------------------------------------------------------------
// kernels (the Eq. (1) tables are read from global memory: at N = 12 they
// are 96 KB, and shared memory holds the register files).  The FP64 kernels
// evaluate P points per thread with one instruction stream: sample i and
// i + (threads in the grid) for the per-graph kernels, offset o and
// o + blockDim for the batched one.  A point past the end of the range
// repeats the first one and is discarded.
// ---------------------------------------------------------------------------
template <int N, int P>
__global__ void __launch_bounds__(256) k_integrate_vm(KParams K, VmCode C) {
  extern __shared__ __align__(16) unsigned char vsm[];
  VmFrame<double, P> fr;
  fr.setup(C, vsm);
  KSum sw, sw2;
  unsigned long long nflag = 0;
  const uint64_t nth = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i0 = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i0 < K.n; i0 += nth * P) {
    double z[P][N], lp[P], f[P], ab[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const uint64_t i = i0 + p * nth;
      lp[p] = draw_point<N>(K.begin + (i < K.n ? i : i0), K, K.F, K.G, K.invdeg, z[p]);
    }
    fr.template eval<N>(C, z, f, ab);
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const uint64_t i = i0 + p * nth;
      if (i >= K.n) continue;
      const double w = f[p] * exp(-lp[p]);
      if (!isfinite(w) || !(rel_err_estimate(f[p], ab[p], 1.1102230246251565e-16) <= K.thresh)) {
        ++nflag;
        const unsigned int slot = atomicAdd(K.queue_len, 1u);
        if (slot < K.queue_cap) K.queue[slot] = i;
      } else {
        sw.add(w);
        sw2.add(w * w);
      }
    }
  }
  block_reduce_store(sw, sw2, nflag, 0ull, K.partials, K.counts, blockIdx.x);
}

// Double-double re-evaluation of the queued samples (offsets from K.begin).
template <int N>
__global__ void __launch_bounds__(256) k_redo_dd_vm(KParams K, VmCode C, unsigned int qn) {
  extern __shared__ __align__(16) unsigned char vsm[];
  VmFrame<dd, 1> fr;
  fr.setup(C, vsm);
  KSum sw, sw2;
  unsigned long long nunst = 0;
  double uw = 0.0;
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < qn; i += stride) {
    double z[N];
    const double lp = draw_point<N>(K.begin + K.queue[i], K, K.F, K.G, K.invdeg, z);
    dd zd[1][N], f[1];
    double ab[1];
#pragma unroll
    for (int L = 0; L < N; ++L) zd[0][L] = dd{z[L], 0.0};
    fr.template eval<N>(C, zd, f, ab);
    const double w = (f[0].hi + f[0].lo) * exp(-lp);
    if (!isfinite(w) || !(rel_err_estimate(f[0].hi, ab[0], 1.2325951644078309e-32) <= K.thresh)) {
      ++nunst;
      if (isfinite(w)) uw += fabs(w);
      continue;
    }
    sw.add(w);
    sw2.add(w * w);
  }
  block_reduce_store(sw, sw2, 0ull, nunst, K.partials, K.counts, blockIdx.x, uw);
}

template <int N, int P>
__global__ void __launch_bounds__(256) k_dump_vm(KParams K, VmCode C) {
  extern __shared__ __align__(16) unsigned char vsm[];
  VmFrame<double, P> fr;
  fr.setup(C, vsm);
  const uint64_t nth = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i0 = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i0 < K.n; i0 += nth * P) {
    double z[P][N], lp[P], f[P], ab[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const uint64_t i = i0 + p * nth;
      lp[p] = draw_point<N>(K.begin + (i < K.n ? i : i0), K, K.F, K.G, K.invdeg, z[p]);
    }
    fr.template eval<N>(C, z, f, ab);
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const uint64_t i = i0 + p * nth;
      if (i >= K.n) continue;
      const double w = f[p] * exp(-lp[p]);
      uint8_t flag = 0;
      if (!(rel_err_estimate(f[p], ab[p], 1.1102230246251565e-16) <= K.thresh)) flag |= 1;
      if (!isfinite(w)) flag |= 2;
#pragma unroll
      for (int L = 0; L < N; ++L) K.z_out[i * N + L] = z[p][L];
      K.f_out[i] = f[p];
      K.lp_out[i] = lp[p];
      K.flag_out[i] = flag;
    }
  }
}

// prec 0: FP64 with P points per thread; prec 1: double-double, one point
template <int N, int P>
__global__ void __launch_bounds__(256) k_eval_vm(const double *__restrict__ zin, uint64_t n, int prec,
                                                 double *__restrict__ fout, VmCode C) {
  extern __shared__ __align__(16) unsigned char vsm[];
  const uint64_t nth = uint64_t(gridDim.x) * blockDim.x;
  if (prec == 0) {
    VmFrame<double, P> fr;
    fr.setup(C, vsm);
    for (uint64_t i0 = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i0 < n; i0 += nth * P) {
      double z[P][N], f[P], ab[P];
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const uint64_t i = i0 + p * nth, src = i < n ? i : i0;
#pragma unroll
        for (int L = 0; L < N; ++L) z[p][L] = zin[src * N + L];
      }
      fr.template eval<N>(C, z, f, ab);
#pragma unroll
      for (int p = 0; p < P; ++p)
        if (i0 + p * nth < n) fout[i0 + p * nth] = f[p];
    }
  } else {
    VmFrame<dd, 1> fr;
    fr.setup(C, vsm);
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += nth) {
      dd z[1][N], f[1];
      double ab[1];
#pragma unroll
      for (int L = 0; L < N; ++L) z[0][L] = dd{zin[i * N + L], 0.0};
      fr.template eval<N>(C, z, f, ab);
      fout[i] = f[0].hi + f[0].lo;
    }
  }
}

// Adjoint of the second moment over recomputed samples (same sums as
// k_pdf_grad; the integrand is the program).  out: [gridDim.x][2N + 1].
// Adjoint sums of the second moment (see k_pdf_grad): points whose FP64
// estimate fails the threshold are queued for k_pdf_grad_dd_vm.
template <int N, int P>
__global__ void __launch_bounds__(256) k_pdf_grad_vm(KParams K, VmCode C, const uint8_t *__restrict__ act, double *out) {
  extern __shared__ __align__(16) unsigned char vsm[];
  VmFrame<double, P> fr;
  fr.setup(C, vsm);
  double m2 = 0.0, ga[N], gb[N];
#pragma unroll
  for (int m = 0; m < N; ++m) { ga[m] = 0.0; gb[m] = 0.0; }
  const uint64_t nth = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i0 = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i0 < K.n; i0 += nth * P) {
    double z[P][N], lt[P][N], lp[P], f[P], ab[P];
    int order[P][N];
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const uint64_t i = i0 + p * nth;
      lp[p] = draw_point<N, true>(K.begin + (i < K.n ? i : i0), K, K.F, K.G, K.invdeg, z[p], order[p], lt[p]);
    }
    fr.template eval<N>(C, z, f, ab);
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const uint64_t i = i0 + p * nth;
      if (i >= K.n) continue;
      const double w = f[p] * exp(-lp[p]);
      if (!isfinite(w) || !(rel_err_estimate(f[p], ab[p], 1.1102230246251565e-16) <= K.thresh)) {
        const unsigned int slot = atomicAdd(K.queue_len, 1u);
        if (slot < K.queue_cap) K.queue[slot] = i;
        continue;
      }
      grad_add<N>(w * w, order[p], lt[p], act, m2, ga, gb);
    }
  }
  grad_store<N>(m2, ga, gb, out);
}

// The queued points of k_pdf_grad_vm in double-double; a point that fails
// the threshold there too contributes w = 0, as in the estimator.
template <int N>
__global__ void __launch_bounds__(256) k_pdf_grad_dd_vm(KParams K, VmCode C, unsigned int qn,
                                                        const uint8_t *__restrict__ act, double *out) {
  extern __shared__ __align__(16) unsigned char vsm[];
  VmFrame<dd, 1> fr;
  fr.setup(C, vsm);
  double m2 = 0.0, ga[N], gb[N];
#pragma unroll
  for (int m = 0; m < N; ++m) { ga[m] = 0.0; gb[m] = 0.0; }
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < qn; i += stride) {
    double z[N], lt[N];
    int order[N];
    const double lp = draw_point<N, true>(K.begin + K.queue[i], K, K.F, K.G, K.invdeg, z, order, lt);
    dd zd[1][N], f[1];
    double ab[1];
#pragma unroll
    for (int L = 0; L < N; ++L) zd[0][L] = dd{z[L], 0.0};
    fr.template eval<N>(C, zd, f, ab);
    const double w = (f[0].hi + f[0].lo) * exp(-lp);
    if (!isfinite(w) || !(rel_err_estimate(f[0].hi, ab[0], 1.2325951644078309e-32) <= K.thresh)) continue;
    grad_add<N>(w * w, order, lt, act, m2, ga, gb);
  }
  grad_store<N>(m2, ga, gb, out);
}

// ---------------------------------------------------------------------------
// batched integration of a set of bytecode graphs (one line count N): the
// same scheduler as k_batch_fp64 / k_batch_dd.  The flagged list of an item
// holds a whole chunk, so it never overflows and the dd pass needs no rescan.
// The list order is the order of the offsets, whatever P is.
// ---------------------------------------------------------------------------
template <int N, int P>
__global__ void __launch_bounds__(256) k_batch_vm_fp64(BatchParams B) {
  extern __shared__ __align__(16) unsigned char vsm[];
  __shared__ unsigned int s_item;
  __shared__ unsigned int wcount[32];
  __shared__ unsigned int s_base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(B.next_item, 1u);
    __syncthreads();
    const unsigned int it = s_item;
    __syncthreads();
    if (it >= B.n_items) break;
    const BatchItem I = B.items[it];
    const BatchDiag &D = B.diags[I.diag];
    const KParams K = batch_kparams(B, D);
    const VmCode C = {D.vins, D.vkon, D.vnk, D.vnr};
    VmFrame<double, P> fr;
    fr.setup(C, vsm);
    if (threadIdx.x == 0) s_base = 0;
    __syncthreads();
    KSum sw, sw2;
    for (uint32_t off0 = 0; off0 < I.count; off0 += blockDim.x * P) {
      double z[P][N], lp[P], f[P], ab[P];
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const uint32_t off = off0 + p * blockDim.x + threadIdx.x;
        lp[p] = draw_point<N>(I.begin + (off < I.count ? off : off0 + threadIdx.x < I.count ? off0 + threadIdx.x : 0),
                              K, K.F, K.G, K.invdeg, z[p]);
      }
      fr.template eval<N>(C, z, f, ab);
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const uint32_t off = off0 + p * blockDim.x + threadIdx.x;
        bool flagged = false;
        if (off < I.count) {
          const double w = f[p] * exp(-lp[p]);
          if (!isfinite(w) || !(rel_err_estimate(f[p], ab[p], 1.1102230246251565e-16) <= K.thresh)) flagged = true;
          else { sw.add(w); sw2.add(w * w); }
        }
        const unsigned int m = __ballot_sync(0xffffffffu, flagged);
        if (lane == 0) wcount[warp] = __popc(m);
        __syncthreads();
        unsigned int before = s_base, total = 0;
        for (int w = 0; w < nwarp; ++w) { if (w < warp) before += wcount[w]; total += wcount[w]; }
        if (flagged) {
          const unsigned int pos = before + __popc(m & ((1u << lane) - 1u));
          if (pos < B.list_cap) B.lists[size_t(it) * B.list_cap + pos] = off;
        }
        __syncthreads();
        if (threadIdx.x == 0) s_base += total;
        __syncthreads();
      }
    }
    block_reduce_store(sw, sw2, threadIdx.x == 0 ? (unsigned long long)s_base : 0ull, 0ull, B.part, B.cnt, it);
    __syncthreads();
  }
}

// The double-double pass of a bytecode batch, in three kernels:
//  1. k_batch_vm_dd_plan numbers the flagged points of the round in item
//     order (dd_start) and cuts each graph's points -- its items are
//     consecutive in the queue -- into tiles of dd_tile points, so that a
//     tile holds one program and every tile but a graph's last is full (the
//     double-double frame leaves room for one block per SM, and an item's
//     list alone fills a fraction of a block);
//  2. k_batch_vm_dd: blocks take tiles from a device counter, one point per
//     thread, and write each point's result to its list slot;
//  3. k_batch_vm_dd_fold: one warp per item folds its slots in list order
//     into the item's double-double partial, so the result does not depend
//     on which block ran which tile.
__global__ void k_batch_vm_dd_plan(BatchParams B) {
  if (threadIdx.x != 0) return;
  unsigned int t = 0;
  uint32_t flat = 0;
  unsigned int it = 0;
  while (it < B.n_items) {
    const uint32_t g = B.items[it].diag;
    const unsigned int seg0 = it;
    const uint32_t f0 = flat;
    for (; it < B.n_items && B.items[it].diag == g; ++it) {
      B.dd_start[it] = flat;
      const unsigned long long c = B.cnt[2 * size_t(it)];
      flat += uint32_t(c < B.list_cap ? c : B.list_cap);
    }
    unsigned int cur = seg0;                       // item holding flat point f
    for (uint32_t f = f0; f < flat && t < B.dd_tab_cap; f += B.dd_tile) {
      while (cur + 1 < it && B.dd_start[cur + 1] <= f) ++cur;
      const uint32_t e = flat - f < B.dd_tile ? flat : f + B.dd_tile;
      B.dd_tab[t++] = make_uint4(cur, f, e, it);
    }
  }
  B.dd_start[B.n_items] = flat;
  *B.dd_ntiles = t;
}

template <int N>
__global__ void __launch_bounds__(256) k_batch_vm_dd(BatchParams B) {
  extern __shared__ __align__(16) unsigned char vsm[];
  __shared__ unsigned int s_tile;
  const unsigned int n_tiles = *B.dd_ntiles;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(B.next_tile, 1u);
    __syncthreads();
    const unsigned int t = s_tile;
    __syncthreads();
    if (t >= n_tiles) break;
    const uint4 T = B.dd_tab[t];
    const BatchDiag &D = B.diags[B.items[T.x].diag];
    const KParams K = batch_kparams(B, D);
    const VmCode C = {D.vins, D.vkon, D.vnk, D.vnr};
    VmFrame<dd, 1> fr;
    fr.setup(C, vsm);
    const uint32_t p = T.y + threadIdx.x;
    if (p < T.z) {
      unsigned int it = T.x;
      while (it + 1 < T.w && B.dd_start[it + 1] <= p) ++it;
      const uint32_t pos = p - B.dd_start[it];
      const size_t slot = size_t(it) * B.list_cap + pos;
      const uint32_t off = B.lists[slot];
      double z[N];
      const double lp = draw_point<N>(B.items[it].begin + off, K, K.F, K.G, K.invdeg, z);
      dd zd[1][N], f[1];
      double ab[1];
#pragma unroll
      for (int L = 0; L < N; ++L) zd[0][L] = dd{z[L], 0.0};
      fr.template eval<N>(C, zd, f, ab);
      const double w = (f[0].hi + f[0].lo) * exp(-lp);
      if (!isfinite(w) || !(rel_err_estimate(f[0].hi, ab[0], 1.2325951644078309e-32) <= K.thresh)) {
        B.dd_w[slot] = 0.0;
        B.dd_u[slot] = isfinite(w) ? fabs(w) : 0.0;
      } else {
        B.dd_w[slot] = w;
        B.dd_u[slot] = -1.0;
      }
    }
    __syncthreads();     // the frame is set up again for the next tile
  }
}

// One 32-thread block per item.
__global__ void __launch_bounds__(32) k_batch_vm_dd_fold(BatchParams B) {
  const unsigned int it = blockIdx.x;
  if (it >= B.n_items) return;
  const unsigned long long c = B.cnt[2 * size_t(it)];
  const uint32_t total = uint32_t(c < B.list_cap ? c : B.list_cap);
  KSum sw, sw2;
  unsigned long long nunst = 0;
  double uw = 0.0;
  for (uint32_t pos = threadIdx.x; pos < total; pos += 32) {
    const size_t slot = size_t(it) * B.list_cap + pos;
    const double u = B.dd_u[slot];
    if (u < 0.0) {
      const double w = B.dd_w[slot];
      sw.add(w);
      sw2.add(w * w);
    } else {
      ++nunst;
      uw += u;
    }
  }
  block_reduce_store(sw, sw2, 0ull, nunst, B.part_dd, B.cnt_dd, it, uw);
}

// ---------------------------------------------------------------------------
// interval pass (Sec. 3: interval arithmetic with different precisions
// removes the round-off of the numerical subtraction).  Each point is
// evaluated in FP64 interval arithmetic; its value is the midpoint of
// [lo, hi], accepted when both ends have one sign and
// hi - lo <= 2 thresh min(|lo|, |hi|), which bounds the relative error of the
// midpoint against every value in the interval by thresh.  Other points go
// to the flagged queue and are re-evaluated in double-double (k_redo_dd_vm).
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool ivl_accept(ivl f, double thresh, double &mid) {
  mid = 0.5 * f.lo + 0.5 * f.hi;
  const double m = fmin(fabs(f.lo), fabs(f.hi));
  return (f.lo > 0.0 || f.hi < 0.0) && (f.hi - f.lo) <= 2.0 * thresh * m;
}

template <int N>
__global__ void __launch_bounds__(256) k_eval_vm_ivl(const double *__restrict__ zin, uint64_t n,
                                                     double *__restrict__ lo, double *__restrict__ hi, VmCode C) {
  extern __shared__ __align__(16) unsigned char vsm[];
  VmFrame<ivl, 1> fr;
  fr.setup(C, vsm);
  const uint64_t nth = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += nth) {
    ivl z[1][N], f[1];
    double ab[1];
#pragma unroll
    for (int L = 0; L < N; ++L) z[0][L] = ivl(zin[i * N + L]);
    fr.template eval<N>(C, z, f, ab);
    lo[i] = f[0].lo;
    hi[i] = f[0].hi;
  }
}

template <int N>
__global__ void __launch_bounds__(256) k_integrate_vm_ivl(KParams K, VmCode C) {
  extern __shared__ __align__(16) unsigned char vsm[];
  VmFrame<ivl, 1> fr;
  fr.setup(C, vsm);
  KSum sw, sw2;
  unsigned long long nflag = 0;
  const uint64_t nth = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < K.n; i += nth) {
    double z[N];
    const double lp = draw_point<N>(K.begin + i, K, K.F, K.G, K.invdeg, z);
    ivl zi[1][N], f[1];
    double ab[1];
#pragma unroll
    for (int L = 0; L < N; ++L) zi[0][L] = ivl(z[L]);
    fr.template eval<N>(C, zi, f, ab);
    double mid;
    const bool ok = ivl_accept(f[0], K.thresh, mid);
    const double w = mid * exp(-lp);
    if (!ok || !isfinite(w)) {
      ++nflag;
      const unsigned int slot = atomicAdd(K.queue_len, 1u);
      if (slot < K.queue_cap) K.queue[slot] = i;
    } else {
      sw.add(w);
      sw2.add(w * w);
    }
  }
  block_reduce_store(sw, sw2, nflag, 0ull, K.partials, K.counts, blockIdx.x);
}

// Kernel table of the bytecode path for one line count N and P points per
// thread in the FP64 kernels.
struct VmKernelSet {
  const void *integrate, *redo, *dump, *eval, *grad, *batch64, *batchdd, *grad_dd, *eval_ivl, *integrate_ivl;
};
#define QED_VM_KSET(N, P)                                                                                       \
  VmKernelSet{(const void *)k_integrate_vm<N, P>, (const void *)k_redo_dd_vm<N>, (const void *)k_dump_vm<N, P>, \
              (const void *)k_eval_vm<N, P>, (const void *)k_pdf_grad_vm<N, P>,                                 \
              (const void *)k_batch_vm_fp64<N, P>, (const void *)k_batch_vm_dd<N>,                              \
              (const void *)k_pdf_grad_dd_vm<N>, (const void *)k_eval_vm_ivl<N>,                                \
              (const void *)k_integrate_vm_ivl<N>}
