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

enum VmOp : uint32_t { VM_END = 0, VM_LD, VM_ADD, VM_MUL, VM_FMA, VM_FMAC, VM_RCP, VM_ABS, VM_ST, VM_ACCW, VM_LDMUL };
#define VM_KFLAG 512u

struct VmCode {
  const uint32_t *ins;    // instruction words, END-padded to a multiple of 4
  const double *kon;      // constants
  int n_kon, n_regs;
};

// Smallest magnitude of a forest term's block value that the FP32 e lane
// represents with margin: below it, parts of the absolute sum may have
// underflowed, and the point is handed to the double-double pass (whose e
// lane is double).
#define VM_E_FLOOR 1e-30f

template <class R> struct VmE;
template <> struct VmE<double> { typedef float T; };
template <> struct VmE<dd> { typedef double T; };

__device__ __forceinline__ double vm_mag(double x) { return fabs(x); }
__device__ __forceinline__ double vm_mag(dd x) { return fabs(x.hi + x.lo); }
__device__ __forceinline__ double vm_fma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ dd vm_fma(dd a, dd b, dd c) { return a * b + c; }
__device__ __forceinline__ double vm_rcp(double a) { return 1.0 / a; }
__device__ __forceinline__ dd vm_rcp(dd a) { return dd(1.0) / a; }
template <class E> __device__ __forceinline__ E vm_abs_e(double m);
template <> __device__ __forceinline__ float vm_abs_e<float>(double m) { return float(m); }
template <> __device__ __forceinline__ double vm_abs_e<double>(double m) { return m; }

// Evaluate one program for this thread's point (already in R[0..N)).
// kv/ke: constants and their magnitudes (shared memory); rv/re: this
// thread's register file (shared memory, stride T).  Returns the integrand;
// absum receives its monomial absolute sum (+inf when the FP32 lane lost
// range, which flags the point).
template <class R>
__device__ __forceinline__ R vm_run(const uint32_t *__restrict__ ins, const double *__restrict__ kv,
                                    const typename VmE<R>::T *__restrict__ ke, R *__restrict__ rv,
                                    typename VmE<R>::T *__restrict__ re, int T, double &absum) {
  typedef typename VmE<R>::T E;
  R acc(0.0);
  E ae = E(0);
  double W = 0.0;
  auto get = [&](uint32_t a, R &v, E &e) {
    if (a >= VM_KFLAG) { v = R(kv[a - VM_KFLAG]); e = ke[a - VM_KFLAG]; }
    else { v = rv[a * T]; e = re[a * T]; }
  };
  // the next group of four words is loaded while this one executes (the
  // host leaves at least 16 readable bytes after every program)
  const uint4 *p = reinterpret_cast<const uint4 *>(ins);
  uint4 qn = __ldg(p);
  for (;; ++p) {
    const uint4 q = qn;
    qn = __ldg(p + 1);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t w = j == 0 ? q.x : (j == 1 ? q.y : (j == 2 ? q.z : q.w));
      const uint32_t op = w & 15u, a = (w >> 4) & 1023u, b = (w >> 14) & 1023u;
      R va, vb;
      E ea, eb;
      switch (op) {
        case VM_END:
          absum = W;
          return acc;
        case VM_LD: get(a, acc, ae); break;
        case VM_ADD: get(a, va, ea); acc = acc + va; ae = ae + ea; break;
        case VM_MUL: get(a, va, ea); acc = acc * va; ae = ae * ea; break;
        case VM_FMA: get(a, va, ea); get(b, vb, eb); acc = vm_fma(acc, va, vb); ae = ae * ea + eb; break;
        case VM_FMAC: get(a, va, ea); get(b, vb, eb); acc = vm_fma(va, vb, acc); ae = ea * eb + ae; break;
        case VM_RCP: acc = vm_rcp(acc); ae = vm_abs_e<E>(vm_mag(acc)); break;
        case VM_ABS: ae = vm_abs_e<E>(vm_mag(acc)); break;
        case VM_ST: rv[a * T] = acc; re[a * T] = ae; break;
        case VM_ACCW:
          get(a, va, ea); get(b, vb, eb);
          // range guard of the FP32 lane: a block value whose absolute sum
          // is (near) underflow or overflow cannot bound the rounding error
          if (sizeof(E) == 4 && (!(double(eb) < 3.0e38) || (double(eb) < double(VM_E_FLOOR) && vm_mag(vb) != 0.0)))
            W = __longlong_as_double(0x7ff0000000000000ll);
          else
            W = fma(vm_mag(va), double(eb), W);
          break;
        case VM_LDMUL: get(a, va, ea); get(b, vb, eb); acc = va * vb; ae = ea * eb; break;
        default: break;
      }
    }
  }
}

// Shared-memory layout of a VM kernel: constants (value, magnitude), then the
// register files (value lanes, then e lanes).
template <class R>
__host__ __device__ __forceinline__ size_t vm_smem_bytes(int n_kon, int n_regs, int T) {
  typedef typename VmE<R>::T E;
  const size_t k = (size_t(n_kon) * (sizeof(double) + sizeof(E)) + 15) & ~size_t(15);
  return k + size_t(n_regs) * T * (sizeof(R) + sizeof(E));
}

template <class R>
struct VmFrame {
  typedef typename VmE<R>::T E;
  const double *kv;
  const E *ke;
  R *rv;
  E *re;
  int T;
  __device__ __forceinline__ void setup(const VmCode &C, unsigned char *smem) {
    double *k = reinterpret_cast<double *>(smem);
    E *kabs = reinterpret_cast<E *>(smem + size_t(C.n_kon) * sizeof(double));
    for (int i = threadIdx.x; i < C.n_kon; i += blockDim.x) {
      const double c = C.kon[i];
      k[i] = c;
      kabs[i] = E(fabs(c));
    }
    const size_t off = (size_t(C.n_kon) * (sizeof(double) + sizeof(E)) + 15) & ~size_t(15);
    T = blockDim.x;
    R *rbase = reinterpret_cast<R *>(smem + off);
    E *ebase = reinterpret_cast<E *>(smem + off + size_t(C.n_regs) * T * sizeof(R));
    kv = k;
    ke = kabs;
    rv = rbase + threadIdx.x;
    re = ebase + threadIdx.x;
    __syncthreads();
  }
  template <int N>
  __device__ __forceinline__ R eval(const VmCode &C, const R *z, double &absum) {
#pragma unroll
    for (int i = 0; i < N; ++i) { rv[i * T] = z[i]; re[i * T] = E(vm_mag(z[i])); }
    return vm_run<R>(C.ins, kv, ke, rv, re, T, absum);
  }
};

// ---------------------------------------------------------------------------
// kernels (the Eq. (1) tables are read from global memory: at N = 12 they
// are 96 KB, and shared memory holds the register files)
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(256) k_integrate_vm(KParams P, VmCode C) {
  extern __shared__ __align__(16) unsigned char vsm[];
  VmFrame<double> fr;
  fr.setup(C, vsm);
  KSum sw, sw2;
  unsigned long long nflag = 0;
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < P.n; i += stride) {
    const uint64_t s = P.begin + i;
    double z[N];
    const double lp = draw_point<N>(s, P, P.F, P.G, P.invdeg, z);
    double absum;
    const double f = fr.eval<N>(C, z, absum);
    const double w = f * exp(-lp);
    const bool bad = !isfinite(w) || !(rel_err_estimate(f, absum, 1.1102230246251565e-16) <= P.thresh);
    if (bad) {
      ++nflag;
      const unsigned int slot = atomicAdd(P.queue_len, 1u);
      if (slot < P.queue_cap) P.queue[slot] = i;
    } else {
      sw.add(w);
      sw2.add(w * w);
    }
  }
  block_reduce_store(sw, sw2, nflag, 0ull, P.partials, P.counts, blockIdx.x);
}

// Double-double re-evaluation of the queued samples (offsets from P.begin).
// A queue overflow is handled on the host by re-collecting the flagged
// offsets of sub-ranges no longer than the queue.
template <int N>
__global__ void __launch_bounds__(256) k_redo_dd_vm(KParams P, VmCode C, unsigned int qn) {
  extern __shared__ __align__(16) unsigned char vsm[];
  VmFrame<dd> fr;
  fr.setup(C, vsm);
  KSum sw, sw2;
  unsigned long long nunst = 0;
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < qn; i += stride) {
    double z[N];
    const double lp = draw_point<N>(P.begin + P.queue[i], P, P.F, P.G, P.invdeg, z);
    dd zd[N];
#pragma unroll
    for (int L = 0; L < N; ++L) zd[L] = dd{z[L], 0.0};
    double absum;
    const dd f = fr.eval<N>(C, zd, absum);
    const double w = (f.hi + f.lo) * exp(-lp);
    if (!isfinite(w) || !(rel_err_estimate(f.hi, absum, 1.2325951644078309e-32) <= P.thresh)) {
      ++nunst;
      continue;
    }
    sw.add(w);
    sw2.add(w * w);
  }
  block_reduce_store(sw, sw2, 0ull, nunst, P.partials, P.counts, blockIdx.x);
}

template <int N>
__global__ void __launch_bounds__(256) k_dump_vm(KParams P, VmCode C) {
  extern __shared__ __align__(16) unsigned char vsm[];
  VmFrame<double> fr;
  fr.setup(C, vsm);
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < P.n; i += stride) {
    double z[N];
    const double lp = draw_point<N>(P.begin + i, P, P.F, P.G, P.invdeg, z);
    double absum;
    const double f = fr.eval<N>(C, z, absum);
    const double w = f * exp(-lp);
    uint8_t flag = 0;
    if (!(rel_err_estimate(f, absum, 1.1102230246251565e-16) <= P.thresh)) flag |= 1;
    if (!isfinite(w)) flag |= 2;
#pragma unroll
    for (int L = 0; L < N; ++L) P.z_out[i * N + L] = z[L];
    P.f_out[i] = f;
    P.lp_out[i] = lp;
    P.flag_out[i] = flag;
  }
}

// prec 0: FP64 (smem frame of doubles), prec 1: double-double
template <int N>
__global__ void __launch_bounds__(256) k_eval_vm(const double *__restrict__ zin, uint64_t n, int prec,
                                                 double *__restrict__ fout, VmCode C) {
  extern __shared__ __align__(16) unsigned char vsm[];
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  if (prec == 0) {
    VmFrame<double> fr;
    fr.setup(C, vsm);
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
      double z[N];
#pragma unroll
      for (int L = 0; L < N; ++L) z[L] = zin[i * N + L];
      double absum;
      fout[i] = fr.eval<N>(C, z, absum);
    }
  } else {
    VmFrame<dd> fr;
    fr.setup(C, vsm);
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
      dd z[N];
#pragma unroll
      for (int L = 0; L < N; ++L) z[L] = dd{zin[i * N + L], 0.0};
      double absum;
      const dd f = fr.eval<N>(C, z, absum);
      fout[i] = f.hi + f.lo;
    }
  }
}

// Adjoint of the second moment over recomputed samples (same sums as
// k_pdf_grad; the integrand is the program).  out: [gridDim.x][2N + 1].
template <int N>
__global__ void __launch_bounds__(256) k_pdf_grad_vm(KParams P, VmCode C, const uint8_t *__restrict__ act, double *out) {
  extern __shared__ __align__(16) unsigned char vsm[];
  VmFrame<double> fr;
  fr.setup(C, vsm);
  double m2 = 0.0, ga[N], gb[N];
#pragma unroll
  for (int m = 0; m < N; ++m) { ga[m] = 0.0; gb[m] = 0.0; }
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < P.n; i += stride) {
    double z[N], lt[N];
    int order[N];
    const double lp = draw_point<N, true>(P.begin + i, P, P.F, P.G, P.invdeg, z, order, lt);
    double absum;
    const double f = fr.eval<N>(C, z, absum);
    double w = f * exp(-lp);
    if (!isfinite(w)) w = 0.0;
    const double w2 = w * w;
    m2 += w2;
    double cum = 0.0;
    uint32_t S = (1u << N) - 1u;
#pragma unroll
    for (int r = 0; r < N; ++r) {
      if (r > 0) {
        S &= ~(1u << order[r - 1]);
        if (act[S]) cum += lt[r];
      }
#pragma unroll
      for (int m = 0; m < N; ++m) if (order[r] == m) ga[m] += w2 * cum;
    }
#pragma unroll
    for (int m = 0; m < N; ++m) if (order[0] == m) gb[m] += w2;
  }
  __shared__ double red[8][2 * N + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double v[2 * N + 1];
  v[0] = m2;
#pragma unroll
  for (int m = 0; m < N; ++m) { v[1 + m] = ga[m]; v[1 + N + m] = gb[m]; }
#pragma unroll
  for (int k = 0; k < 2 * N + 1; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0) red[warp][k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x < 2 * N + 1) {
    double acc = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) acc += red[w][threadIdx.x];
    out[size_t(blockIdx.x) * (2 * N + 1) + threadIdx.x] = acc;
  }
}

// ---------------------------------------------------------------------------
// batched integration of a set of bytecode graphs (one line count N): the
// same scheduler as k_batch_fp64 / k_batch_dd.  The flagged list of an item
// holds a whole chunk, so it never overflows and the dd pass needs no rescan.
// ---------------------------------------------------------------------------
template <int N>
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
    const KParams P = batch_kparams(B, D);
    const VmCode C = {D.vins, D.vkon, D.vnk, D.vnr};
    VmFrame<double> fr;
    fr.setup(C, vsm);
    if (threadIdx.x == 0) s_base = 0;
    __syncthreads();
    KSum sw, sw2;
    for (uint32_t off0 = 0; off0 < I.count; off0 += blockDim.x) {
      const uint32_t off = off0 + threadIdx.x;
      bool flagged = false;
      if (off < I.count) {
        double z[N];
        const double lp = draw_point<N>(I.begin + off, P, P.F, P.G, P.invdeg, z);
        double absum;
        const double f = fr.eval<N>(C, z, absum);
        const double w = f * exp(-lp);
        if (!isfinite(w) || !(rel_err_estimate(f, absum, 1.1102230246251565e-16) <= P.thresh)) flagged = true;
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
    block_reduce_store(sw, sw2, threadIdx.x == 0 ? (unsigned long long)s_base : 0ull, 0ull, B.part, B.cnt, it);
    __syncthreads();
  }
}

template <int N>
__global__ void __launch_bounds__(256) k_batch_vm_dd(BatchParams B) {
  extern __shared__ __align__(16) unsigned char vsm[];
  for (unsigned int it = blockIdx.x; it < B.n_items; it += gridDim.x) {
    const BatchItem I = B.items[it];
    const unsigned long long nflag = B.cnt[2 * size_t(it)];
    if (nflag == 0) {
      if (threadIdx.x == 0) {
        double *p = B.part_dd + 4 * size_t(it);
        p[0] = p[1] = p[2] = p[3] = 0.0;
        B.cnt_dd[2 * size_t(it)] = 0;
        B.cnt_dd[2 * size_t(it) + 1] = 0;
      }
      continue;
    }
    const BatchDiag &D = B.diags[I.diag];
    const KParams P = batch_kparams(B, D);
    const VmCode C = {D.vins, D.vkon, D.vnk, D.vnr};
    VmFrame<dd> fr;
    fr.setup(C, vsm);
    const uint64_t total = nflag < B.list_cap ? nflag : B.list_cap;
    KSum sw, sw2;
    unsigned long long nunst = 0;
    for (uint64_t i = threadIdx.x; i < total; i += blockDim.x) {
      const uint32_t off = B.lists[size_t(it) * B.list_cap + i];
      double z[N];
      const double lp = draw_point<N>(I.begin + off, P, P.F, P.G, P.invdeg, z);
      dd zd[N];
#pragma unroll
      for (int L = 0; L < N; ++L) zd[L] = dd{z[L], 0.0};
      double absum;
      const dd f = fr.eval<N>(C, zd, absum);
      const double w = (f.hi + f.lo) * exp(-lp);
      if (!isfinite(w) || !(rel_err_estimate(f.hi, absum, 1.2325951644078309e-32) <= P.thresh)) { ++nunst; continue; }
      sw.add(w);
      sw2.add(w * w);
    }
    block_reduce_store(sw, sw2, 0ull, nunst, B.part_dd, B.cnt_dd, it);
    __syncthreads();
  }
}

// Kernel table of the bytecode path for one line count.
struct VmKernelSet {
  const void *integrate, *redo, *dump, *eval, *grad, *batch64, *batchdd;
};
#define QED_VM_KSET(N)                                                                                       \
  VmKernelSet{(const void *)k_integrate_vm<N>, (const void *)k_redo_dd_vm<N>, (const void *)k_dump_vm<N>,   \
              (const void *)k_eval_vm<N>, (const void *)k_pdf_grad_vm<N>, (const void *)k_batch_vm_fp64<N>, \
              (const void *)k_batch_vm_dd<N>}
