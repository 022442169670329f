// Device side of qedmc: Philox4x32-10, the Eq. (1) point generator, the
// integration / re-evaluation / dump / evaluation kernels.  Each kernel is a
// template over the generated integrand id (FID) and the number of lines N;
// one translation unit per generated graph instantiates them
// (QED_DEFINE_KSET) so that the graphs compile in parallel.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "qed_dd.cuh"

template <int FID> struct qed_gen_f;   // specialised by the generated headers

// ---------------------------------------------------------------------------
// device: Philox4x32-10 and the uniform map
// ---------------------------------------------------------------------------
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ double u01(uint32_t hi, uint32_t lo) {
  // 52 random bits plus half a step: exactly representable, strictly in (0,1)
  const uint64_t x = ((uint64_t(hi) << 32) | uint64_t(lo)) >> 12;
  return (double(x) + 0.5) * 2.220446049250313080847e-16;   // 2^-52
}

// ---------------------------------------------------------------------------
// device: MRG32k3a (L'Ecuyer 1999; the paper's Calc 1 generator, Sec. 3)
//   x1[n] = (1403580 x1[n-2] - 810728 x1[n-3]) mod m1,   m1 = 2^32 - 209
//   x2[n] = (527612 x2[n-1] - 1370589 x2[n-3]) mod m2,   m2 = 2^32 - 22853
//   z = (x1[n] - x2[n]) mod m1 (z = 0 -> m1), u = z * (double nearest 1/(m1+1)).
// Sample s of a graph owns the 32 draws from position s * 2^5 of the
// graph's stream; the host gives the stream's start state (position
// seed * 2^127 + stream id * 2^96 from the all-12345 state) and a table of
// the jump matrices A^(2^(5+k)), k = 0..63, of both recurrences.  A thread
// jumps to its sample by the bits of s (one 3x3 product per bit, modulo m,
// on the integer pipe), then steps the recurrences draw by draw.
// ---------------------------------------------------------------------------
#define QED_MRG_M1 4294967087ull
#define QED_MRG_M2 4294944443ull

// x mod m1 for any 64-bit x: 2^32 = 209 (mod m1), folded twice
__device__ __forceinline__ uint32_t mrg_mod1(uint64_t x) {
  uint64_t t = (x >> 32) * 209ull + (x & 0xffffffffull);      // < 2^40
  t = (t >> 32) * 209ull + (t & 0xffffffffull);               // < 2^32 + 2^16 < 2 m1
  return uint32_t(t >= QED_MRG_M1 ? t - QED_MRG_M1 : t);
}
// x mod m2 for any 64-bit x: 2^32 = 22853 (mod m2), folded twice
__device__ __forceinline__ uint32_t mrg_mod2(uint64_t x) {
  uint64_t t = (x >> 32) * 22853ull + (x & 0xffffffffull);    // < 2^47
  t = (t >> 32) * 22853ull + (t & 0xffffffffull);             // < 2^32 + 2^30 < 2 m2
  return uint32_t(t >= QED_MRG_M2 ? t - QED_MRG_M2 : t);
}
// v <- A v (mod m) for a row-major 3x3 matrix A read from the jump table
template <int C>
__device__ __forceinline__ void mrg_matvec(const uint32_t *__restrict__ A, uint32_t (&v)[3]) {
  uint32_t r[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    uint64_t acc = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const uint64_t p = uint64_t(__ldg(A + 3 * i + k)) * v[k];
      acc += C == 1 ? mrg_mod1(p) : mrg_mod2(p);              // three terms < 3 m
    }
    r[i] = C == 1 ? mrg_mod1(acc) : mrg_mod2(acc);
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) v[i] = r[i];
}

struct KParams {
  const double *F;        // F(S), 2^N
  const double *G;        // F(S) / Deg(S), 2^N
  const double *invdeg;   // 1 / Deg(S), 2^N
  double logZ;            // log Z (normaliser of Eq. (1) with the sector weights)
  const double *off;      // [N] beta_j - log Z: log p offset of a point whose largest line is j
  uint64_t begin, n;
  uint32_t key0, key1, stream;
  double thresh;          // relative rounding-error threshold
  // outputs
  double *partials;       // [gridDim.x][QED_PART]: sum w (hi, lo), sum w^2 (hi, lo), unstable sum |w|
  unsigned long long *counts;   // [gridDim.x][2]: flagged, unstable
  unsigned long long *queue;    // flagged sample offsets
  unsigned int *queue_len;
  unsigned int queue_cap;
  // dump mode
  double *z_out, *f_out, *lp_out;
  uint8_t *flag_out;
  // random numbers: rng 0 = Philox4x32-10, 1 = MRG32k3a (stream start state
  // mrg[0..2] = x1, mrg[3..5] = x2; jump table [64][18]; sample indices
  // below 2^mrg_bits)
  uint32_t rng, mrg_bits;
  uint32_t mrg[6];
  const uint32_t *mrg_jump;
};

// The ND uniforms of sample s from MRG32k3a.
template <int ND>
__device__ __forceinline__ void mrg_draws(uint64_t s, const KParams &P, double (&u)[ND]) {
  uint32_t a[3] = {P.mrg[0], P.mrg[1], P.mrg[2]}, b[3] = {P.mrg[3], P.mrg[4], P.mrg[5]};
  for (uint32_t k = 0; k < P.mrg_bits; ++k) {
    if ((s >> k) & 1ull) {
      mrg_matvec<1>(P.mrg_jump + 18 * k, a);
      mrg_matvec<2>(P.mrg_jump + 18 * k + 9, b);
    }
  }
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    // 810728 x1[n-3] < 2^20 m1 and 1370589 x2[n-3] < 2^21 m2: no wrap
    const uint32_t p1 = mrg_mod1(1403580ull * a[1] + (QED_MRG_M1 << 20) - 810728ull * a[0]);
    const uint32_t p2 = mrg_mod2(527612ull * b[2] + (QED_MRG_M2 << 21) - 1370589ull * b[0]);
    a[0] = a[1]; a[1] = a[2]; a[2] = p1;
    b[0] = b[1]; b[1] = b[2]; b[2] = p2;
    const uint32_t z = p1 > p2 ? p1 - p2 : uint32_t(uint64_t(p1) + QED_MRG_M1 - p2);
    u[d] = double(z) * 2.328306549295727688e-10;        // the double nearest 1 / (m1 + 1)
  }
}

// Error model of the FP64 integrand: every monomial is computed to a few ulps
// and the sum loses log2(sum|m| / |sum m|) bits, so the relative error is
// about ulp * kappa with kappa = sum|m| / |f|; measured against an extended
// precision evaluation it stays below 2 ulp * kappa, and the factor 8 leaves
// room for that.
__device__ __forceinline__ double rel_err_estimate(double f, double absum, double ulp) {
  return 8.0 * ulp * absum / fabs(f);
}

// Draw the point of sample `s`: z[line] (largest component 1) and log p.
// Tables live in shared memory: sF (F), sG (F / Deg, with the sector weight
// folded into the sets of N-1 lines), sInv (1 / Deg), and sInv + 2^N holds
// the N first-line offsets beta_j - log Z.  With GRAD the sector order and
// log t_l (l = 1..N-1) are returned for the adjoint kernel.
template <int N, bool GRAD = false>
__device__ __forceinline__ double draw_point(uint64_t s, const KParams &P, const double *__restrict__ sF,
                                             const double *__restrict__ sG, const double *__restrict__ sInv,
                                             double *__restrict__ z, int *order_out = nullptr,
                                             double *logt_out = nullptr) {
  constexpr int ND = 2 * (N - 1);
  double u[ND];
  if (P.rng == 1) {
    mrg_draws<ND>(s, P, u);
  } else {
#pragma unroll
    for (int b = 0; b < (ND + 1) / 2; ++b) {
      U4 w = philox4x32_10(U4{uint32_t(s), uint32_t(s >> 32), P.stream, uint32_t(b)}, P.key0, P.key1);
      u[2 * b] = u01(w.x, w.y);
      if (2 * b + 1 < ND) u[2 * b + 1] = u01(w.z, w.w);
    }
  }
  const uint32_t full = (1u << N) - 1u;
  uint32_t S = full;
  int order[N];
#pragma unroll
  for (int l = 0; l < N - 1; ++l) {
    const double target = u[l] * sF[S];
    double cum = 0.0;
    int pick = -1, last = 0;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      if (pick < 0 && ((S >> j) & 1u)) {
        cum += sG[S & ~(1u << j)];
        last = j;
        if (target < cum) pick = j;
      }
    }
    if (pick < 0) pick = last;
    order[l] = pick;
    S &= ~(1u << pick);
  }
  order[N - 1] = __ffs(S) - 1;
  // radial variables: t_l = u^(1/Deg(S_l)), z_{j_l} = z_{j_(l-1)} t_l
  double lp = sInv[(1 << N) + order[0]], logx = 0.0;
  S = full;
  double xs[N];
  xs[0] = 1.0;
#pragma unroll
  for (int l = 1; l < N; ++l) {
    S &= ~(1u << order[l - 1]);
    const double lu = log(u[N - 1 + (l - 1)]);
    const double lt = lu * sInv[S];
    logx += lt;
    xs[l] = exp(logx);
    lp += lu - logx;
    if (GRAD) logt_out[l] = lt;
  }
  if (GRAD) {
#pragma unroll
    for (int l = 0; l < N; ++l) order_out[l] = order[l];
  }
  // scatter sector order -> line index with constant register indices
#pragma unroll
  for (int L = 0; L < N; ++L) {
    double v = 0.0;
#pragma unroll
    for (int l = 0; l < N; ++l) v = (order[l] == L) ? xs[l] : v;
    z[L] = v;
  }
  return lp;
}

template <int N>
__device__ __forceinline__ void load_tables(const KParams &P, double *sF, double *sG, double *sInv) {
  for (int i = threadIdx.x; i < (1 << N); i += blockDim.x) {
    sF[i] = P.F[i];
    sG[i] = P.G[i];
    sInv[i] = P.invdeg[i];
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) sInv[(1 << N) + i] = P.off[i];
  __syncthreads();
}

// Neumaier-compensated running sum
struct KSum {
  double s = 0.0, c = 0.0;
  __device__ __forceinline__ void add(double x) {
    const double t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x; else c += (x - t) + s;
    s = t;
  }
};

// Doubles per partial slot: sum w (hi, lo), sum w^2 (hi, lo), and the sum
// of |w| over the points that failed the threshold in double-double too.
#define QED_PART 5

// Reduce (hi, lo) pairs of a block into partials[slot] (slot = blockIdx.x
// for the per-graph kernels, the work-item index for the batched kernels).
// uw: this thread's sum of |w| over its unstable points (0 in FP64 passes).
__device__ __forceinline__ void block_reduce_store(KSum a, KSum b, unsigned long long nf, unsigned long long nu,
                                                   double *partials, unsigned long long *counts,
                                                   unsigned int slot, double uw = 0.0) {
  dd x = dd_from_sum(a.s, a.c), y = dd_from_sum(b.s, b.c);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dd xo{__shfl_down_sync(0xffffffffu, x.hi, o), __shfl_down_sync(0xffffffffu, x.lo, o)};
    dd yo{__shfl_down_sync(0xffffffffu, y.hi, o), __shfl_down_sync(0xffffffffu, y.lo, o)};
    x = x + xo;
    y = y + yo;
    nf += __shfl_down_sync(0xffffffffu, nf, o);
    nu += __shfl_down_sync(0xffffffffu, nu, o);
    uw += __shfl_down_sync(0xffffffffu, uw, o);
  }
  __shared__ double red[32][QED_PART];
  __shared__ unsigned long long redc[32][2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red[warp][0] = x.hi; red[warp][1] = x.lo; red[warp][2] = y.hi; red[warp][3] = y.lo; red[warp][4] = uw;
    redc[warp][0] = nf; redc[warp][1] = nu;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    dd X{0.0, 0.0}, Y{0.0, 0.0};
    double Uw = 0.0;
    unsigned long long F = 0, Un = 0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) {
      X = X + dd{red[w][0], red[w][1]};
      Y = Y + dd{red[w][2], red[w][3]};
      Uw += red[w][4];
      F += redc[w][0];
      Un += redc[w][1];
    }
    double *p = partials + QED_PART * size_t(slot);
    p[0] = X.hi; p[1] = X.lo; p[2] = Y.hi; p[3] = Y.lo; p[4] = Uw;
    counts[2 * size_t(slot)] = F;
    counts[2 * size_t(slot) + 1] = Un;
  }
  __syncthreads();   // red[] is reused by the next call in persistent loops
}

// Main FP64 kernel: grid-stride over samples [begin, begin + n).
template <int FID, int N>
__global__ void __launch_bounds__(256) k_integrate(KParams P) {
  extern __shared__ double smem[];
  double *sF = smem, *sG = smem + (1 << N), *sInv = smem + 2 * (1 << N);
  load_tables<N>(P, sF, sG, sInv);
  KSum sw, sw2;
  unsigned long long nflag = 0;
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < P.n; i += stride) {
    const uint64_t s = P.begin + i;
    double z[N];
    const double lp = draw_point<N>(s, P, sF, sG, sInv, z);
    double absum;
    const double f = qed_gen_f<FID>::template eval<double>(z, absum);
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

// Double-double re-evaluation of flagged samples.  mode 0: the queue holds
// the offsets the FP64 kernel flagged, and only they are summed here.
// mode 1 (the queue overflowed): a complete second pass over [0, n) that
// replaces the first one -- every point is evaluated in FP64 again, summed
// when its estimate passes and re-evaluated in double-double when it does
// not, and counted as flagged here -- so that every point is accepted or
// flagged by one decision taken in one kernel.
template <int FID, int N>
__global__ void __launch_bounds__(256) k_redo_dd(KParams P, int mode, unsigned int qn) {
  extern __shared__ double smem[];
  double *sF = smem, *sG = smem + (1 << N), *sInv = smem + 2 * (1 << N);
  load_tables<N>(P, sF, sG, sInv);
  KSum sw, sw2;
  unsigned long long nflag = 0, nunst = 0;
  double uw = 0.0;
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  const uint64_t total = mode == 0 ? uint64_t(qn) : P.n;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += stride) {
    const uint64_t off = mode == 0 ? P.queue[i] : i;
    const uint64_t s = P.begin + off;
    double z[N];
    const double lp = draw_point<N>(s, P, sF, sG, sInv, z);
    if (mode == 1) {
      double ab;
      const double f0 = qed_gen_f<FID>::template eval<double>(z, ab);
      const double w0 = f0 * exp(-lp);
      if (isfinite(w0) && rel_err_estimate(f0, ab, 1.1102230246251565e-16) <= P.thresh) {
        sw.add(w0);
        sw2.add(w0 * w0);
        continue;
      }
      ++nflag;
    }
    dd zd[N];
#pragma unroll
    for (int L = 0; L < N; ++L) zd[L] = dd{z[L], 0.0};
    double absum;
    const dd f = qed_gen_f<FID>::template eval<dd>(zd, absum);
    const double w = (f.hi + f.lo) * exp(-lp);
    if (!isfinite(w) || !(rel_err_estimate(f.hi, absum, 1.2325951644078309e-32) <= P.thresh)) {
      ++nunst;
      if (isfinite(w)) uw += fabs(w);
      continue;
    }
    sw.add(w);
    sw2.add(w * w);
  }
  block_reduce_store(sw, sw2, nflag, nunst, P.partials, P.counts, blockIdx.x, uw);
}

template <int FID, int N>
__global__ void __launch_bounds__(256) k_dump(KParams P) {
  extern __shared__ double smem[];
  double *sF = smem, *sG = smem + (1 << N), *sInv = smem + 2 * (1 << N);
  load_tables<N>(P, sF, sG, sInv);
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < P.n; i += stride) {
    double z[N];
    const double lp = draw_point<N>(P.begin + i, P, sF, sG, sInv, z);
    double absum;
    const double f = qed_gen_f<FID>::template eval<double>(z, absum);
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

template <int FID, int N>
__global__ void __launch_bounds__(256) k_eval(const double *__restrict__ zin, uint64_t n, int prec, double *__restrict__ fout) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    double absum;
    if (prec == 0) {
      double z[N];
#pragma unroll
      for (int L = 0; L < N; ++L) z[L] = zin[i * N + L];
      fout[i] = qed_gen_f<FID>::template eval<double>(z, absum);
    } else {
      dd z[N];
#pragma unroll
      for (int L = 0; L < N; ++L) z[L] = dd{zin[i * N + L], 0.0};
      const dd f = qed_gen_f<FID>::template eval<dd>(z, absum);
      fout[i] = f.hi + f.lo;
    }
  }
}


// Adjoint of the second moment M2 = E_p[w^2] with respect to the density's
// parameters (per-line Deg shifts alpha_m, first-level sector weights
// beta_m): accumulates, over samples recomputed from their Philox counters,
//   w^2,  w^2 * sum_{l: m in S_l, Deg(S_l) not clamped} log t_l,  w^2 [j_1 = m].
// The host adds the d log Z / d theta terms (reverse pass over the F table).
// The weights follow the estimator's rule: a point whose FP64 rounding-error
// estimate exceeds the threshold is queued and summed by k_pdf_grad_dd with
// its double-double value, and contributes w = 0 if it fails there too.
template <int N>
__device__ __forceinline__ void grad_add(double w2, const int *order, const double *lt,
                                         const uint8_t *__restrict__ act, double &m2, double *ga, double *gb) {
  m2 += w2;
  // cumulative sum over sector positions: line at position r gets
  // sum_{l=1..r} act(S_l) log t_l
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

// Block sums of (w^2, the N alpha sums, the N beta sums) in a fixed order
// (warp shuffles, then shared memory) into out[blockIdx.x][2N + 1].
template <int N>
__device__ __forceinline__ void grad_store(double m2, const double *ga, const double *gb, double *out) {
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

template <int FID, int N>
__global__ void __launch_bounds__(256) k_pdf_grad(KParams P, const uint8_t *__restrict__ act, double *out) {
  extern __shared__ double smem[];
  double *sF = smem, *sG = smem + (1 << N), *sInv = smem + 2 * (1 << N);
  load_tables<N>(P, sF, sG, sInv);
  double m2 = 0.0, ga[N], gb[N];
#pragma unroll
  for (int m = 0; m < N; ++m) { ga[m] = 0.0; gb[m] = 0.0; }
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < P.n; i += stride) {
    double z[N], lt[N];
    int order[N];
    const double lp = draw_point<N, true>(P.begin + i, P, sF, sG, sInv, z, order, lt);
    double absum;
    const double f = qed_gen_f<FID>::template eval<double>(z, absum);
    const double w = f * exp(-lp);
    if (!isfinite(w) || !(rel_err_estimate(f, absum, 1.1102230246251565e-16) <= P.thresh)) {
      const unsigned int slot = atomicAdd(P.queue_len, 1u);
      if (slot < P.queue_cap) P.queue[slot] = i;
      continue;
    }
    grad_add<N>(w * w, order, lt, act, m2, ga, gb);
  }
  grad_store<N>(m2, ga, gb, out);
}

// The flagged points of k_pdf_grad (offsets in P.queue[0..qn)) in double-double.
template <int FID, int N>
__global__ void __launch_bounds__(256) k_pdf_grad_dd(KParams P, unsigned int qn, const uint8_t *__restrict__ act,
                                                     double *out) {
  extern __shared__ double smem[];
  double *sF = smem, *sG = smem + (1 << N), *sInv = smem + 2 * (1 << N);
  load_tables<N>(P, sF, sG, sInv);
  double m2 = 0.0, ga[N], gb[N];
#pragma unroll
  for (int m = 0; m < N; ++m) { ga[m] = 0.0; gb[m] = 0.0; }
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < qn; i += stride) {
    double z[N], lt[N];
    int order[N];
    const double lp = draw_point<N, true>(P.begin + P.queue[i], P, sF, sG, sInv, z, order, lt);
    dd zd[N];
#pragma unroll
    for (int L = 0; L < N; ++L) zd[L] = dd{z[L], 0.0};
    double absum;
    const dd f = qed_gen_f<FID>::template eval<dd>(zd, absum);
    const double w = (f.hi + f.lo) * exp(-lp);
    if (!isfinite(w) || !(rel_err_estimate(f.hi, absum, 1.2325951644078309e-32) <= P.thresh)) continue;
    grad_add<N>(w * w, order, lt, act, m2, ga, gb);
  }
  grad_store<N>(m2, ga, gb, out);
}

// ---------------------------------------------------------------------------
// per-graph kernel set
// ---------------------------------------------------------------------------
struct KernelSet {
  const void *integrate, *redo, *dump, *eval, *grad, *grad_dd;
  int lines;
};
#define QED_DEFINE_KSET(id, lines)                                                              \
  extern const KernelSet qed_kset_##id;                                                        \
  const KernelSet qed_kset_##id = {(const void *)k_integrate<id, lines>, (const void *)k_redo_dd<id, lines>, \
                                   (const void *)k_dump<id, lines>, (const void *)k_eval<id, lines>,            \
                                   (const void *)k_pdf_grad<id, lines>, (const void *)k_pdf_grad_dd<id, lines>, \
                                   lines};
