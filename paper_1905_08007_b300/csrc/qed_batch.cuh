// Batched integration of every graph of a loop order in one persistent
// launch (the scheduler of the hot path).
//
// Work items are (graph, first counter, count) blocks of samples.  Kernel 1
// (k_batch_fp64) is persistent: each block takes the next item from a device
// counter, stages that graph's Eq. (1) tables in shared memory, evaluates the
// item's samples in FP64 and writes one partial per item; flagged samples go
// to the item's own list in a fixed order (warp ballots and a block prefix
// sum, not atomics).  Kernel 2 (k_batch_dd) re-evaluates each item's list in
// double-double (bytecode batches: k_batch_vm_dd over full tiles of each
// graph's flagged points, between a plan and a per-item fold kernel; see
// qed_vm.cuh).  All partials are per item, so the host fold (items in index
// order) is deterministic whatever block ran an item.  The host sets the
// items of each round from the running per-graph variances (Neyman
// allocation) and replays a captured CUDA graph.
#pragma once
#include "qed_kernels.cuh"

struct BatchDiag {
  const double *F, *G, *inv, *off;
  double logZ;
  uint32_t stream;
  int fid;
  int N;
  int pad;
  // bytecode integrand (fid < 0): program, constants, their counts
  const uint2 *vins;
  const double *vkon;
  int vnk, vnr;
  uint32_t mrg[6];                  // MRG32k3a start state of this graph's stream
  uint32_t pad2[2];
};

struct BatchItem {
  uint64_t begin;
  uint32_t diag;
  uint32_t count;
};

struct BatchParams {
  const BatchDiag *diags;
  const BatchItem *items;
  unsigned int n_items;
  unsigned int *next_item;          // work counter, zeroed every round
  uint32_t key0, key1;
  double thresh;
  double *part;                     // [n_items][QED_PART]  FP64 moments
  unsigned long long *cnt;          // [n_items][2]  flagged, (unused)
  uint32_t *lists;                  // [n_items][list_cap] flagged offsets
  uint32_t list_cap;
  double *part_dd;                  // [n_items][QED_PART]  double-double moments (one partial per item)
  unsigned long long *cnt_dd;       // [n_items][2]  (unused), unstable
  uint32_t dd_tiles;                // double-double partials per item (1)
  unsigned int *next_tile;          // tile counter of the bytecode dd pass, zeroed every round
  uint32_t rng, mrg_bits;           // generator (0 Philox, 1 MRG32k3a), sample index bits
  const uint32_t *mrg_jump;         // MRG32k3a jump table
  // compacted double-double pass of bytecode batches: flat numbering of the
  // flagged points (item it's list starts at dd_start[it]), tiles that never
  // straddle two graphs, per-point results folded per item afterwards
  uint32_t *dd_start;               // [n_items + 1]
  uint4 *dd_tab;                    // [dd_tab_cap] (item holding the tile's first point, flat begin, flat end, segment end item)
  unsigned int *dd_ntiles;          // tiles of this round (written by the plan kernel)
  uint32_t dd_tab_cap, dd_tile;     // tile table capacity, points per tile (the dd kernel's block size)
  double *dd_w;                     // [n_items][list_cap] w of an accepted point
  double *dd_u;                     // [n_items][list_cap] -1 for an accepted point, else |w| (0 if not finite)
};

__device__ __forceinline__ KParams batch_kparams(const BatchParams &B, const BatchDiag &D) {
  KParams P;
  P.F = D.F; P.G = D.G; P.invdeg = D.inv; P.off = D.off;
  P.logZ = D.logZ;
  P.begin = 0; P.n = 0;
  P.key0 = B.key0; P.key1 = B.key1; P.stream = D.stream;
  P.thresh = B.thresh;
  P.partials = nullptr; P.counts = nullptr; P.queue = nullptr; P.queue_len = nullptr; P.queue_cap = 0;
  P.z_out = P.f_out = P.lp_out = nullptr; P.flag_out = nullptr;
  P.rng = B.rng; P.mrg_bits = B.mrg_bits; P.mrg_jump = B.mrg_jump;
#pragma unroll
  for (int i = 0; i < 6; ++i) P.mrg[i] = D.mrg[i];
  return P;
}

template <int FID, int N>
__device__ __forceinline__ void batch_item_fp64(const BatchParams &B, unsigned int it, const BatchItem &I,
                                                double *smem) {
  const BatchDiag &D = B.diags[I.diag];
  const KParams P = batch_kparams(B, D);
  double *sF = smem, *sG = smem + (1 << N), *sInv = smem + 2 * (1 << N);
  load_tables<N>(P, sF, sG, sInv);
  __shared__ unsigned int wcount[32];
  __shared__ unsigned int s_base;
  if (threadIdx.x == 0) s_base = 0;
  __syncthreads();
  KSum sw, sw2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (uint32_t off0 = 0; off0 < I.count; off0 += blockDim.x) {
    const uint32_t off = off0 + threadIdx.x;
    bool flagged = false;
    if (off < I.count) {
      double z[N];
      const double lp = draw_point<N>(I.begin + off, P, sF, sG, sInv, z);
      double absum;
      const double f = qed_gen_f<FID>::template eval<double>(z, absum);
      const double w = f * exp(-lp);
      if (!isfinite(w) || !(rel_err_estimate(f, absum, 1.1102230246251565e-16) <= P.thresh)) flagged = true;
      else { sw.add(w); sw2.add(w * w); }
    }
    // deterministic compaction of the flagged offsets
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
}

template <int FID, int N>
__device__ __forceinline__ void batch_item_dd(const BatchParams &B, unsigned int it, const BatchItem &I,
                                              double *smem) {
  const BatchDiag &D = B.diags[I.diag];
  const KParams P = batch_kparams(B, D);
  double *sF = smem, *sG = smem + (1 << N), *sInv = smem + 2 * (1 << N);
  load_tables<N>(P, sF, sG, sInv);
  const unsigned long long nflag = B.cnt[2 * size_t(it)];
  const bool overflow = nflag > B.list_cap;
  const uint64_t total = overflow ? uint64_t(I.count) : nflag;
  KSum sw, sw2;
  unsigned long long nflg = 0, nunst = 0;
  double uw = 0.0;
  for (uint64_t i = threadIdx.x; i < total; i += blockDim.x) {
    const uint32_t off = overflow ? uint32_t(i) : B.lists[size_t(it) * B.list_cap + i];
    double z[N];
    const double lp = draw_point<N>(I.begin + off, P, sF, sG, sInv, z);
    if (overflow) {
      // the list overflowed: this pass evaluates the whole item again and
      // replaces the FP64 pass's sums for it (the host uses this pass
      // alone), so each point is accepted or flagged by one decision
      double ab;
      const double f0 = qed_gen_f<FID>::template eval<double>(z, ab);
      const double w0 = f0 * exp(-lp);
      if (isfinite(w0) && rel_err_estimate(f0, ab, 1.1102230246251565e-16) <= P.thresh) {
        sw.add(w0);
        sw2.add(w0 * w0);
        continue;
      }
      ++nflg;
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
  block_reduce_store(sw, sw2, nflg, nunst, B.part_dd, B.cnt_dd, it, uw);
}

// The generated batch translation unit defines QED_BATCH_TU, includes every
// generated graph and defines the two dispatch functions (a switch over the
// graph ids); the kernels below then exist once, in that unit.
#ifdef QED_BATCH_TU
__device__ void batch_dispatch_fp64(const BatchParams &B, unsigned int it, const BatchItem &I, double *smem);
__device__ void batch_dispatch_dd(const BatchParams &B, unsigned int it, const BatchItem &I, double *smem);

__global__ void __launch_bounds__(256) k_batch_fp64(BatchParams B) {
  extern __shared__ double smem[];
  __shared__ unsigned int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(B.next_item, 1u);
    __syncthreads();
    const unsigned int it = s_item;
    __syncthreads();
    if (it >= B.n_items) break;
    const BatchItem I = B.items[it];
    batch_dispatch_fp64(B, it, I, smem);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_batch_dd(BatchParams B) {
  extern __shared__ double smem[];
  for (unsigned int it = blockIdx.x; it < B.n_items; it += gridDim.x) {
    const BatchItem I = B.items[it];
    if (B.cnt[2 * size_t(it)] == 0) {
      if (threadIdx.x == 0) {
        double *p = B.part_dd + QED_PART * size_t(it);
        p[0] = p[1] = p[2] = p[3] = p[4] = 0.0;
        B.cnt_dd[2 * size_t(it)] = 0;
        B.cnt_dd[2 * size_t(it) + 1] = 0;
      }
      continue;
    }
    batch_dispatch_dd(B, it, I, smem);
    __syncthreads();
  }
}

extern const void *const qed_batch_kernels[2];
const void *const qed_batch_kernels[2] = {(const void *)k_batch_fp64, (const void *)k_batch_dd};
#endif
