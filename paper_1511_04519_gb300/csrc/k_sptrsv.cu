// Multi-right-hand-side supernodal triangular solves with the once-factorised
// M = L D L^T: the operator apply of Alg. 1, one forward and one backward
// substitution per Arnoldi step (here X1 = C + gamma G or G, both SPD, so the
// upper factor is D L^T).
//
// Layout: the right-hand sides live node-major in Y[n][ldy] (permuted node
// order), so the K columns of one row are contiguous.  The forward result y
// goes to a second buffer Y2 of the same shape, because the tasks of one
// supernode read b_s while their siblings write y_s; the backward reads y_s
// from Y2 and writes x into Y.  Each supernode s
// carries the panel P_s = [L_ss^{-1}; L_Rs L_ss^{-1}] built at setup, which
// turns both substitutions inside a supernode into dense products:
//   forward : [y_s; u_R] = P_s b_s, then b_R -= u_R (FP64 atomics into the
//             ancestors' rows, which a later level reads);
//   backward: x_s = P_s^T [D_s^{-1} y_s; -x_R], pulling the ancestors' final
//             x_R (solved one level up).
// One launch covers one level of the supernodal elimination tree (or one
// persistent launch covers all levels).  A task is (supernode, 32 panel rows
// or columns) x (column block of KB right-hand sides) with four threads per
// panel row/column, or a pack of small supernodes of one level.  In a split
// task the four threads of a row either share its panel entries (each holds
// all KB columns; partials added through shared memory) or, from KB = 8,
// share out its columns (KB/4 each, no partial sums).  Packed tasks run one
// thread per row/column or warp-wide (row, column-of-Y) chunks, chosen per
// level at setup (the task's count carries the choice).
#include "kernels.h"

#include <algorithm>
#include <mutex>

namespace matex {

namespace {

constexpr int kSolveThreads = 128;
constexpr int kSplit = kSolveThreads / kRowBlock;  // threads sharing one dot product

// Sum of the kSplit partial dot products of every (row, column) pair of a
// task through shared memory: each partial is added once, instead of a
// shuffle butterfly whose adds run on every lane.  `part` (the task's staging
// buffer, no longer read once the first barrier has passed) must hold
// kSolveThreads * (KB + 1) doubles.  out(r, q, v) receives the sum of pair
// (r, q), r < rows; consecutive threads take consecutive q of one row.
template <int KB, typename Out>
__device__ __forceinline__ void split_sum(const double (&acc)[KB], double* part, int rows, Out out) {
  constexpr int ld = KB + 1;  // padded: the writes below hit distinct banks
  __syncthreads();
#pragma unroll
  for (int q = 0; q < KB; ++q) part[threadIdx.x * ld + q] = acc[q];
  __syncthreads();
  for (int o = threadIdx.x; o < rows * KB; o += blockDim.x) {
    const int r = o / KB, q = o - r * KB;
    const double* p = part + r * kSplit * ld + q;
    out(r, q, (p[0] + p[ld]) + (p[2 * ld] + p[3 * ld]));
  }
}

// One CTA's share of a split task: chunk c of n over the task's reduction,
// with the scratch slot of its (task, column block) when n > 1.
struct Chunk {
  int c = 0, n = 1;
  double* part = nullptr;
  int* cnt = nullptr;
  int slot = 0;
};

// [a, b) = chunk ch of the range [lo, hi), chunk widths rounded up to 16 so
// that the four-load steps of the dot products stay whole
__device__ __forceinline__ void chunk_range(Chunk ch, int lo, int hi, int& a, int& b) {
  if (ch.n == 1) { a = lo; b = hi; return; }
  const int span = ((hi - lo + ch.n - 1) / ch.n + 15) & ~15;
  a = min(hi, lo + ch.c * span);
  b = min(hi, a + span);
}

// Partial sums of the task's `rows` x KB outputs are in part[slot][chunk];
// every thread has written its share.  The CTA that completes the slot's
// count adds the chunks in order and hands each sum to out(r, q, v).
template <int KB, typename Out>
__device__ __forceinline__ void chunk_finish(Chunk ch, int rows, Out out) {
  __shared__ int sh_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const int old = atomicAdd(ch.cnt + ch.slot, 1);
    sh_last = old == ch.n - 1;
  }
  __syncthreads();
  if (!sh_last) return;
  __threadfence();
  const double* base = ch.part + (int64_t)ch.slot * ch.n * kRowBlock * KB;
  for (int e = threadIdx.x; e < rows * KB; e += blockDim.x) {
    const int r = e / KB, q = e - r * KB;
    double v = 0.0;
    for (int c = 0; c < ch.n; ++c) v += __ldcg(base + ((int64_t)c * kRowBlock + r) * KB + q);
    out(r, q, v);
  }
  if (threadIdx.x == 0) ch.cnt[ch.slot] = 0;
}

__device__ __forceinline__ double* chunk_part(Chunk ch, int KB, int r, int q) {
  return ch.part + (((int64_t)ch.slot * ch.n + ch.c) * kRowBlock + r) * KB + q;
}

// Forward task: rows [i0, i0+32) of P_s b_s for KB right-hand sides, over the
// panel columns of chunk ch.  Thread (row, sub) accumulates all KB columns of
// its row over panel columns j = sub, sub+4, ..., so each panel entry is
// loaded once per task.  Loads of Y go through L2 only (__ldcg): other CTAs
// of a persistent launch write them.
template <int KB>
__device__ __forceinline__ void fwd_task(const DevFactor& F, int s, int i0, int c0,
                                         double* __restrict__ Y, double* __restrict__ Y2, int ldy,
                                         double* sb, Chunk ch) {
  const int f = F.sup_first[s];
  const int w = F.sup_first[s + 1] - f;
  const int64_t rp = F.sup_rowptr[s];
  const int ld = (int)(F.sup_rowptr[s + 1] - rp);  // w + r
  // L_ss^{-1} is lower triangular: rows below i0 + 32 of the diagonal block
  // have no entries right of column i0 + 32, so the block stops there
  const int jend = min(w, i0 + kRowBlock);
  int ja, jb;
  chunk_range(ch, 0, jend, ja, jb);
  for (int e = threadIdx.x; e < (jb - ja) * KB; e += blockDim.x) {
    const int j = e / KB, q = e - j * KB;
    sb[e] = __ldcg(Y + (int64_t)(f + ja + j) * ldy + c0 + q);
  }
  __syncthreads();
  const double* __restrict__ P = F.pan_cm + F.pan_off[s];
  const int sub = threadIdx.x % kSplit;
  const int i = i0 + threadIdx.x / kSplit;
  // the same bound per warp (its 8 rows), uniform across the warp
  const int jw = min(jb, i0 + (int)(threadIdx.x / 32 + 1) * (32 / kSplit));
  const int32_t* __restrict__ rows = F.sup_rows + rp;
  const int ndiag = max(0, min(kRowBlock, w - i0));  // rows of the block in the diagonal block
  if constexpr (KB >= 2 * kSplit) {
    // enough right-hand sides to share them out: thread `sub` of a row takes
    // KB / 4 of them (two or more independent FMA chains) over the whole row,
    // so no partial sums need adding
    constexpr int QS = KB / kSplit;
    const int qa = sub * QS;
    const double* bq = sb + qa - ja * KB;
    double acc[QS];
#pragma unroll
    for (int q = 0; q < QS; ++q) acc[q] = 0.0;
    if (i < ld) {
      const double* __restrict__ Pi = P + i;
      int j = ja;
      for (; j + 3 < jw; j += 4) {
        const double p0 = Pi[(int64_t)j * ld];
        const double p1 = Pi[(int64_t)(j + 1) * ld];
        const double p2 = Pi[(int64_t)(j + 2) * ld];
        const double p3 = Pi[(int64_t)(j + 3) * ld];
#pragma unroll
        for (int q = 0; q < QS; ++q) {
          double a = fma(p0, bq[j * KB + q], acc[q]);
          a = fma(p1, bq[(j + 1) * KB + q], a);
          a = fma(p2, bq[(j + 2) * KB + q], a);
          acc[q] = fma(p3, bq[(j + 3) * KB + q], a);
        }
      }
      for (; j < jw; ++j) {
        const double p = Pi[(int64_t)j * ld];
#pragma unroll
        for (int q = 0; q < QS; ++q) acc[q] = fma(p, bq[j * KB + q], acc[q]);
      }
      if (i >= w) {
        double* __restrict__ dst = Y + (int64_t)rows[i] * ldy + c0 + qa;
#pragma unroll
        for (int q = 0; q < QS; ++q) atomicAdd(dst + q, -acc[q]);
      } else if (ch.n == 1) {
        double* __restrict__ dst = Y2 + (int64_t)(f + i) * ldy + c0 + qa;
#pragma unroll
        for (int q = 0; q < QS; ++q) dst[q] = acc[q];
      } else {
#pragma unroll
        for (int q = 0; q < QS; ++q) *chunk_part(ch, KB, i - i0, qa + q) = acc[q];
      }
    }
    if (ch.n > 1 && ndiag > 0)
      chunk_finish<KB>(ch, ndiag, [&](int r, int q, double v) {
        Y2[(int64_t)(f + i0 + r) * ldy + c0 + q] = v;
      });
  } else {
  double acc[KB];
#pragma unroll
  for (int q = 0; q < KB; ++q) acc[q] = 0.0;
  if (i < ld) {
    int j = ja + sub;
    const double* sbj = sb - ja * KB;
    // four panel loads in flight per thread, then their FMAs
    for (; j + 3 * kSplit < jw; j += 4 * kSplit) {
      const double p0 = P[(int64_t)j * ld + i];
      const double p1 = P[(int64_t)(j + kSplit) * ld + i];
      const double p2 = P[(int64_t)(j + 2 * kSplit) * ld + i];
      const double p3 = P[(int64_t)(j + 3 * kSplit) * ld + i];
#pragma unroll
      for (int q = 0; q < KB; ++q) {
        double a = fma(p0, sbj[j * KB + q], acc[q]);
        a = fma(p1, sbj[(j + kSplit) * KB + q], a);
        a = fma(p2, sbj[(j + 2 * kSplit) * KB + q], a);
        acc[q] = fma(p3, sbj[(j + 3 * kSplit) * KB + q], a);
      }
    }
    for (; j < jw; j += kSplit) {
      const double p = P[(int64_t)j * ld + i];
#pragma unroll
      for (int q = 0; q < KB; ++q) acc[q] = fma(p, sbj[j * KB + q], acc[q]);
    }
  }
  split_sum<KB>(acc, sb, min(kRowBlock, ld - i0), [&](int r, int q, double v) {
    const int ir = i0 + r;
    if (ir >= w) atomicAdd(Y + (int64_t)rows[ir] * ldy + c0 + q, -v);
    else if (ch.n == 1) Y2[(int64_t)(f + ir) * ldy + c0 + q] = v;
    else *chunk_part(ch, KB, r, q) = v;
  });
  if (ch.n > 1 && ndiag > 0)
    chunk_finish<KB>(ch, ndiag, [&](int r, int q, double v) {
      Y2[(int64_t)(f + i0 + r) * ldy + c0 + q] = v;
    });
  }
}

// Backward task: panel columns [j0, j0+32) of P_s^T [D_s^{-1} y_s; -x_R], over
// the panel rows of chunk ch.
template <int KB>
__device__ __forceinline__ void bwd_task(const DevFactor& F, int s, int j0, int c0,
                                         double* __restrict__ Y, const double* __restrict__ Y2,
                                         int ldy, double* ub, Chunk ch) {
  const int f = F.sup_first[s];
  const int w = F.sup_first[s + 1] - f;
  const int64_t rp = F.sup_rowptr[s];
  const int ld = (int)(F.sup_rowptr[s + 1] - rp);
  const int32_t* __restrict__ rows = F.sup_rows + rp;
  // column j of the lower-triangular L_ss^{-1} is zero above row j, so the
  // panel rows of this block of columns start at j0
  int ia, ib;
  chunk_range(ch, j0, ld, ia, ib);
  for (int e = threadIdx.x; e < (ib - ia) * KB; e += blockDim.x) {
    const int i = ia + e / KB, q = e % KB;
    ub[e] = i < w ? __ldcg(Y2 + (int64_t)(f + i) * ldy + c0 + q) * F.dinv[f + i]
                  : -__ldcg(Y + (int64_t)rows[i] * ldy + c0 + q);
  }
  __syncthreads();
  const double* __restrict__ P = F.pan_rm + F.pan_off[s];
  const int sub = threadIdx.x % kSplit;
  const int j = j0 + threadIdx.x / kSplit;
  const double* ubi = ub - ia * KB;
  double acc[KB];
#pragma unroll
  for (int q = 0; q < KB; ++q) acc[q] = 0.0;
  if (j < w) {
    // the warp's 8 columns start at j0 + 8 * warp: rows above are zero for all of them
    int i = max(ia, j0 + (int)(threadIdx.x / 32) * (32 / kSplit)) + sub;
    for (; i + 3 * kSplit < ib; i += 4 * kSplit) {
      const double p0 = P[(int64_t)i * w + j];
      const double p1 = P[(int64_t)(i + kSplit) * w + j];
      const double p2 = P[(int64_t)(i + 2 * kSplit) * w + j];
      const double p3 = P[(int64_t)(i + 3 * kSplit) * w + j];
#pragma unroll
      for (int q = 0; q < KB; ++q) {
        double a = fma(p0, ubi[i * KB + q], acc[q]);
        a = fma(p1, ubi[(i + kSplit) * KB + q], a);
        a = fma(p2, ubi[(i + 2 * kSplit) * KB + q], a);
        acc[q] = fma(p3, ubi[(i + 3 * kSplit) * KB + q], a);
      }
    }
    for (; i < ib; i += kSplit) {
      const double p = P[(int64_t)i * w + j];
#pragma unroll
      for (int q = 0; q < KB; ++q) acc[q] = fma(p, ubi[i * KB + q], acc[q]);
    }
  }
  const int ncol = min(kRowBlock, w - j0);
  split_sum<KB>(acc, ub, ncol, [&](int r, int q, double v) {
    if (ch.n == 1) Y[(int64_t)(f + j0 + r) * ldy + c0 + q] = v;
    else *chunk_part(ch, KB, r, q) = v;
  });
  if (ch.n > 1)
    chunk_finish<KB>(ch, ncol, [&](int r, int q, double v) {
      Y[(int64_t)(f + j0 + r) * ldy + c0 + q] = v;
    });
}

// Descriptors of the supernodes of a packed task, staged in shared memory by
// one parallel load (no per-thread walk over the list).
struct PackDesc {
  int f[kPackMax], w[kPackMax], ld[kPackMax];
  int a[kPackMax], b[kPackMax];  // rows / columns of the earlier entries of the task
  long long pan[kPackMax], rp[kPackMax];
};

__device__ __forceinline__ void load_pack(const DevFactor& F, int e0, int ne, PackDesc& d) {
  for (int k = threadIdx.x; k < ne; k += blockDim.x) {
    const int s = F.pack[e0 + k];
    const int f = F.sup_first[s];
    const long long rp = F.sup_rowptr[s];
    d.f[k] = f;
    d.w[k] = F.sup_first[s + 1] - f;
    d.ld[k] = (int)(F.sup_rowptr[s + 1] - rp);
    d.a[k] = F.pack_a[e0 + k];
    d.b[k] = F.pack_b[e0 + k];
    d.pan[k] = F.pan_off[s];
    d.rp[k] = rp;
  }
  __syncthreads();
}

// The entry k of a packed task with pre[k] <= x < pre[k + 1] (pre ascending, pre[0] = 0).
__device__ __forceinline__ int pack_find(const int* pre, int ne, int x) {
  int lo = 0, hi = ne - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Packed forward task: several small supernodes of one level.  Lanes are
// (panel row, right-hand side) pairs: a warp takes 32 / KB consecutive rows of
// the task at a time, the four warps taking turns, so every lane of a warp
// runs a dot product of the same length w (packing in order of width keeps
// neighbouring supernodes alike; a masked lane costs the FP64 pipe as much
// as an active one).  The zero upper triangle of L_ss^{-1} is multiplied like
// any other entry for that reason.
template <int KB>
__device__ __forceinline__ void fwd_small(const DevFactor& F, int e0, int ne, int c0,
                                          double* __restrict__ Y, double* __restrict__ Y2, int ldy,
                                          double* sb, PackDesc& d) {
  constexpr int R = 32 / KB;
  load_pack(F, e0, ne, d);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  // right-hand sides b_s of every entry, one warp per entry
  for (int k = warp; k < ne; k += nwarps) {
    const int f = d.f[k], cnt = d.w[k] * KB;
    double* dst = sb + d.b[k] * KB;
    for (int e = lane; e < cnt; e += 32) {
      const int j = e / KB, q = e - j * KB;
      dst[e] = __ldcg(Y + (int64_t)(f + j) * ldy + c0 + q);
    }
  }
  __syncthreads();
  const int rows_total = d.a[ne - 1] + d.ld[ne - 1];
  const int rl = lane / KB, q = lane - rl * KB;
  for (int x0 = warp * R; x0 < rows_total; x0 += nwarps * R) {
    const int x = min(x0 + rl, rows_total - 1);  // past the task: a valid row, result dropped
    const int k = pack_find(d.a, ne, x);
    const int r = x - d.a[k], w = d.w[k], ld = d.ld[k], f = d.f[k];
    const double* __restrict__ P = F.pan_cm + d.pan[k] + r;
    const double* bs = sb + d.b[k] * KB + q;
    double acc = 0.0;
#pragma unroll 4
    for (int j = 0; j < w; ++j) acc = fma(P[(int64_t)j * ld], bs[j * KB], acc);
    if (x0 + rl < rows_total) {
      if (r < w) Y2[(int64_t)(f + r) * ldy + c0 + q] = acc;
      else atomicAdd(Y + (int64_t)F.sup_rows[d.rp[k] + r] * ldy + c0 + q, -acc);
    }
  }
}

// Packed backward task: several small supernodes.  Lanes are (panel column,
// right-hand side) pairs, 32 / KB consecutive columns of the task per warp
// step, each an ld-long dot product (packing in order of ld keeps them alike).
template <int KB>
__device__ __forceinline__ void bwd_small(const DevFactor& F, int e0, int ne, int c0,
                                          double* __restrict__ Y, const double* __restrict__ Y2,
                                          int ldy, double* ub, PackDesc& d) {
  constexpr int R = 32 / KB;
  load_pack(F, e0, ne, d);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  // u = [D_s^{-1} y_s; -x_R] of every entry, one warp per entry
  for (int k = warp; k < ne; k += nwarps) {
    const int f = d.f[k], w = d.w[k], cnt = d.ld[k] * KB;
    const int32_t* __restrict__ rows = F.sup_rows + d.rp[k];
    double* dst = ub + d.a[k] * KB;
    for (int e = lane; e < cnt; e += 32) {
      const int i = e / KB, q = e - i * KB;
      dst[e] = i < w ? __ldcg(Y2 + (int64_t)(f + i) * ldy + c0 + q) * F.dinv[f + i]
                     : -__ldcg(Y + (int64_t)rows[i] * ldy + c0 + q);
    }
  }
  __syncthreads();
  const int cols_total = d.b[ne - 1] + d.w[ne - 1];
  const int cl = lane / KB, q = lane - cl * KB;
  for (int x0 = warp * R; x0 < cols_total; x0 += nwarps * R) {
    const int x = min(x0 + cl, cols_total - 1);
    const int k = pack_find(d.b, ne, x);
    const int j = x - d.b[k], w = d.w[k], ld = d.ld[k];
    const double* __restrict__ P = F.pan_rm + d.pan[k] + j;
    const double* u = ub + d.a[k] * KB + q;
    double acc = 0.0;
#pragma unroll 4
    for (int i = 0; i < ld; ++i) acc = fma(P[(int64_t)i * w], u[i * KB], acc);
    if (x0 + cl < cols_total) Y[(int64_t)(d.f[k] + j) * ldy + c0 + q] = acc;
  }
}

// Packed forward task, one thread per panel row (all rows of the task at
// once; for levels whose packed work cannot fill the GPU, where the solve is
// latency-bound): each thread holds KB accumulators over its row's w entries.
template <int KB>
__device__ __forceinline__ void fwd_small_rows(const DevFactor& F, int e0, int ne, int c0,
                                               double* __restrict__ Y, double* __restrict__ Y2,
                                               int ldy, double* sb, PackDesc& d) {
  load_pack(F, e0, ne, d);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (int k = warp; k < ne; k += nwarps) {
    const int f = d.f[k], cnt = d.w[k] * KB;
    double* dst = sb + d.b[k] * KB;
    for (int e = lane; e < cnt; e += 32) {
      const int j = e / KB, q = e - j * KB;
      dst[e] = __ldcg(Y + (int64_t)(f + j) * ldy + c0 + q);
    }
  }
  __syncthreads();
  const int x = threadIdx.x;
  if (x >= d.a[ne - 1] + d.ld[ne - 1]) return;
  const int k = pack_find(d.a, ne, x);
  const int r = x - d.a[k], w = d.w[k], ld = d.ld[k], f = d.f[k];
  const double* __restrict__ P = F.pan_cm + d.pan[k];
  const double* bs = sb + d.b[k] * KB;
  const int jend = r < w ? r + 1 : w;  // L_ss^{-1} is lower triangular
  double acc[KB];
#pragma unroll
  for (int q = 0; q < KB; ++q) acc[q] = 0.0;
  for (int j = 0; j < jend; ++j) {
    const double p = P[(int64_t)j * ld + r];
#pragma unroll
    for (int q = 0; q < KB; ++q) acc[q] = fma(p, bs[j * KB + q], acc[q]);
  }
  if (r < w) {
    double* __restrict__ dst = Y2 + (int64_t)(f + r) * ldy + c0;
#pragma unroll
    for (int q = 0; q < KB; ++q) dst[q] = acc[q];
  } else {
    double* __restrict__ dst = Y + (int64_t)F.sup_rows[d.rp[k] + r] * ldy + c0;
#pragma unroll
    for (int q = 0; q < KB; ++q) atomicAdd(dst + q, -acc[q]);
  }
}

// Packed backward task, one thread per panel column.
template <int KB>
__device__ __forceinline__ void bwd_small_rows(const DevFactor& F, int e0, int ne, int c0,
                                               double* __restrict__ Y,
                                               const double* __restrict__ Y2, int ldy, double* ub,
                                               PackDesc& d) {
  load_pack(F, e0, ne, d);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (int k = warp; k < ne; k += nwarps) {
    const int f = d.f[k], w = d.w[k], cnt = d.ld[k] * KB;
    const int32_t* __restrict__ rows = F.sup_rows + d.rp[k];
    double* dst = ub + d.a[k] * KB;
    for (int e = lane; e < cnt; e += 32) {
      const int i = e / KB, q = e - i * KB;
      dst[e] = i < w ? __ldcg(Y2 + (int64_t)(f + i) * ldy + c0 + q) * F.dinv[f + i]
                     : -__ldcg(Y + (int64_t)rows[i] * ldy + c0 + q);
    }
  }
  __syncthreads();
  const int x = threadIdx.x;
  if (x >= d.b[ne - 1] + d.w[ne - 1]) return;
  const int k = pack_find(d.b, ne, x);
  const int j = x - d.b[k], w = d.w[k], ld = d.ld[k];
  const double* __restrict__ P = F.pan_rm + d.pan[k];
  const double* u = ub + d.a[k] * KB;
  double acc[KB];
#pragma unroll
  for (int q = 0; q < KB; ++q) acc[q] = 0.0;
  for (int i = j; i < ld; ++i) {  // column j of L_ss^{-1} is zero above row j
    const double p = P[(int64_t)i * w + j];
#pragma unroll
    for (int q = 0; q < KB; ++q) acc[q] = fma(p, u[i * KB + q], acc[q]);
  }
  double* __restrict__ dst = Y + (int64_t)(d.f[k] + j) * ldy + c0;
#pragma unroll
  for (int q = 0; q < KB; ++q) dst[q] = acc[q];
}

template <int KB>
__device__ __forceinline__ void run_fwd(const DevFactor& F, int2 tk, int c0, double* Y, double* Y2,
                                        int ldy, double* sm, PackDesc& pd,
                                        Chunk ch = Chunk()) {
  const int ne = tk.y & (kPackRowwise - 1);
  if (tk.x >= 0) fwd_task<KB>(F, tk.x, tk.y, c0, Y, Y2, ldy, sm, ch);
  else if (ch.c > 0) return;  // packed tasks are not chunked: the first chunk's CTA runs them
  else if (tk.y & kPackRowwise) fwd_small_rows<KB>(F, -1 - tk.x, ne, c0, Y, Y2, ldy, sm, pd);
  else fwd_small<KB>(F, -1 - tk.x, ne, c0, Y, Y2, ldy, sm, pd);
}

template <int KB>
__device__ __forceinline__ void run_bwd(const DevFactor& F, int2 tk, int c0, double* Y,
                                        const double* Y2, int ldy, double* sm, PackDesc& pd,
                                        Chunk ch = Chunk()) {
  const int ne = tk.y & (kPackRowwise - 1);
  if (tk.x >= 0) bwd_task<KB>(F, tk.x, tk.y, c0, Y, Y2, ldy, sm, ch);
  else if (ch.c > 0) return;
  else if (tk.y & kPackRowwise) bwd_small_rows<KB>(F, -1 - tk.x, ne, c0, Y, Y2, ldy, sm, pd);
  else bwd_small<KB>(F, -1 - tk.x, ne, c0, Y, Y2, ldy, sm, pd);
}

// One CTA per (task, column block, chunk), chunks innermost: blockIdx.x =
// (task * ncb + column block) * nchunk + chunk; the (task, column block) pair
// is the chunks' scratch slot.
__device__ __forceinline__ Chunk level_chunk(int ncb, int nchunk, const SplitScratch& sp,
                                             int& task, int& cb) {
  const int slot = blockIdx.x / nchunk;
  task = slot / ncb;
  cb = slot - task * ncb;
  Chunk ch;
  ch.c = blockIdx.x - slot * nchunk;
  ch.n = nchunk;
  ch.part = sp.part;
  ch.cnt = sp.cnt;
  ch.slot = slot;
  return ch;
}

// Level launches are chained with programmatic dependent launch: each lets
// the next level's grid be scheduled as soon as all of its own CTAs run
// (launch_dependents), and waits for the previous grid to complete and its
// writes to be visible (griddepcontrol.wait) before reading anything.
__device__ __forceinline__ void level_chain_wait() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <int KB>
__global__ void __launch_bounds__(kSolveThreads, 8)
fwd_level_kernel(DevFactor F, const int2* __restrict__ tasks, int ncb, int nchunk,
                 SplitScratch sp, double* __restrict__ Y, double* __restrict__ Y2, int ldy) {
  extern __shared__ double sb[];
  __shared__ PackDesc pd;
  level_chain_wait();
  if (F.abort && *F.abort) return;
  int task, cb;
  const Chunk ch = level_chunk(ncb, nchunk, sp, task, cb);
  run_fwd<KB>(F, tasks[task], cb * KB, Y, Y2, ldy, sb, pd, ch);
}

template <int KB>
__global__ void __launch_bounds__(kSolveThreads, 8)
bwd_level_kernel(DevFactor F, const int2* __restrict__ tasks, int ncb, int nchunk,
                 SplitScratch sp, double* __restrict__ Y, const double* __restrict__ Y2, int ldy) {
  extern __shared__ double ub[];
  __shared__ PackDesc pd;
  level_chain_wait();
  if (F.abort && *F.abort) return;
  int task, cb;
  const Chunk ch = level_chunk(ncb, nchunk, sp, task, cb);
  run_bwd<KB>(F, tasks[task], cb * KB, Y, Y2, ldy, ub, pd, ch);
}

// ---------------------------------------------------------------------------
// Persistent solve: one launch runs every forward task (levels bottom-up) and
// then every backward task (top-down).  CTAs take tickets in that order; a
// task starts when its dependencies are met:
//   forward (s, .)  : every forward task of every child of s is done
//                     (fpend[s] counts children not yet complete);
//   backward (s, .) : every backward task of parent(s) is done, or for a root
//                     every forward task of s.
// Tickets go out in dependency order and a CTA only waits on tasks holding
// earlier tickets (already running), so the waits end; each wait is still
// bounded, and on expiry the kernel raises the error flag and stops.
// ---------------------------------------------------------------------------
constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // 1 s per wait

__device__ __forceinline__ int ld_volatile(const int* p) { return *((const volatile int*)p); }

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Spin (thread 0 only) until *p >= target (or *p <= 0 when zero); gives up
// after kWaitLimitNs or when another CTA has raised the error flag.
__device__ bool wait_until(const int* p, int target, bool zero, int* err) {
  const unsigned long long t0 = global_ns();
  for (;;) {
    const int v = ld_volatile(p);
    if (zero ? v <= 0 : v >= target) break;
    if (ld_volatile(err) || global_ns() - t0 > kWaitLimitNs) {
      atomicExch(err, 1);
      return false;
    }
    __nanosleep(64);
  }
  __threadfence();
  return true;
}

__global__ void bump_kernel(int* p) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *p += 1;
}

__global__ void __launch_bounds__(kSolveThreads, 6)
persistent_solve_kernel(DevFactor F, PersistSched ps, double* __restrict__ Y,
                        double* __restrict__ Y2, int ldy) {
  extern __shared__ double sm[];
  __shared__ long long sh_t;
  __shared__ int sh_ok;
  __shared__ PackDesc pd;
  if (F.abort && *F.abort) return;  // set before the launch: every CTA leaves, none waits
  const long long total = ps.nf_total + ps.nb_total;
  for (;;) {
    if (threadIdx.x == 0) sh_t = (long long)atomicAdd(ps.ticket, 1ull);
    __syncthreads();
    const long long t = sh_t;
    if (t >= total) break;
    const bool fwd = t < ps.nf_total;
    // locate the level of this ticket and its first task
    int l;
    long long unit;
    if (fwd) {
      l = 0;
      while (l + 1 < ps.nlev && ps.lev[l + 1].fbase <= t) ++l;
      unit = t - ps.lev[l].fbase;
    } else {
      const long long tb = t - ps.nf_total;
      l = ps.nlev - 1;
      while (l > 0 && ps.lev[l - 1].bbase <= tb) --l;
      unit = tb - ps.lev[l].bbase;
    }
    const PersistLevel& L = ps.lev[l];
    const int batch = fwd ? L.fbatch : L.bbatch;
    const long long ntask = (long long)(fwd ? L.nf : L.nb) * L.ncb;
    const long long lo = unit * batch, hi = min(ntask, lo + batch);
    bool failed = false;
    for (long long local = lo; local < hi; ++local) {
      const int task = (int)(local / L.ncb);
      const int c0 = (int)(local % L.ncb) * L.kb;
      const int2 tk = fwd ? L.ftasks[task] : L.btasks[task];
      // supernodes of this task: one, or a packed list
      const int32_t* ents = tk.x >= 0 ? nullptr : F.pack + (-1 - tk.x);
      const int ne = tk.x >= 0 ? 1 : (tk.y & (kPackRowwise - 1));
      if (threadIdx.x == 0) {
        bool ok = true;
        for (int k = 0; k < ne && ok; ++k) {
          const int s = ents ? ents[k] : tk.x;
          if (fwd) {
            ok = wait_until(ps.fpend + s, 0, true, ps.err);
          } else {
            const int p = F.sup_parent[s];
            if (p >= 0) {
              const PersistLevel& Lp = ps.lev[ps.sup_level[p]];
              ok = wait_until(ps.bdone + p, ps.nbt[p] * Lp.ncb, false, ps.err);
            } else {
              ok = wait_until(ps.fdone + s, ps.nft[s] * L.ncb, false, ps.err);
            }
          }
        }
        sh_ok = ok;
      }
      __syncthreads();
      if (!sh_ok) { failed = true; break; }
      if (fwd) {
        switch (L.kb) {
          case 1: run_fwd<1>(F, tk, c0, Y, Y2, ldy, sm, pd); break;
          case 2: run_fwd<2>(F, tk, c0, Y, Y2, ldy, sm, pd); break;
          case 4: run_fwd<4>(F, tk, c0, Y, Y2, ldy, sm, pd); break;
          default: run_fwd<8>(F, tk, c0, Y, Y2, ldy, sm, pd); break;
        }
      } else {
        switch (L.kb) {
          case 1: run_bwd<1>(F, tk, c0, Y, Y2, ldy, sm, pd); break;
          case 2: run_bwd<2>(F, tk, c0, Y, Y2, ldy, sm, pd); break;
          case 4: run_bwd<4>(F, tk, c0, Y, Y2, ldy, sm, pd); break;
          default: run_bwd<8>(F, tk, c0, Y, Y2, ldy, sm, pd); break;
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        for (int k = 0; k < ne; ++k) {
          const int s = ents ? ents[k] : tk.x;
          if (fwd) {
            const int old = atomicAdd(ps.fdone + s, 1);
            const int p = F.sup_parent[s];
            if (old == ps.nft[s] * L.ncb - 1 && p >= 0) {
              __threadfence();
              atomicSub(ps.fpend + p, 1);
            }
          } else {
            atomicAdd(ps.bdone + s, 1);
          }
        }
      }
    }
    if (failed) break;
  }
}

template <int KB>
void launch_level(bool fwd, const DevFactor& F, const LevelPlan& L, double* Y, double* Y2, int ldy,
                  int ncols, cudaStream_t st, const SplitScratch* split) {
  const int ncb = (ncols + KB - 1) / KB;
  const size_t part = (size_t)kSolveThreads * (KB + 1);  // split_sum's partials
  // Chunks: when the level's (task, column block) pairs leave most of the GPU
  // idle and its split tasks have long reductions, each such task runs as
  // several CTAs over slices of its reduction (at least kSplitMinWidth long).
  const int tasks = fwd ? L.nf : L.nb;
  const int extent = fwd ? L.split_w : L.split_ld;
  int nchunk = 1;
  SplitScratch sp;
  if (split && split->part && extent >= 2 * kSplitMinWidth && (long long)tasks * ncb < kSplitSlots) {
    const int want = (kSplitTarget + tasks * ncb - 1) / (tasks * ncb);
    nchunk = std::max(1, std::min({want, extent / kSplitMinWidth, kSplitMaxChunks}));
    // scratch holds 2 * kSplitSlots (slot, chunk) pairs
    while (nchunk > 1 && (long long)tasks * ncb * nchunk > 2LL * kSplitSlots) --nchunk;
    if (nchunk > 1) sp = *split;
  }
  const unsigned grid = (unsigned)((long long)tasks * ncb * nchunk);
  if (grid == 0) return;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kSolveThreads);
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (fwd) {
    cfg.dynamicSmemBytes = std::max((size_t)L.max_w * KB, part) * sizeof(double);
    cudaLaunchKernelEx(&cfg, fwd_level_kernel<KB>, F, L.ftasks, ncb, nchunk, sp, Y, Y2, ldy);
  } else {
    cfg.dynamicSmemBytes = std::max((size_t)L.max_wr * KB, part) * sizeof(double);
    cudaLaunchKernelEx(&cfg, bwd_level_kernel<KB>, F, L.btasks, ncb, nchunk, sp, Y,
                       (const double*)Y2, ldy);
  }
}

void run_level(bool fwd, const DevFactor& F, const LevelPlan& L, double* Y, double* Y2, int ldy,
               int ncols, cudaStream_t st, const SplitScratch* split, int force_kb = 0) {
  int kb = force_kb > 0 ? force_kb : fwd ? L.kbf : L.kbb;
  while (kb > 1 && kb / 2 >= ncols) kb /= 2;
  switch (kb) {
    case 1: launch_level<1>(fwd, F, L, Y, Y2, ldy, ncols, st, split); break;
    case 2: launch_level<2>(fwd, F, L, Y, Y2, ldy, ncols, st, split); break;
    case 4: launch_level<4>(fwd, F, L, Y, Y2, ldy, ncols, st, split); break;
    default: launch_level<8>(fwd, F, L, Y, Y2, ldy, ncols, st, split); break;
  }
}

// 32x32 tiles through shared memory for the node-major <-> vector-major moves
__global__ void gather_cols_kernel(double* __restrict__ Y, int ldy, int ncols,
                                   const double* __restrict__ src, int64_t stride,
                                   const int32_t* __restrict__ cols,
                                   const double* __restrict__ scale,
                                   const int32_t* __restrict__ rowmap, int64_t n) {
  __shared__ double tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  const int q0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int q = q0 + k;
    const int64_t i = i0 + threadIdx.x;
    double v = 0.0;
    if (q < ncols && i < n) {
      const int64_t g = cols ? cols[q] : q;
      v = src[g * stride + (rowmap ? rowmap[i] : i)];
      if (scale) v *= scale[i];
    }
    tile[k][threadIdx.x] = v;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t i = i0 + k;
    const int q = q0 + threadIdx.x;
    if (i < n && q < ncols) Y[i * ldy + q] = tile[threadIdx.x][k];
  }
}

__global__ void scatter_cols_kernel(const double* __restrict__ Y, int ldy, int ncols,
                                    double* __restrict__ dst, int64_t stride,
                                    const int32_t* __restrict__ cols,
                                    const int32_t* __restrict__ rowmap, int64_t n) {
  __shared__ double tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  const int q0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t i = i0 + k;
    const int q = q0 + threadIdx.x;
    tile[k][threadIdx.x] = (i < n && q < ncols) ? Y[i * ldy + q] : 0.0;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int q = q0 + k;
    const int64_t i = i0 + threadIdx.x;
    if (q < ncols && i < n) {
      const int64_t g = cols ? cols[q] : q;
      dst[g * stride + (rowmap ? rowmap[i] : i)] = tile[threadIdx.x][k];
    }
  }
}

}  // namespace

void persistent_solve(const DevFactor& F, const PersistSched& ps, int grid, size_t smem,
                      double* Y, double* Y2, int ldy, cudaStream_t st) {
  persistent_solve_kernel<<<grid, kSolveThreads, smem, st>>>(F, ps, Y, Y2, ldy);
}

void bump_counter(int* p, cudaStream_t st) { bump_kernel<<<1, 32, 0, st>>>(p); }

// The dynamic shared-memory cap of a kernel is a process-wide attribute (per
// device), while each context needs its own amount: only ever raise it, so a
// context set up later with smaller panels does not lower it below what an
// earlier context launches with.
namespace {
std::mutex g_smem_mu;
int g_solve_smem[64] = {0};
int g_persist_smem[64] = {0};
int cur_device_slot() {
  int dev = 0;
  cudaGetDevice(&dev);
  return dev >= 0 && dev < 64 ? dev : 63;
}
}  // namespace

int persistent_blocks_per_sm(size_t smem) {
  {
    std::lock_guard<std::mutex> lk(g_smem_mu);
    int& cur = g_persist_smem[cur_device_slot()];
    if ((int)smem > cur) {
      cudaFuncSetAttribute(persistent_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
      cur = (int)smem;
    }
  }
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, persistent_solve_kernel, kSolveThreads, smem);
  return nb;
}
float time_level(bool fwd, const DevFactor& F, const LevelPlan& L, int kb, double* Y, double* Y2,
                 int ldy, int ncols, cudaStream_t st, const SplitScratch* split, int reps) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaGetLastError();
    return -1.f;
  }
  run_level(fwd, F, L, Y, Y2, ldy, ncols, st, split, kb);
  float best = 1e30f;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(e0, st);
    run_level(fwd, F, L, Y, Y2, ldy, ncols, st, split, kb);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return cudaGetLastError() == cudaSuccess ? best : -1.f;
}

bool preload_solve_kernels() {
  cudaFuncAttributes a;
  bool ok = cudaFuncGetAttributes(&a, persistent_solve_kernel) == cudaSuccess &&
            cudaFuncGetAttributes(&a, gather_cols_kernel) == cudaSuccess &&
            cudaFuncGetAttributes(&a, scatter_cols_kernel) == cudaSuccess &&
            cudaFuncGetAttributes(&a, fwd_level_kernel<1>) == cudaSuccess &&
            cudaFuncGetAttributes(&a, fwd_level_kernel<2>) == cudaSuccess &&
            cudaFuncGetAttributes(&a, fwd_level_kernel<4>) == cudaSuccess &&
            cudaFuncGetAttributes(&a, fwd_level_kernel<8>) == cudaSuccess &&
            cudaFuncGetAttributes(&a, bwd_level_kernel<1>) == cudaSuccess &&
            cudaFuncGetAttributes(&a, bwd_level_kernel<2>) == cudaSuccess &&
            cudaFuncGetAttributes(&a, bwd_level_kernel<4>) == cudaSuccess &&
            cudaFuncGetAttributes(&a, bwd_level_kernel<8>) == cudaSuccess;
  if (!ok) cudaGetLastError();
  return ok;
}

void set_solve_smem_limit(int bytes) {
  std::lock_guard<std::mutex> lk(g_smem_mu);
  int& cur = g_solve_smem[cur_device_slot()];
  if (bytes <= cur) return;
  cur = bytes;
  cudaFuncSetAttribute(fwd_level_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(fwd_level_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(fwd_level_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(fwd_level_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(bwd_level_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(bwd_level_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(bwd_level_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(bwd_level_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

void solve_level(bool fwd, const DevFactor& F, const LevelPlan& L, double* Y, double* Y2, int ldy,
                 int ncols, cudaStream_t st, const SplitScratch* split) {
  if (ncols > 0 && (fwd ? L.nf : L.nb) > 0) run_level(fwd, F, L, Y, Y2, ldy, ncols, st, split);
}

int solve_inplace(const DevFactor& F, const LevelPlan* levels, int nlev, double* Y, double* Y2,
                  int ldy, int ncols, cudaStream_t st, const SplitScratch* split) {
  if (ncols <= 0) return 0;
  for (int l = 0; l < nlev; ++l) run_level(true, F, levels[l], Y, Y2, ldy, ncols, st, split);
  for (int l = nlev - 1; l >= 0; --l) run_level(false, F, levels[l], Y, Y2, ldy, ncols, st, split);
  return 2 * nlev;
}

void gather_cols(double* Y, int ldy, int ncols, const double* src, int64_t stride,
                 const int32_t* cols, const double* scale, const int32_t* rowmap, int64_t n,
                 cudaStream_t st) {
  if (ncols <= 0 || n <= 0) return;
  dim3 grid((unsigned)((n + 31) / 32), (unsigned)((ncols + 31) / 32));
  gather_cols_kernel<<<grid, dim3(32, 8), 0, st>>>(Y, ldy, ncols, src, stride, cols, scale, rowmap,
                                                    n);
}

void scatter_cols(const double* Y, int ldy, int ncols, double* dst, int64_t stride,
                  const int32_t* cols, const int32_t* rowmap, int64_t n, cudaStream_t st) {
  if (ncols <= 0 || n <= 0) return;
  dim3 grid((unsigned)((n + 31) / 32), (unsigned)((ncols + 31) / 32));
  scatter_cols_kernel<<<grid, dim3(32, 8), 0, st>>>(Y, ldy, ncols, dst, stride, cols, rowmap, n);
}

}  // namespace matex
