// Basis recombination and superposition (the final step of Alg. 1, Alg. 2 snapshots,
// and the scheduler's sum of group responses, Sec. 3.2):
//   x_k(t_o) = V_k y_k(t_o) + z_k + (t_o - l_j) z'_k - w_k     (Eq. 6 with -P)
//   X[o]    += sum over the round's groups whose segment holds t_o.
// Each thread owns one node and a tile of 16 output times; the groups are
// summed in registers in a fixed order, so a round writes each output entry
// once.  The coefficient rows hold beta e^{h H_m} e_1 and h = t_o - l_j.
#include "kernels.h"

namespace matex {

namespace {

constexpr int kRecThreads = 128;
constexpr int kOT = 16;  // output times per thread

// One group's contribution to a thread's node over the tile's output times,
// from its basis vectors J0..J1-1 (and its -P term when P).  A group of
// Krylov dimension M takes one call <0, M, true>, or for M > kSplitM two calls
// (<0, kSplitM, true> and <kSplitM, M, false>) so that no instance holds more
// than kSplitM basis values in registers.  Every FP64 instruction issued is
// useful work.  When the group's segment covers the whole tile (warp-uniform),
// its -P term z + (t_o - l_j) z' - w = (z - w - l_j z') + t_o z' is folded into
// two per-tile sums (asum, zsum) applied once per output after all groups,
// leaving one FMA per (node, output, group, basis vector).  A partially
// covering group runs a loop over its covered outputs only (trip count
// uniform across the block) and adds its term, -P included, into the
// thread's slots of a shared-memory accumulator (`part`, stride kRecThreads),
// which a register array could not take at a run-time index.
constexpr int kSplitM = 10;

template <int J0, int J1, bool P>
__device__ __forceinline__ void group_tile(double (&acc)[kOT], double& asum, double& zsum,
                                           double* __restrict__ part,
                                           const double* __restrict__ vcol, int64_t n, double z,
                                           double zp, double w, double l0,
                                           const double* __restrict__ cq, int o0, int ob, int lo,
                                           int hi) {
  constexpr int M = J1 - J0;
  const double zmw = z - w;
  if (lo == o0 && hi == o0 + kOT) {
    double v[M > 0 ? M : 1];
#pragma unroll
    for (int j = 0; j < M; ++j) v[j] = vcol[(int64_t)(J0 + j) * n];
    if (P) {
      asum += fma(-l0, zp, zmw);
      zsum += zp;
    }
#pragma unroll
    for (int t = 0; t < kOT; ++t) {
      const double* __restrict__ y = cq + (int64_t)(o0 + t - ob) * kCoefLd + J0;
      double a = acc[t];
#pragma unroll
      for (int j = 0; j < M; ++j) a = fma(v[j], y[j], a);
      acc[t] = a;
    }
  } else {
#pragma unroll 1
    for (int o = lo; o < hi; ++o) {
      const double* __restrict__ y = cq + (int64_t)(o - ob) * kCoefLd;
      double a = P ? fma(y[kMaxM], zp, zmw) : 0.0;
#pragma unroll
      for (int j = J0; j < J1; ++j) a = fma(vcol[(int64_t)j * n], y[j], a);  // L1 after the first o
      part[(o - o0) * kRecThreads] += a;
    }
  }
}

__global__ void __launch_bounds__(kRecThreads)
recombine_kernel(double* __restrict__ Xp, int64_t n, const double* __restrict__ Vb, int64_t vstride,
                 const double* __restrict__ Z, const double* __restrict__ Zp,
                 const double* __restrict__ W, int64_t gstride, RoundCols rc,
                 const int32_t* __restrict__ mcol, const double* __restrict__ coef, int ldo, int K,
                 int obeg_min, double dt_out, const int32_t* __restrict__ tcut) {
  __shared__ double part_s[kOT * kRecThreads];
  const int64_t i = (int64_t)blockIdx.x * kRecThreads + threadIdx.x;
  const int o0 = obeg_min + blockIdx.y * kOT;
  if (i >= n || (rc.abort && *rc.abort)) return;
  double* __restrict__ part = part_s + threadIdx.x;  // this thread's slots only: no barrier
  double acc[kOT];
#pragma unroll
  for (int t = 0; t < kOT; ++t) {
    acc[t] = 0.0;
    part[t * kRecThreads] = 0.0;
  }
  double asum = 0.0, zsum = 0.0;
  unsigned covered = 0;
  for (int q = 0; q < K; ++q) {
    const int ob = rc.obeg[q], no = rc.nout[q];
    const int lo = max(ob, o0), hi = min(ob + no, o0 + kOT);
    if (lo >= hi) continue;
    int mq = mcol[q];
    if (tcut && o0 >= ob + tcut[2 * q]) {  // the tile lies past the column's tail cut
      if (tcut[2 * q + 1]) continue;
      mq = 0;
    }
    covered |= ((1u << (hi - lo)) - 1u) << (lo - o0);
    const int64_t g = rc.group[q];
    const double* __restrict__ vcol = Vb + (int64_t)rc.vslot[q] * vstride + i;
    const double z = Z[g * gstride + i], zp = Zp[g * gstride + i], w = W[g * gstride + i];
    const double l0 = rc.l0[q];
    const double* __restrict__ cq = coef + (int64_t)q * ldo * kCoefLd;
    switch (mq) {
#define MATEX_GT(MM)                                                                           \
  case MM:                                                                                     \
    group_tile<0, MM, true>(acc, asum, zsum, part, vcol, n, z, zp, w, l0, cq, o0, ob, lo, hi); \
    break;
#define MATEX_GT2(MM)                                                                          \
  case MM:                                                                                     \
    group_tile<0, kSplitM, true>(acc, asum, zsum, part, vcol, n, z, zp, w, l0, cq, o0, ob, lo, \
                                 hi);                                                          \
    group_tile<kSplitM, MM, false>(acc, asum, zsum, part, vcol, n, z, zp, w, l0, cq, o0, ob,   \
                                   lo, hi);                                                    \
    break;
      MATEX_GT(0) MATEX_GT(1) MATEX_GT(2) MATEX_GT(3) MATEX_GT(4) MATEX_GT(5) MATEX_GT(6)
      MATEX_GT(7) MATEX_GT(8) MATEX_GT(9) MATEX_GT(10) MATEX_GT2(11) MATEX_GT2(12) MATEX_GT2(13)
      MATEX_GT2(14) MATEX_GT2(15) MATEX_GT2(16) MATEX_GT2(17) MATEX_GT2(18) MATEX_GT2(19)
      MATEX_GT2(20)
#undef MATEX_GT
#undef MATEX_GT2
      default: break;
    }
  }
#pragma unroll
  for (int t = 0; t < kOT; ++t)
    if (covered & (1u << t)) {
      const double to = (double)(o0 + t) * dt_out;
      Xp[(int64_t)(o0 + t) * n + i] += (acc[t] + part[t * kRecThreads]) + fma(to, zsum, asum);
    }
}

// Per column, the largest |z - w| and |z'| of its group over a chunk of nodes,
// folded into pbound by an atomic max.  Both are >= 0 (or NaN with the sign
// bit clear), so their bit patterns order like the values and a NaN, whose
// pattern is above +inf's, is kept.
constexpr int kPbThreads = 256;
constexpr int kPbPer = 8;  // nodes per thread

__global__ void __launch_bounds__(kPbThreads)
p_bound_kernel(const double* __restrict__ Z, const double* __restrict__ Zp,
               const double* __restrict__ W, int64_t gstride, RoundCols rc, int64_t n,
               unsigned long long* __restrict__ pbound) {
  const int q = blockIdx.y;
  const int64_t g = rc.group[q];
  const double* __restrict__ z = Z + g * gstride;
  const double* __restrict__ zp = Zp + g * gstride;
  const double* __restrict__ w = W + g * gstride;
  unsigned long long a = 0, b = 0;
  const int64_t base = (int64_t)blockIdx.x * kPbThreads * kPbPer + threadIdx.x;
#pragma unroll
  for (int k = 0; k < kPbPer; ++k) {
    const int64_t i = base + (int64_t)k * kPbThreads;
    if (i < n) {
      a = max(a, (unsigned long long)__double_as_longlong(fabs(z[i] - w[i])));
      b = max(b, (unsigned long long)__double_as_longlong(fabs(zp[i])));
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    a = max(a, __shfl_xor_sync(0xffffffffu, a, off));
    b = max(b, __shfl_xor_sync(0xffffffffu, b, off));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(pbound + 2 * q, a);
    atomicMax(pbound + 2 * q + 1, b);
  }
}

__global__ void next_state_kernel(double* __restrict__ X, const double* __restrict__ Vb,
                                  int64_t vstride, const double* __restrict__ Z,
                                  const double* __restrict__ Zp, const double* __restrict__ W,
                                  int64_t gstride, RoundCols rc, const int32_t* __restrict__ mcol,
                                  const double* __restrict__ yend, int64_t n) {
  const int q = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t g = rc.group[q];
  const int m = mcol[q];
  const double L = rc.len[q];
  double s = Z[g * gstride + i] + L * Zp[g * gstride + i] - W[g * gstride + i];
  const double* __restrict__ base = Vb + (int64_t)rc.vslot[q] * vstride + i;
  for (int j = 0; j < m; ++j) s = fma(base[(int64_t)j * n], yend[q * kMaxM + j], s);
  X[g * gstride + i] = s;
}

// The -P terms of a round alone, X[o] += sum over the columns whose segment
// holds o of z + (t_o - l_j) z' - w = (z - w - l_j z') + t_o z'.  Which
// columns hold o changes only where a column's output range starts or ends:
// one thread per node sweeps the outputs in order, keeping the two running
// sums A = sum (z - w - l_j z') and B = sum z' of the columns holding o and
// updating them at those events (sorted by output: ev_o; ev_q = q + 1 when
// column q enters, -(q + 1) when it leaves).  Each column's z, z', w are read
// once per node, not once per output tile.
__global__ void __launch_bounds__(128)
recombine_p_kernel(double* __restrict__ Xp, int64_t n, const double* __restrict__ Z,
                   const double* __restrict__ Zp, const double* __restrict__ W, int64_t gstride,
                   RoundCols rc, const int32_t* __restrict__ ev_o, const int32_t* __restrict__ ev_q,
                   int nev, int o_begin, int o_end, double dt_out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || (rc.abort && *rc.abort)) return;
  double A = 0.0, B = 0.0;
  int active = 0, e = 0;
  for (int o = o_begin; o < o_end; ++o) {
    for (; e < nev && ev_o[e] <= o; ++e) {
      const int qs = ev_q[e];
      const int q = (qs > 0 ? qs : -qs) - 1;
      const int64_t g = rc.group[q];
      const double zp = Zp[g * gstride + i];
      const double a = fma(-rc.l0[q], zp, Z[g * gstride + i] - W[g * gstride + i]);
      if (qs > 0) {
        A += a;
        B += zp;
        active++;
      } else {
        A -= a;
        B -= zp;
        active--;
      }
    }
    if (active > 0) {
      double* x = Xp + (int64_t)o * n + i;
      *x += fma((double)o * dt_out, B, A);
    }
  }
}

// Checkpoint of column q: CK[q] = {X[group q], Z[group q]} (save), or back (restore).
__global__ void checkpoint_kernel(double* __restrict__ CK, double* __restrict__ X,
                                  double* __restrict__ Z, const int32_t* __restrict__ groups,
                                  int64_t n, int restore) {
  const int q = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t g = groups[q];
  double* ck = CK + (int64_t)q * 2 * n;
  if (restore) {
    X[g * n + i] = ck[i];
    Z[g * n + i] = ck[n + i];
  } else {
    ck[i] = X[g * n + i];
    ck[n + i] = Z[g * n + i];
  }
}

__global__ void fill_rows_kernel(double* __restrict__ Xp, const double* __restrict__ base,
                                 int64_t n, int n_times) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = base ? base[i] : 0.0;
  for (int o = 0; o < n_times; ++o) Xp[(int64_t)o * n + i] = v;
}

__global__ void add_row_sum_kernel(double* __restrict__ Xp, const double* __restrict__ Y, int ldy,
                                   int K, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int q = 0; q < K; ++q) s += Y[i * ldy + q];
  Xp[i] += s;
}

__global__ void permute_out_kernel(double* __restrict__ out, const double* __restrict__ Xp,
                                   const int32_t* __restrict__ map, int64_t nrows, int64_t n) {
  const int o = blockIdx.y;
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  out[(int64_t)o * nrows + r] = Xp[(int64_t)o * n + map[r]];
}

}  // namespace

void recombine(double* Xp, int64_t n, int n_times, const double* Vbase, int64_t vstride,
               const double* Z, const double* Zp, const double* W, int64_t gstride,
               const RoundCols& rc, const int32_t* mcol, const double* coef, int ldo, int K,
               int obeg_min, int oend_max, double dt_out, cudaStream_t st,
               const int32_t* tcut) {
  (void)n_times;
  if (K <= 0 || oend_max <= obeg_min) return;
  dim3 grid((unsigned)((n + kRecThreads - 1) / kRecThreads),
            (unsigned)((oend_max - obeg_min + kOT - 1) / kOT));
  recombine_kernel<<<grid, kRecThreads, 0, st>>>(Xp, n, Vbase, vstride, Z, Zp, W, gstride, rc, mcol,
                                                  coef, ldo, K, obeg_min, dt_out, tcut);
}

void p_bound(const double* Z, const double* Zp, const double* W, int64_t gstride,
             const RoundCols& rc, int K, int64_t n, double* pbound, cudaStream_t st) {
  if (K <= 0) return;
  cudaMemsetAsync(pbound, 0, sizeof(double) * 2 * (size_t)K, st);
  const int64_t per = (int64_t)kPbThreads * kPbPer;
  dim3 grid((unsigned)((n + per - 1) / per), (unsigned)K);
  p_bound_kernel<<<grid, kPbThreads, 0, st>>>(Z, Zp, W, gstride, rc, n,
                                              reinterpret_cast<unsigned long long*>(pbound));
}

void next_state(double* X, const double* Vbase, int64_t vstride, const double* Z, const double* Zp,
                const double* W, int64_t gstride, const RoundCols& rc, const int32_t* mcol,
                const double* yend, int K, int64_t n, cudaStream_t st) {
  if (K <= 0) return;
  dim3 grid((unsigned)((n + 255) / 256), (unsigned)K);
  next_state_kernel<<<grid, 256, 0, st>>>(X, Vbase, vstride, Z, Zp, W, gstride, rc, mcol, yend, n);
}

void recombine_p(double* Xp, int64_t n, const double* Z, const double* Zp, const double* W,
                 int64_t gstride, const RoundCols& rc, const int32_t* ev_o, const int32_t* ev_q,
                 int nev, int o_begin, int o_end, double dt_out, cudaStream_t st) {
  if (nev <= 0 || o_end <= o_begin) return;
  recombine_p_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(Xp, n, Z, Zp, W, gstride, rc, ev_o,
                                                                  ev_q, nev, o_begin, o_end, dt_out);
}

void checkpoint_states(double* CK, double* X, double* Z, const int32_t* groups, int K, int64_t n,
                       bool restore, cudaStream_t st) {
  if (K <= 0) return;
  dim3 grid((unsigned)((n + 255) / 256), (unsigned)K);
  checkpoint_kernel<<<grid, 256, 0, st>>>(CK, X, Z, groups, n, restore ? 1 : 0);
}

void fill_rows(double* Xp, const double* base, int64_t n, int n_times, cudaStream_t st) {
  fill_rows_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Xp, base, n, n_times);
}

void add_row_sum(double* Xp, const double* Y, int ldy, int K, int64_t n, cudaStream_t st) {
  add_row_sum_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Xp, Y, ldy, K, n);
}

void permute_out(double* out, const double* Xp, const int32_t* map, int64_t nrows, int64_t n,
                 int n_times, cudaStream_t st) {
  dim3 grid((unsigned)((nrows + 255) / 256), (unsigned)n_times);
  permute_out_kernel<<<grid, 256, 0, st>>>(out, Xp, map, nrows, n);
}

}  // namespace matex
