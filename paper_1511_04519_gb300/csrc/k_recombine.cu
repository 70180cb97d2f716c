// Basis recombination and superposition (Alg. 1 last line, Alg. 2 snapshots,
// and the scheduler's sum of group responses, Sec. 3.2):
//   x_k(t_o) = V_k y_k(t_o) + z_k + (t_o - l_j) z'_k - w_k     (Eq. 6 with -P)
//   X[o]    += sum over the round's groups whose segment holds t_o.
// Each thread owns one node and a tile of output times; the groups are summed
// in registers in a fixed order, so a round writes each output entry once.
#include "kernels.h"

namespace matex {

namespace {

constexpr int kRecThreads = 128;
constexpr int kOT = 8;  // output times per thread

__global__ void __launch_bounds__(kRecThreads)
recombine_kernel(double* __restrict__ Xp, int64_t n, const double* __restrict__ Vb, int64_t vstride,
                 const double* __restrict__ Z, const double* __restrict__ Zp,
                 const double* __restrict__ W, int64_t gstride, RoundCols rc,
                 const int32_t* __restrict__ mcol, const double* __restrict__ coef, int ldo, int K,
                 int obeg_min, double dt_out) {
  const int64_t i = (int64_t)blockIdx.x * kRecThreads + threadIdx.x;
  const int o0 = obeg_min + blockIdx.y * kOT;
  if (i >= n) return;
  double acc[kOT];
#pragma unroll
  for (int t = 0; t < kOT; ++t) acc[t] = 0.0;
  bool touched = false;
  for (int q = 0; q < K; ++q) {
    const int ob = rc.obeg[q], no = rc.nout[q];
    const int lo = max(ob, o0), hi = min(ob + no, o0 + kOT);
    if (lo >= hi) continue;
    touched = true;
    const int64_t g = rc.group[q];
    const int m = mcol[q];
    double v[kMaxM];
    const double* __restrict__ base = Vb + g * vstride + i;
#pragma unroll
    for (int j = 0; j < kMaxM; ++j) v[j] = (j < m) ? base[(int64_t)j * n] : 0.0;
    const double z = Z[g * gstride + i], zp = Zp[g * gstride + i], w = W[g * gstride + i];
    const double l0 = rc.l0[q];
    const double* __restrict__ cq = coef + (int64_t)q * ldo * kMaxM;
#pragma unroll
    for (int t = 0; t < kOT; ++t) {
      const int o = o0 + t;
      if (o < lo || o >= hi) continue;
      const double h = (double)o * dt_out - l0;
      double s = z + h * zp - w;
      const double* __restrict__ y = cq + (int64_t)(o - ob) * kMaxM;
#pragma unroll
      for (int j = 0; j < kMaxM; ++j)
        if (j < m) s = fma(v[j], y[j], s);
      acc[t] += s;
    }
  }
  if (!touched) return;
#pragma unroll
  for (int t = 0; t < kOT; ++t) {
    const int o = o0 + t;
    bool any = false;
    for (int q = 0; q < K; ++q) {
      const int ob = rc.obeg[q], no = rc.nout[q];
      if (o >= ob && o < ob + no) { any = true; break; }
    }
    if (any) Xp[(int64_t)o * n + i] += acc[t];
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
  const double* __restrict__ base = Vb + g * vstride + i;
  for (int j = 0; j < m; ++j) s = fma(base[(int64_t)j * n], yend[q * kMaxM + j], s);
  X[g * gstride + i] = s;
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
               int obeg_min, int oend_max, double dt_out, cudaStream_t st) {
  (void)n_times;
  if (K <= 0 || oend_max <= obeg_min) return;
  dim3 grid((unsigned)((n + kRecThreads - 1) / kRecThreads),
            (unsigned)((oend_max - obeg_min + kOT - 1) / kOT));
  recombine_kernel<<<grid, kRecThreads, 0, st>>>(Xp, n, Vbase, vstride, Z, Zp, W, gstride, rc, mcol,
                                                  coef, ldo, K, obeg_min, dt_out);
}

void next_state(double* X, const double* Vbase, int64_t vstride, const double* Z, const double* Zp,
                const double* W, int64_t gstride, const RoundCols& rc, const int32_t* mcol,
                const double* yend, int K, int64_t n, cudaStream_t st) {
  if (K <= 0) return;
  dim3 grid((unsigned)((n + 255) / 256), (unsigned)K);
  next_state_kernel<<<grid, 256, 0, st>>>(X, Vbase, vstride, Z, Zp, W, gstride, rc, mcol, yend, n);
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
