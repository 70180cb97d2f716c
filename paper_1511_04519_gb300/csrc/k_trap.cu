// Fixed-step trapezoidal integration (Eq. 2) on the GPU: the comparison
// baseline of the paper (its TR with h = 10 ps), built from the same batched
// triangular solves as R-MATEX.  One step, scaled by h:
//   (C + h/2 G) x_{n+1} = (C - h/2 G) x_n + h/2 (b_n + b_{n+1}),
//   b(t) = B u(t) + dc_inject  (every source at once, no decomposition).
// Everything is in the factor's permuted node order.
#include "kernels.h"

namespace matex {

namespace {

constexpr int kTrThreads = 256;

__device__ __forceinline__ double pwl_value_at(const double* t, const double* v, int np, double x) {
  if (x <= t[0]) return v[0];
  if (x >= t[np - 1]) return v[np - 1];
  int j = 0;
  while (j + 1 < np && t[j + 1] <= x) ++j;
  return (v[j + 1] - v[j]) / (t[j + 1] - t[j]) * (x - t[j]) + v[j];
}

// b = dc (or 0)
__global__ void tr_fill_kernel(double* __restrict__ b, const double* __restrict__ dc, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = dc ? dc[i] : 0.0;
}

// b[node(s)] += u_s(t) for every source
__global__ void tr_sources_kernel(double* __restrict__ b, SourceTable src, int n_src, double t) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_src) return;
  const int o = src.pwl_off[s], np = src.pwl_off[s + 1] - o;
  atomicAdd(b + src.node[s], pwl_value_at(src.pwl_t + o, src.pwl_v + o, np, t));
}

// Y[i][0] = c_i x_i - g (G x)_i + g (bp_i + bn_i), G in CSR (permuted order)
__global__ void tr_rhs_kernel(double* __restrict__ Y, int ldy, const double* __restrict__ x,
                              const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                              const double* __restrict__ val, const double* __restrict__ c,
                              double g, const double* __restrict__ bp,
                              const double* __restrict__ bn, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double gx = 0.0;
  for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) gx = fma(val[k], x[col[k]], gx);
  Y[i * ldy] = fma(c[i], x[i], fma(-g, gx, g * (bp[i] + bn[i])));
}

// x = Y[.][0]; the state is also an output row when row >= 0
__global__ void tr_store_kernel(double* __restrict__ x, const double* __restrict__ Y, int ldy,
                                double* __restrict__ Xp, int64_t row, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = Y[i * ldy];
  x[i] = v;
  if (row >= 0) Xp[row * n + i] = v;
}

unsigned blocks(int64_t n) { return (unsigned)((n + kTrThreads - 1) / kTrThreads); }

}  // namespace

void tr_input(double* b, const double* dc, const SourceTable& src, int n_src, double t, int64_t n,
              cudaStream_t st) {
  tr_fill_kernel<<<blocks(n), kTrThreads, 0, st>>>(b, dc, n);
  if (n_src > 0) tr_sources_kernel<<<blocks(n_src), kTrThreads, 0, st>>>(b, src, n_src, t);
}

void tr_rhs(double* Y, int ldy, const double* x, const int64_t* rowptr, const int32_t* col,
            const double* val, const double* c, double g, const double* bp, const double* bn,
            int64_t n, cudaStream_t st) {
  tr_rhs_kernel<<<blocks(n), kTrThreads, 0, st>>>(Y, ldy, x, rowptr, col, val, c, g, bp, bn, n);
}

void tr_store(double* x, const double* Y, int ldy, double* Xp, int64_t row, int64_t n,
              cudaStream_t st) {
  tr_store_kernel<<<blocks(n), kTrThreads, 0, st>>>(x, Y, ldy, Xp, row, n);
}

}  // namespace matex
