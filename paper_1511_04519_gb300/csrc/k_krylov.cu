// Krylov-side kernels of batched R-MATEX: segment inputs (Eq. 5/6), the start
// vector v = x(t) + F, Gram-Schmidt (two classical passes; Alg. 1 writes
// modified Gram-Schmidt, which CGS2 matches to rounding), the rational
// Hessenberg map H_m = (I - Htilde_m^{-1})/gamma (Eq. 9), the residual test of
// Sec. 3.3.3 and the coefficient vectors ||v|| e^{h H_m} e_1 at the output
// times of a segment (Alg. 2, "snapshots" reuse the basis).
#include "kernels.h"
#include "column_steps.cuh"

namespace matex {

namespace {

__global__ void input_rhs_kernel(double* __restrict__ Y, int ldy, int K, RoundCols rc,
                                 SourceTable src) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= K) return;
  const int g = rc.sgroup ? rc.sgroup[q] : rc.group[q];
  const double l0 = rc.l0[q], L = rc.len[q], l1 = l0 + L;
  for (int p = src.grp_ptr[g]; p < src.grp_ptr[g + 1]; ++p) {
    const int s = src.grp_src[p];
    const int o = src.pwl_off[s], np = src.pwl_off[s + 1] - o;
    const double u0 = pwl_eval(src.pwl_t + o, src.pwl_v + o, np, l0);
    const double val = (pwl_eval(src.pwl_t + o, src.pwl_v + o, np, l1) - u0) / L;
    Y[(int64_t)src.node[s] * ldy + q] += val;
  }
}

__global__ void advance_z_kernel(double* __restrict__ Z, const double* __restrict__ Zp,
                                 const double* __restrict__ X, int64_t gstride, RoundCols rc,
                                 int64_t n) {
  const int q = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t g = rc.group[q];
  const int64_t k = g * gstride + i;
  if (rc.seg[q] == 0) Z[k] = X[k];
  else Z[k] = fma(rc.lprev[q], Zp[k], Z[k]);
}

__global__ void initial_rhs_kernel(double* __restrict__ Y, int ldy, int K, SourceTable src,
                                   const int32_t* __restrict__ groups) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= K) return;
  const int g = groups[q];
  for (int p = src.grp_ptr[g]; p < src.grp_ptr[g + 1]; ++p) {
    const int s = src.grp_src[p];
    const int o = src.pwl_off[s], np = src.pwl_off[s + 1] - o;
    Y[(int64_t)src.node[s] * ldy + q] += pwl_eval(src.pwl_t + o, src.pwl_v + o, np, 0.0);
  }
}

constexpr int kRedThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;  // valid in thread 0
}

__global__ void __launch_bounds__(kRedThreads)
krylov_start_kernel(double* __restrict__ Vb, int64_t vstride, const double* __restrict__ X,
                    const double* __restrict__ Z, const double* __restrict__ W, int64_t gstride,
                    const int32_t* __restrict__ groups, const int32_t* __restrict__ vslots,
                    int64_t n, double* __restrict__ partials, int nchunks) {
  __shared__ double red[32];
  const int q = blockIdx.y;
  const int64_t g = groups[q];
  const int64_t vs = vslots[q];
  const int64_t b = (int64_t)blockIdx.x * kChunk;
  const int64_t e = min(n, b + kChunk);
  double acc = 0.0;
  for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) {
    const double v = X[g * gstride + i] + (W[g * gstride + i] - Z[g * gstride + i]);
    Vb[vs * vstride + i] = v;
    acc = fma(v, v, acc);
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) partials[(int64_t)q * nchunks + blockIdx.x] = s;
}

// Dot products of w (slot wslot) with NB basis slots first..first+NB-1 over one
// chunk of nodes; NB is a template parameter so no predicated FP64 work is
// issued for slots that do not exist (the FP64 pipe counts those too).
template <int NB>
__device__ __forceinline__ void dots_chunk(const double* __restrict__ base, const double* __restrict__ w,
                                           int first, int64_t n, int64_t b, int64_t e,
                                           double* __restrict__ out, int nchunks, double* red) {
  double acc[NB];
#pragma unroll
  for (int i = 0; i < NB; ++i) acc[i] = 0.0;
  for (int64_t x = b + threadIdx.x; x < e; x += blockDim.x) {
    const double wx = w[x];
#pragma unroll
    for (int i = 0; i < NB; ++i) acc[i] = fma(base[(int64_t)(first + i) * n + x], wx, acc[i]);
  }
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const double s = block_sum(acc[i], red);
    if (threadIdx.x == 0) out[(int64_t)i * nchunks] = s;
  }
}

__global__ void __launch_bounds__(kRedThreads)
basis_dots_kernel(const double* __restrict__ Vb, int64_t vstride, const int32_t* __restrict__ groups,
                  const int32_t* __restrict__ iter, int first, int nb, int wslot, int64_t n,
                  double* __restrict__ partials, int nchunks) {
  __shared__ double red[32];
  const int q = iter[blockIdx.y];
  const int64_t g = groups[q];
  const double* __restrict__ base = Vb + g * vstride;
  const double* __restrict__ w = base + (int64_t)wslot * n;
  const int64_t b = (int64_t)blockIdx.x * kChunk;
  const int64_t e = min(n, b + kChunk);
  double* out = partials + ((int64_t)q * kMaxB) * nchunks + blockIdx.x;
  switch (nb) {
#define MATEX_DC(NB) \
  case NB: dots_chunk<NB>(base, w, first, n, b, e, out, nchunks, red); break;
    MATEX_DC(1) MATEX_DC(2) MATEX_DC(3) MATEX_DC(4) MATEX_DC(5) MATEX_DC(6) MATEX_DC(7)
    MATEX_DC(8) MATEX_DC(9) MATEX_DC(10) MATEX_DC(11) MATEX_DC(12) MATEX_DC(13) MATEX_DC(14)
    MATEX_DC(15) MATEX_DC(16) MATEX_DC(17) MATEX_DC(18) MATEX_DC(19) MATEX_DC(20) MATEX_DC(21)
#undef MATEX_DC
    default: break;
  }
}

__global__ void basis_update_kernel(double* __restrict__ Vb, int64_t vstride,
                                    const int32_t* __restrict__ groups,
                                    const int32_t* __restrict__ iter, int nb, int wslot,
                                    const double* __restrict__ h, int64_t n) {
  const int q = iter[blockIdx.y];
  const int64_t g = groups[q];
  double* __restrict__ base = Vb + g * vstride;
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= n) return;
  double acc = base[(int64_t)wslot * n + x];
  for (int i = 0; i < nb; ++i) acc = fma(-h[q * kMaxB + i], base[(int64_t)i * n + x], acc);
  base[(int64_t)wslot * n + x] = acc;
}

__global__ void basis_scale_kernel(double* __restrict__ Vb, int64_t vstride,
                                   const int32_t* __restrict__ groups,
                                   const int32_t* __restrict__ iter, int wslot,
                                   const double* __restrict__ scale, int64_t n) {
  const int q = iter[blockIdx.y];
  const int64_t g = groups[q];
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= n) return;
  Vb[g * vstride + (int64_t)wslot * n + x] *= scale[q];
}

__global__ void start_finish_kernel(const double* __restrict__ partials, int nchunks, int K,
                                    SmallState ss, const int32_t* __restrict__ groups,
                                    int32_t* iter_out, int32_t* iter_grp, int32_t* iter_count) {
  // one thread per column, then a serial compaction by thread 0 (K <= a few hundred)
  const int q = threadIdx.x;
  for (int c = q; c < K; c += blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < nchunks; ++k) s += partials[(int64_t)c * nchunks + k];
    const double beta = sqrt(s);
    ss.beta[c] = beta;
    ss.m[c] = 0;
    for (int i = 0; i < kMaxB * kMaxM; ++i) ss.Ht[(int64_t)c * kMaxB * kMaxM + i] = 0.0;
    if (beta <= 1e-300) {
      ss.status[c] = 4;
      ss.scale[c] = 0.0;
    } else {
      ss.status[c] = 0;
      ss.scale[c] = 1.0 / beta;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int cnt = 0;
    for (int c = 0; c < K; ++c)
      if (ss.status[c] == 0) {
        iter_grp[cnt] = groups[c];
        iter_out[cnt++] = c;
      }
    *iter_count = cnt;
  }
}

__global__ void reduce_dots_kernel(const double* __restrict__ partials, int nchunks, int nb,
                                   const int32_t* __restrict__ iter, SmallState ss, int j,
                                   int mode) {
  const int q = iter[blockIdx.x];
  const int i = threadIdx.x;
  if (i >= nb) return;
  double s = 0.0;
  for (int k = 0; k < nchunks; ++k) s += partials[((int64_t)q * kMaxB + i) * nchunks + k];
  double* Ht = ss.Ht + (int64_t)q * kMaxB * kMaxM;
  if (mode == 2) {
    const double nrm = sqrt(s);
    Ht[(j + 1) * kMaxM + j] = nrm;
    ss.scale[q] = nrm > 0.0 ? 1.0 / nrm : 0.0;
  } else {
    ss.hbuf[q * kMaxB + i] = s;
    Ht[i * kMaxM + j] += s;
  }
}

__global__ void __launch_bounds__(kSmallThreads)
residual_kernel(SmallState ss, RoundCols rc, const int32_t* __restrict__ iter, int j, double gamma,
                double tol, int m_max, const int32_t* __restrict__ replay) {
  extern __shared__ double smem_raw[];
  SmallShared& sh = *reinterpret_cast<SmallShared*>(smem_raw);
  residual_column(ss, rc, iter[blockIdx.x], j, gamma, tol, m_max, replay, sh);
}

__global__ void compact_kernel(SmallState ss, const int32_t* __restrict__ groups,
                               const int32_t* __restrict__ iter_in, int K_in,
                               int32_t* __restrict__ iter_out, int32_t* __restrict__ iter_grp,
                               int32_t* __restrict__ count) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int c = 0;
  for (int p = 0; p < K_in; ++p) {
    const int q = iter_in[p];
    if (ss.status[q] == 0) {
      iter_grp[c] = groups[q];
      iter_out[c++] = q;
    }
  }
  *count = c;
}

__global__ void record_kernel(SmallState ss, RoundCols rc, int K, int32_t* m_rec, int32_t* st_rec) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= K) return;
  m_rec[rc.segid[q]] = ss.m[q];
  st_rec[rc.segid[q]] = ss.status[q];
}

__global__ void __launch_bounds__(kSmallThreads)
coef_kernel(SmallState ss, RoundCols rc, double gamma, double dt_out, double* __restrict__ coef,
            int ldo, double* __restrict__ yend, double tail_eps, const double* __restrict__ pbound,
            int32_t* __restrict__ tcut) {
  extern __shared__ double smem_raw[];
  SmallShared& sh = *reinterpret_cast<SmallShared*>(smem_raw);
  if (threadIdx.x == 0) sh.cm = 0;  // no residual test ran in this CTA
  __syncthreads();
  coef_column(ss, rc, blockIdx.x, gamma, dt_out, coef, ldo, yend, tail_eps, pbound, tcut, sh);
}

__global__ void __launch_bounds__(kSmallThreads)
expm_batch_kernel(int m, const double* __restrict__ A, const double* __restrict__ h,
                  double* __restrict__ E) {
  extern __shared__ double smem_raw[];
  SmallShared& sh = *reinterpret_cast<SmallShared*>(smem_raw);
  const int b = blockIdx.x;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e - i * m;
    sh.H[i * kLd + j] = A[(int64_t)b * m * m + e];
  }
  __syncthreads();
  expm_dev(sh.H, h[b], sh.E, m, sh.w);
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e - i * m;
    E[(int64_t)b * m * m + e] = sh.E[i * kLd + j];
  }
}

}  // namespace

void build_input_rhs(double* Y, int ldy, int K, const RoundCols& rc, const SourceTable& src,
                     int64_t n, cudaStream_t st) {
  cudaMemsetAsync(Y, 0, sizeof(double) * (size_t)n * ldy, st);
  input_rhs_kernel<<<(K + 127) / 128, 128, 0, st>>>(Y, ldy, K, rc, src);
}

void advance_z(double* Z, const double* Zp, const double* X, int64_t gstride, const RoundCols& rc,
               int K, int64_t n, cudaStream_t st) {
  if (K <= 0) return;
  dim3 grid((unsigned)((n + 255) / 256), (unsigned)K);
  advance_z_kernel<<<grid, 256, 0, st>>>(Z, Zp, X, gstride, rc, n);
}

void build_initial_rhs(double* Y, int ldy, int K, const SourceTable& src, const int32_t* groups,
                       int64_t n, cudaStream_t st) {
  cudaMemsetAsync(Y, 0, sizeof(double) * (size_t)n * ldy, st);
  initial_rhs_kernel<<<(K + 127) / 128, 128, 0, st>>>(Y, ldy, K, src, groups);
}

void krylov_start(double* Vbase, int64_t vstride, const double* X, const double* Z, const double* W,
                  int64_t gstride, const int32_t* groups, const int32_t* vslots, int K, int64_t n,
                  double* partials, int nchunks, cudaStream_t st) {
  dim3 grid((unsigned)nchunks, (unsigned)K);
  krylov_start_kernel<<<grid, kRedThreads, 0, st>>>(Vbase, vstride, X, Z, W, gstride, groups,
                                                    vslots, n, partials, nchunks);
}

void basis_dots(const double* Vbase, int64_t vstride, const int32_t* groups, const int32_t* iter,
                int K, int first, int nb, int wslot, int64_t n, double* partials, int nchunks,
                cudaStream_t st) {
  dim3 grid((unsigned)nchunks, (unsigned)K);
  basis_dots_kernel<<<grid, kRedThreads, 0, st>>>(Vbase, vstride, groups, iter, first, nb, wslot,
                                                  n, partials, nchunks);
}

void basis_update(double* Vbase, int64_t vstride, const int32_t* groups, const int32_t* iter, int K,
                  int nb, int wslot, const double* h, int64_t n, cudaStream_t st) {
  dim3 grid((unsigned)((n + 255) / 256), (unsigned)K);
  basis_update_kernel<<<grid, 256, 0, st>>>(Vbase, vstride, groups, iter, nb, wslot, h, n);
}

void basis_scale(double* Vbase, int64_t vstride, const int32_t* groups, const int32_t* iter, int K,
                 int wslot, const double* scale, int64_t n, cudaStream_t st) {
  dim3 grid((unsigned)((n + 255) / 256), (unsigned)K);
  basis_scale_kernel<<<grid, 256, 0, st>>>(Vbase, vstride, groups, iter, wslot, scale, n);
}

void start_finish(const double* partials, int nchunks, int K, SmallState ss, const int32_t* groups,
                  int32_t* iter_out, int32_t* iter_grp, int32_t* iter_count, cudaStream_t st) {
  start_finish_kernel<<<1, 256, 0, st>>>(partials, nchunks, K, ss, groups, iter_out, iter_grp,
                                         iter_count);
}

void reduce_dots(const double* partials, int nchunks, int K, int nb, const int32_t* iter,
                 SmallState ss, int j, int mode, cudaStream_t st) {
  reduce_dots_kernel<<<K, 32, 0, st>>>(partials, nchunks, nb, iter, ss, j, mode);
}

namespace {
__global__ void apply_A_kernel(double* __restrict__ Vb, int64_t vstride,
                               const int32_t* __restrict__ iter_grp, int jsrc, int jdst,
                               const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                               const double* __restrict__ val, const double* __restrict__ c,
                               int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double* __restrict__ v = Vb + (int64_t)iter_grp[blockIdx.y] * vstride + (int64_t)jsrc * n;
  double gv = 0.0;
  for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) gv = fma(val[k], v[col[k]], gv);
  Vb[(int64_t)iter_grp[blockIdx.y] * vstride + (int64_t)jdst * n + i] = -gv / c[i];
}

__global__ void expect_count_kernel(const int32_t* __restrict__ count, int expected,
                                    int32_t* __restrict__ iter, int32_t* __restrict__ iter_grp,
                                    const int32_t* __restrict__ vslot, int32_t* __restrict__ flag) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int got = *count;
  if (got == expected) return;
  *flag = 1;
  for (int k = got > 0 ? got : 0; k < expected; ++k) {
    iter[k] = 0;
    iter_grp[k] = vslot[0];
  }
}
}  // namespace

void krylov_apply_A(double* Vb, int64_t vstride, const int32_t* iter_grp, int K, int jsrc, int jdst,
                    const int64_t* rowptr, const int32_t* col, const double* val, const double* c,
                    int64_t n, cudaStream_t st) {
  if (K <= 0) return;
  dim3 grid((unsigned)((n + 255) / 256), (unsigned)K);
  apply_A_kernel<<<grid, 256, 0, st>>>(Vb, vstride, iter_grp, jsrc, jdst, rowptr, col, val, c, n);
}

void expect_count(const int32_t* count, int expected, int32_t* iter, int32_t* iter_grp,
                  const int32_t* vslot, int32_t* flag, cudaStream_t st) {
  expect_count_kernel<<<1, 32, 0, st>>>(count, expected, iter, iter_grp, vslot, flag);
}

void residual_check(SmallState ss, const RoundCols& rc, int K, int j, double gamma, double tol,
                    int m_max, const int32_t* replay, const int32_t* iter_in, int32_t* iter_out,
                    int32_t* iter_grp, int32_t* iter_count, cudaStream_t st) {
  const size_t smem = sizeof(SmallShared);
  residual_kernel<<<K, kSmallThreads, smem, st>>>(ss, rc, iter_in, j, gamma, tol, m_max, replay);
  compact_kernel<<<1, 32, 0, st>>>(ss, rc.vslot, iter_in, K, iter_out, iter_grp, iter_count);
}

void record_segments(const SmallState& ss, const RoundCols& rc, int K, int32_t* m_rec,
                     int32_t* st_rec, cudaStream_t st) {
  if (K <= 0) return;
  record_kernel<<<(K + 127) / 128, 128, 0, st>>>(ss, rc, K, m_rec, st_rec);
}

void output_coefficients(SmallState ss, const RoundCols& rc, int K, double gamma, double dt_out,
                         double* coef, int ldo, double* yend, cudaStream_t st, double tail_eps,
                         const double* pbound, int32_t* tcut) {
  const size_t smem = sizeof(SmallShared);
  coef_kernel<<<K, kSmallThreads, smem, st>>>(ss, rc, gamma, dt_out, coef, ldo, yend, tail_eps,
                                              pbound, tcut);
}

void expm_batch(int batch, int m, const double* A, const double* h, double* E, cudaStream_t st) {
  const size_t smem = sizeof(SmallShared);
  expm_batch_kernel<<<batch, kSmallThreads, smem, st>>>(m, A, h, E);
}

size_t small_shared_bytes() { return sizeof(SmallShared); }

void set_small_smem_limits() {
  const int bytes = (int)sizeof(SmallShared);
  cudaFuncSetAttribute(residual_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(coef_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(expm_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

}  // namespace matex
