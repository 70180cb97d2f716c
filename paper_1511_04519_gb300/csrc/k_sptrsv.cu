// Multi-right-hand-side supernodal triangular solves with the once-factorised
// M = L D L^T (Alg. 1: "a pair of forward and backward substitutions",
// w = U \ (L \ (X2 v_j)); here X1 = C + gamma G or G, both SPD, so U = D L^T).
//
// Layout: the right-hand sides live node-major in Y[n][ldy] (permuted node
// order), so the K columns of one row are contiguous.  A task is one
// (supernode, column block) pair; one launch covers one level of the
// supernodal elimination tree.
//   forward : y_s = L_ss^{-1} b_s  (unit lower, dense, in shared memory);
//             b_R -= L_Rs y_s pushed to the ancestors' rows with FP64 atomics.
//   backward: x_s = L_ss^{-T} (D_s^{-1} y_s - L_Rs^T x_R), pulling the final
//             x_R of the ancestors (already solved one level up).
#include "kernels.h"

namespace matex {

namespace {

constexpr int kSolveThreads = 128;

template <int KB>
__global__ void __launch_bounds__(kSolveThreads)
fwd_level_kernel(DevFactor F, const int32_t* __restrict__ sups, int ncb, double* __restrict__ Y,
                 int ldy) {
  extern __shared__ double sb[];  // [w][KB]
  const int t = blockIdx.x;
  const int s = sups[t / ncb];
  const int c0 = (t % ncb) * KB;
  const int f = F.sup_first[s];
  const int w = F.sup_first[s + 1] - f;
  const int64_t rp = F.sup_rowptr[s];
  const int r = (int)(F.sup_rowptr[s + 1] - rp) - w;
  for (int e = threadIdx.x; e < w * KB; e += blockDim.x) {
    const int i = e / KB, q = e - i * KB;
    sb[e] = Y[(int64_t)(f + i) * ldy + c0 + q];
  }
  __syncthreads();
  const double* __restrict__ Lc = F.diag_cm + F.diag_off[s];
  for (int j = 0; j < w - 1; ++j) {
    const int cnt = (w - 1 - j) * KB;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int ii = e / KB, q = e - ii * KB;
      const int i = j + 1 + ii;
      sb[i * KB + q] -= Lc[i + j * w] * sb[j * KB + q];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < w * KB; e += blockDim.x) {
    const int i = e / KB, q = e - i * KB;
    Y[(int64_t)(f + i) * ldy + c0 + q] = sb[e];
  }
  if (r == 0) return;
  const double* __restrict__ Oc = F.offd_cm + F.offd_off[s];
  const int32_t* __restrict__ rows = F.sup_rows + rp + w;
  for (int e = threadIdx.x; e < r * KB; e += blockDim.x) {
    const int q = e / r, i = e - q * r;
    double acc = 0.0;
    for (int j = 0; j < w; ++j) acc = fma(Oc[i + (int64_t)j * r], sb[j * KB + q], acc);
    atomicAdd(&Y[(int64_t)rows[i] * ldy + c0 + q], -acc);
  }
}

template <int KB>
__global__ void __launch_bounds__(kSolveThreads)
bwd_level_kernel(DevFactor F, const int32_t* __restrict__ sups, int ncb, double* __restrict__ Y,
                 int ldy) {
  extern __shared__ double sb[];  // [w][KB]
  const int t = blockIdx.x;
  const int s = sups[t / ncb];
  const int c0 = (t % ncb) * KB;
  const int f = F.sup_first[s];
  const int w = F.sup_first[s + 1] - f;
  const int64_t rp = F.sup_rowptr[s];
  const int r = (int)(F.sup_rowptr[s + 1] - rp) - w;
  const double* __restrict__ Or = F.offd_rm + F.offd_off[s];
  const int32_t* __restrict__ rows = F.sup_rows + rp + w;
  for (int e = threadIdx.x; e < w * KB; e += blockDim.x) {
    const int q = e / w, j = e - q * w;
    double acc = Y[(int64_t)(f + j) * ldy + c0 + q] * F.dinv[f + j];
    for (int i = 0; i < r; ++i)
      acc = fma(-Or[(int64_t)i * w + j], Y[(int64_t)rows[i] * ldy + c0 + q], acc);
    sb[j * KB + q] = acc;
  }
  __syncthreads();
  const double* __restrict__ Lr = F.diag_rm + F.diag_off[s];
  for (int j = w - 1; j > 0; --j) {
    const int cnt = j * KB;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int i = e / KB, q = e - i * KB;
      sb[i * KB + q] -= Lr[j * w + i] * sb[j * KB + q];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < w * KB; e += blockDim.x) {
    const int i = e / KB, q = e - i * KB;
    Y[(int64_t)(f + i) * ldy + c0 + q] = sb[e];
  }
}

template <int KB>
void launch_level(bool fwd, const DevFactor& F, const LevelPlan& L, double* Y, int ldy, int ncols,
                  cudaStream_t st) {
  const int ncb = (ncols + KB - 1) / KB;
  const size_t smem = (size_t)L.max_w * KB * sizeof(double);
  dim3 grid((unsigned)(L.count * ncb));
  if (fwd)
    fwd_level_kernel<KB><<<grid, kSolveThreads, smem, st>>>(F, L.sups, ncb, Y, ldy);
  else
    bwd_level_kernel<KB><<<grid, kSolveThreads, smem, st>>>(F, L.sups, ncb, Y, ldy);
}

void run_level(bool fwd, const DevFactor& F, const LevelPlan& L, double* Y, int ldy, int ncols,
               cudaStream_t st) {
  int kb = L.kb;
  while (kb > 1 && kb / 2 >= ncols) kb /= 2;
  switch (kb) {
    case 1: launch_level<1>(fwd, F, L, Y, ldy, ncols, st); break;
    case 2: launch_level<2>(fwd, F, L, Y, ldy, ncols, st); break;
    case 4: launch_level<4>(fwd, F, L, Y, ldy, ncols, st); break;
    default: launch_level<8>(fwd, F, L, Y, ldy, ncols, st); break;
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

int solve_inplace(const DevFactor& F, const LevelPlan* levels, int nlev, double* Y, int ldy,
                  int ncols, cudaStream_t st) {
  if (ncols <= 0) return 0;
  for (int l = 0; l < nlev; ++l) run_level(true, F, levels[l], Y, ldy, ncols, st);
  for (int l = nlev - 1; l >= 0; --l) run_level(false, F, levels[l], Y, ldy, ncols, st);
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
