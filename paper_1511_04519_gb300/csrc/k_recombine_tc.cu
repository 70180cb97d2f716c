// FP64-accurate basis recombination on the tensor cores (the V y part of the
// recombination step, Eq. 6 at every output time of a segment round, Alg. 2).
//
// For one segment round, X[i][o] += sum_k V[i][k] Y[k][o], where k runs over
// the basis vectors of all the round's columns (K_dim = sum of their Krylov
// dimensions) and Y[k][o] is the coefficient of basis vector k at output o
// (zero where the column's segment does not hold o).  The product is a dense
// contraction, so it runs as an error-free slice decomposition on bf16
// tensor cores (the Ozaki scheme: Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012):
//
//   * every row i of V is scaled by a power of two 2^e_i > max_k |V[i][k]|
//     and cut into S = 9 base-64 digits, V[i][k] = 2^e_i sum_p a_p 64^-(p+1)
//     with a_p = sign(V[i][k]) d_p, d_p in [0, 63] the digits of the
//     magnitude (truncated after the ninth), exact in bf16; every column o of
//     Y likewise with 2^f_o and digits b_q;
//   * C_d = sum_{p+q=d} A_p B_q (d = 0..8) on the tensor cores: each product
//     of two digits is below 2^12, so a sum over at most 455 basis vectors
//     and up to nine digit pairs stays below 2^24, an integer that the FP32
//     accumulator holds exactly (no assumption on its rounding);
//   * X = 2^(e_i + f_o - 12) sum_d 64^-d C_d, combined in 64-bit integers and
//     converted to FP64 once.  The digits past the ninth and the pairs with
//     p + q > 8 are left out: together below 2^-52 of max|V[i][:]|
//     max|Y[:][o]| per term, the size of the rounding of an FP64 dot product.
//
// Kernels: tc_kmap (basis-vector table of the round), tc_split_rows (V
// slices in the MMA tile layout), tc_split_cols (Y slices), tc_gemm (bulk
// copies of the slice tiles into shared memory, tcgen05.mma into nine TMEM
// accumulators, integer combination and X += in the epilogue).
#include <cuda_bf16.h>

#include <algorithm>

#include "kernels.h"
#include "tcgen05_util.cuh"

namespace matex {

namespace {

using namespace tcx;

constexpr int kTcM = 128;          // nodes per tile (MMA M)
constexpr int kTcN = 48;           // outputs per tile (MMA N)
constexpr int kTcThreads = 128;
constexpr int kTcABytes = kTcM * kTcK * 2;  // one slice of an A tile: 8 KB
constexpr int kTcBBytes = kTcN * kTcK * 2;  // one slice of a B tile: 3 KB
constexpr int kTcStage = kTcS * (kTcABytes + kTcBBytes);
constexpr int kTcTmemCols = 512;

// kmap[k] = offset of basis vector k (slot * vstride + j * n) and kq[k] =
// (q << 5) | j, its column q and index j, for the round's columns in order;
// one thread.  Entries past the columns' total (only when a replay's counts
// disagree with the recording; the run is then discarded) are empty (-1).
__global__ void tc_kmap_kernel(const int32_t* __restrict__ vslot, const int32_t* __restrict__ mcol,
                               int K, int64_t vstride, int64_t n, int64_t* __restrict__ kmap,
                               int32_t* __restrict__ kq, int kdim) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int k = 0;
  for (int q = 0; q < K && k < kdim; ++q)
    for (int j = 0; j < mcol[q] && k < kdim; ++j, ++k) {
      kmap[k] = (int64_t)vslot[q] * vstride + (int64_t)j * n;
      kq[k] = (q << 5) | j;
    }
  for (; k < kdim; ++k) {
    kmap[k] = -1;
    kq[k] = -1;
  }
}

// V slices: one thread per node (row of V); A tile t = i / 128, K step s:
// block (t, s) holds kTcS slices of kTcM x kTcK bf16 in the core-matrix layout.
__global__ void __launch_bounds__(128)
tc_split_rows_kernel(const double* __restrict__ Vb, const int64_t* __restrict__ kmap, int kdim,
                     int ksteps, int64_t n, __nv_bfloat16* __restrict__ Aslices,
                     double* __restrict__ rowscale, const int32_t* __restrict__ abort) {
  if (abort && *abort) return;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t tiles = (n + kTcM - 1) / kTcM;
  if (i >= tiles * kTcM) return;
  const bool live = i < n;
  double mx = 0.0;
  if (live)
    for (int k = 0; k < kdim; ++k) {
      const int64_t off = kmap[k];
      if (off >= 0) mx = fmax(mx, fabs(Vb[off + i]));
    }
  const double sc = pow2_above(mx);
  if (live) rowscale[i] = sc;
  const double inv = 1.0 / sc;  // a power of two: exact
  const int64_t t = i / kTcM;
  const int r = (int)(i % kTcM);
  for (int s = 0; s < ksteps; ++s) {
    unsigned char* blk = reinterpret_cast<unsigned char*>(Aslices) +
                         ((size_t)t * ksteps + s) * (size_t)kTcS * kTcABytes;
    for (int k8 = 0; k8 < kTcK; k8 += 8) {
      float sl[8][kTcS];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int k = s * kTcK + k8 + u;
        double v = 0.0;
        if (live && k < kdim && kmap[k] >= 0) v = Vb[kmap[k] + i] * inv;
        slice9(v, sl[u]);
      }
#pragma unroll
      for (int p = 0; p < kTcS; ++p) {
        uint4 w;
        w.x = pack_bf16x2(sl[0][p], sl[1][p]);
        w.y = pack_bf16x2(sl[2][p], sl[3][p]);
        w.z = pack_bf16x2(sl[4][p], sl[5][p]);
        w.w = pack_bf16x2(sl[6][p], sl[7][p]);
        *reinterpret_cast<uint4*>(blk + (size_t)p * kTcABytes + tc_off(r, k8)) = w;
      }
    }
  }
}

// Y slices: one thread per output column o of the round's range (o0 + c);
// Y[k][o] = coefficient j of column q at o, zero where q's segment does not
// hold o.  B tile u = c / kTcN, K step s: kTcS slices of kTcN x kTcK.
__global__ void __launch_bounds__(128)
tc_split_cols_kernel(const double* __restrict__ coef, int ldo, const int32_t* __restrict__ obeg,
                     const int32_t* __restrict__ nout, const int32_t* __restrict__ kq, int kdim,
                     int ksteps, int o0, int nouts, __nv_bfloat16* __restrict__ Bslices,
                     double* __restrict__ colscale, const int32_t* __restrict__ abort) {
  if (abort && *abort) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int utiles = (nouts + kTcN - 1) / kTcN;
  if (c >= utiles * kTcN) return;
  const int o = o0 + c;
  const bool live = c < nouts;
  auto yval = [&](int k) -> double {
    if (!live || k >= kdim) return 0.0;
    const int e = kq[k];
    if (e < 0) return 0.0;
    const int q = e >> 5, j = e & 31;
    const int ob = obeg[q];
    if (o < ob || o >= ob + nout[q]) return 0.0;
    return coef[((int64_t)q * ldo + (o - ob)) * kCoefLd + j];
  };
  double mx = 0.0;
  for (int k = 0; k < kdim; ++k) mx = fmax(mx, fabs(yval(k)));
  const double sc = pow2_above(mx);
  colscale[c] = sc;
  const double inv = 1.0 / sc;
  const int u = c / kTcN, r = c % kTcN;
  for (int s = 0; s < ksteps; ++s) {
    unsigned char* blk = reinterpret_cast<unsigned char*>(Bslices) +
                         ((size_t)u * ksteps + s) * (size_t)kTcS * kTcBBytes;
    for (int k8 = 0; k8 < kTcK; k8 += 8) {
      float sl[8][kTcS];
#pragma unroll
      for (int e = 0; e < 8; ++e) slice9(yval(s * kTcK + k8 + e) * inv, sl[e]);
#pragma unroll
      for (int p = 0; p < kTcS; ++p) {
        uint4 w;
        w.x = pack_bf16x2(sl[0][p], sl[1][p]);
        w.y = pack_bf16x2(sl[2][p], sl[3][p]);
        w.z = pack_bf16x2(sl[4][p], sl[5][p]);
        w.w = pack_bf16x2(sl[6][p], sl[7][p]);
        *reinterpret_cast<uint4*>(blk + (size_t)p * kTcBBytes + tc_off(r, k8)) = w;
      }
    }
  }
}

// Instruction descriptor of this kernel's MMAs: M = 128 nodes, N = 48 outputs.
constexpr uint32_t kTcIdesc = tc_idesc(kTcM, kTcN);

struct TcGemm {
  const __nv_bfloat16* A;   // [node tiles][ksteps][kTcS][kTcM x kTcK]
  const __nv_bfloat16* B;   // [output tiles][ksteps][kTcS][kTcN x kTcK]
  const double* rowscale;   // [n]
  const double* colscale;   // [output tiles x kTcN]
  double* Xp;               // [n_times][n]
  int64_t n;
  int o0, nouts, ksteps;
  const int32_t* abort;
  int32_t* err;             // raised when a bounded wait gives up
};

// One CTA per (48-output tile, 128-node tile).  Thread 0 streams the slice
// tiles K step by K step into two shared-memory stages (bulk copies,
// completion by transaction count) and issues the MMAs of every slice pair
// p + q <= 8 into accumulator d = p + q (nine 128 x 48 FP32 accumulators in
// TMEM); every kTcChunk basis vectors all 128 threads drain the accumulators:
// warp w reads TMEM lanes 32w..32w+31 (its nodes), combines the nine integer
// sums exactly in 64-bit integers and adds the FP64 result into X.
__global__ void __launch_bounds__(kTcThreads, 1) tc_gemm_kernel(TcGemm g) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ uint32_t tbase;
  __shared__ __align__(8) uint64_t full[2], freed[2], fin;
  __shared__ int failed;
  if (g.abort && *g.abort) return;
  // output tiles fastest: the CTAs of one node tile run side by side and read
  // its V slices from DRAM once (the coefficient slices stay in L2)
  const int u = blockIdx.x, t = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tbase)),
                 "r"(kTcTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    mbar_init(&freed[0], 1);
    mbar_init(&freed[1], 1);
    mbar_init(&fin, 1);
    failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tbase;
  const int64_t i = (int64_t)t * kTcM + 32 * warp + lane;
  const bool live = i < g.n;
  const double rs = live ? g.rowscale[i] : 0.0;
  const int chunk_steps = kTcChunk / kTcK;
  int it = 0;  // K steps issued so far (stage = it & 1, use = it >> 1)
  int chunk = 0;
  for (int s0 = 0; s0 < g.ksteps; s0 += chunk_steps, ++chunk) {
    const int s1 = min(g.ksteps, s0 + chunk_steps);
    if (threadIdx.x == 0) {
      auto issue_copy = [&](int s, int k) {
        const int st = k & 1;
        unsigned char* a = tc_smem + (size_t)st * kTcStage;
        unsigned char* b = a + kTcS * kTcABytes;
        expect_tx(&full[st], kTcStage);
        bulk_load(a, reinterpret_cast<const unsigned char*>(g.A) +
                         ((size_t)t * g.ksteps + s) * (size_t)kTcS * kTcABytes,
                  kTcS * kTcABytes, &full[st]);
        bulk_load(b, reinterpret_cast<const unsigned char*>(g.B) +
                         ((size_t)u * g.ksteps + s) * (size_t)kTcS * kTcBBytes,
                  kTcS * kTcBBytes, &full[st]);
      };
      bool ok = true;
      // stage of step s0 was last used by step it - 2 (its MMAs must be done)
      if (it >= 2) ok = mbar_wait(&freed[it & 1], ((it >> 1) - 1) & 1);
      if (ok) issue_copy(s0, it);
      for (int s = s0; s < s1 && ok; ++s, ++it) {
        if (s + 1 < s1) {
          const int k = it + 1;
          if (k >= 2) ok = mbar_wait(&freed[k & 1], ((k >> 1) - 1) & 1);
          if (!ok) break;
          issue_copy(s + 1, k);
        }
        const int st = it & 1;
        if (!mbar_wait(&full[st], (it >> 1) & 1)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a = smem_addr(tc_smem + (size_t)st * kTcStage);
        const uint32_t b = a + kTcS * kTcABytes;
        // descriptors of the stage's first A and B slices; the others differ
        // only in the start address field (16-byte units, no carry: shared
        // memory addresses stay below 2^18)
        const uint64_t ad0 = tc_desc(a, 128, kTcSbo), bd0 = tc_desc(b, 128, kTcSbo);
        const uint32_t first = s == s0 ? 0u : 1u;
#pragma unroll
        for (int p = 0; p < kTcS; ++p)
#pragma unroll
          for (int q = 0; q + p < kTcS; ++q)
#pragma unroll
            for (int kk = 0; kk < kTcK; kk += 16) {
              const uint64_t ad = ad0 + (uint64_t)((p * kTcABytes + (kk / 8) * 128) >> 4);
              const uint64_t bd = bd0 + (uint64_t)((q * kTcBBytes + (kk / 8) * 128) >> 4);
              tc_mma(tmem + (uint32_t)((p + q) * kTcN), ad, bd, kTcIdesc,
                     (p == 0 && kk == 0) ? first : 1u);
            }
        tc_commit(&freed[st]);
      }
      if (ok) tc_commit(&fin);
      else failed = 1;
    }
    __syncthreads();
    if (failed) break;
    if (!mbar_wait(&fin, chunk & 1)) {
      failed = 1;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // drain: C_d at TMEM column d * kTcN + c of this warp's lanes
#pragma unroll 1
    for (int cb = 0; cb < kTcN; cb += 8) {
      uint32_t v[kTcS][8];
#pragma unroll
      for (int d = 0; d < kTcS; ++d)
        tc_ld8(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(d * kTcN + cb), v[d]);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int c = u * kTcN + cb + j;
        if (!live || c >= g.nouts) continue;
        long long hi = 0, lo = 0;
#pragma unroll
        for (int d = 0; d < 5; ++d)
          hi += (long long)__float2int_rz(__uint_as_float(v[d][j])) * (1ll << (6 * (4 - d)));
#pragma unroll
        for (int d = 5; d < kTcS; ++d)
          lo += (long long)__float2int_rz(__uint_as_float(v[d][j])) * (1ll << (6 * (8 - d)));
        const double val = fma((double)lo, 0x1p-24, (double)hi) * (rs * g.colscale[c] * 0x1p-36);
        double* x = g.Xp + (int64_t)(g.o0 + c) * g.n + i;
        *x += val;
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  if (failed && threadIdx.x == 0) {
    atomicExch(g.err, 1);
    // let the MMAs already issued finish before the accumulators are freed:
    // `fin` has completed `chunk` phases; this commit completes the next one
    tc_commit(&fin);
    mbar_wait(&fin, chunk & 1);  // bounded: gives up after about two seconds as well
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTcTmemCols));
  }
}

}  // namespace

// ---- host side ------------------------------------------------------------------

size_t tc_slices_bytes(int64_t n, int kdim, int nouts) {
  const int64_t tn = (n + kTcM - 1) / kTcM, tu = (nouts + kTcN - 1) / kTcN;
  const int64_t ks = (kdim + kTcK - 1) / kTcK;
  return (size_t)(tn * ks * kTcS * kTcABytes + tu * ks * kTcS * kTcBBytes);
}

void tc_set_limits() {
  cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * kTcStage);
}

int recombine_tc(double* Xp, int64_t n, const double* Vbase, int64_t vstride, const RoundCols& rc,
                 const int32_t* mcol, const double* coef, int ldo, int K, int kdim, int obeg_min,
                 int oend_max, const TcScratch& ts, cudaStream_t st) {
  const int nouts = oend_max - obeg_min;
  if (K <= 0 || kdim <= 0 || nouts <= 0) return 0;
  const int ksteps = (kdim + kTcK - 1) / kTcK;
  const int64_t tn = (n + kTcM - 1) / kTcM;
  const int tu = (nouts + kTcN - 1) / kTcN;
  __nv_bfloat16* A = reinterpret_cast<__nv_bfloat16*>(ts.slices);
  __nv_bfloat16* B = A + (size_t)tn * ksteps * kTcS * (kTcABytes / 2);
  tc_kmap_kernel<<<1, 32, 0, st>>>(rc.vslot, mcol, K, vstride, n, ts.kmap, ts.kq, kdim);
  tc_split_rows_kernel<<<(unsigned)tn, kTcM, 0, st>>>(Vbase, ts.kmap, kdim, ksteps, n, A,
                                                      ts.rowscale, rc.abort);
  tc_split_cols_kernel<<<(unsigned)((tu * kTcN + 127) / 128), 128, 0, st>>>(
      coef, ldo, rc.obeg, rc.nout, ts.kq, kdim, ksteps, obeg_min, nouts, B, ts.colscale, rc.abort);
  TcGemm g{A, B, ts.rowscale, ts.colscale, Xp, n, obeg_min, nouts, ksteps, rc.abort, ts.err};
  tc_gemm_kernel<<<dim3((unsigned)tu, (unsigned)tn), kTcThreads, 2 * kTcStage, st>>>(g);
  return 4;
}

}  // namespace matex
