// Wide supernodes of the triangular solves (Alg. 1's operator apply) on the
// bf16 tensor cores, FP64-accurate by the same error-free digit split as the
// recombination (tcgen05_util.cuh).
//
// For a supernode s of width w with ld = w + r panel rows and K right-hand
// sides, the two substitutions inside s are dense products (k_sptrsv.cu):
//   forward : [y_s; u_R] = P_s b_s        (ld x w) times (w x K)
//   backward: x_s = P_s^T [D_s^{-1} y_s; -x_R]   (w x ld) times (ld x K)
// On the bench grid the supernodes at least 64 wide hold a third of the panel
// entries, on the 1.44M-node grid three fifths, and there the products have
// tens to hundreds of right-hand sides: dense contractions that the FP64 pipe
// (2 FMA per SM per clock on GB300) runs slowly.  Here every panel row is
// scaled by a power of two and split into nine signed 6-bit digits once at
// setup (both directions, both factors, in the MMA tile layout); the
// right-hand sides are split per call, per column and K slice; the 45
// digit-pair products
// with p + q <= 8 accumulate exactly in FP32 TMEM accumulators (sums below
// 2^24) and are combined in 64-bit integers, so each result carries only the
// truncation of the digits past the ninth (below 2^-52 of max|row| max|column|
// per term, an FP64 dot product's rounding).
//
// Kernels: ts_split_a (setup: panel slices and row scales), ts_clear (per
// level and call: the destination rows), ts_gemm (its K slice of the
// right-hand sides split into shared memory, gathering [D^{-1} y_s; -x_R] in
// the backward; bulk copies of the panel's slice tiles; tcgen05.mma into nine
// TMEM accumulators; the integer combination and the scatter of the solve in
// the epilogue: y_s to Y2, -u_R by FP64 atomics into the ancestors' rows,
// x_s to Y).
#include <cuda_bf16.h>

#include "kernels.h"
#include "tcgen05_util.cuh"

namespace matex {

namespace {

using namespace tcx;

constexpr int kTsM = 128;          // panel rows per tile (MMA M)
constexpr int kTsN = 32;           // right-hand sides per tile (MMA N)
constexpr int kTsThreads = 128;
constexpr int kTsABytes = kTsM * kTcK * 2;  // one slice of an A tile: 8 KB
constexpr int kTsBBytes = kTsN * kTcK * 2;  // one slice of a B tile: 2 KB
constexpr int kTsTmemCols = 512;   // nine accumulators of 32 columns fit in 288
constexpr uint32_t kTsIdesc = tc_idesc(kTsM, kTsN);
constexpr int kTsSliceSteps = 4;   // K steps of one CTA (128 reduction values: exact sums)

// Panel slices of supernode d in direction fwd: one thread per tile row
// (A row: panel row i forward, panel column k backward), all K steps.
__global__ void __launch_bounds__(kTsM)
ts_split_a_kernel(DevFactor F, const TsSup* __restrict__ sups, int fwd,
                  __nv_bfloat16* __restrict__ A, double* __restrict__ rowscale) {
  const TsSup d = sups[blockIdx.x];
  const int mt = blockIdx.y;
  const int mtiles = fwd ? d.mt_f : d.mt_b;
  if (mt >= mtiles) return;
  const int rows = fwd ? d.ld : d.w;    // rows of the product
  const int kdim = fwd ? d.w : d.ld;    // its reduction
  const int ksteps = (kdim + kTcK - 1) / kTcK;
  const int r = threadIdx.x;
  const int row = mt * kTsM + r;
  const bool live = row < rows;
  // forward A(i, k) = P(i, k): row i of the row-major panel; backward
  // A(k, i) = P(i, k): column k of the column-major panel
  const double* src = fwd ? F.pan_rm + d.pan + (int64_t)row * d.w
                          : F.pan_cm + d.pan + (int64_t)row * d.ld;
  double mx = 0.0;
  if (live)
    for (int k = 0; k < kdim; ++k) mx = fmax(mx, fabs(src[k]));
  const double sc = pow2_above(mx);
  if (live) rowscale[(fwd ? d.rs_f : d.rs_b) + row] = sc;
  const double inv = 1.0 / sc;  // a power of two: exact
  unsigned char* base = reinterpret_cast<unsigned char*>(A) + (fwd ? d.a_f : d.a_b) +
                        (size_t)mt * ksteps * kTcS * kTsABytes;
  for (int s = 0; s < ksteps; ++s) {
    unsigned char* blk = base + (size_t)s * kTcS * kTsABytes;
    for (int k8 = 0; k8 < kTcK; k8 += 8) {
      float sl[8][kTcS];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int k = s * kTcK + k8 + u;
        slice9(live && k < kdim ? src[k] * inv : 0.0, sl[u]);
      }
#pragma unroll
      for (int p = 0; p < kTcS; ++p) {
        uint4 w4;
        w4.x = pack_bf16x2(sl[0][p], sl[1][p]);
        w4.y = pack_bf16x2(sl[2][p], sl[3][p]);
        w4.z = pack_bf16x2(sl[4][p], sl[5][p]);
        w4.w = pack_bf16x2(sl[6][p], sl[7][p]);
        *reinterpret_cast<uint4*>(blk + (size_t)p * kTsABytes + tc_off(r, k8)) = w4;
      }
    }
  }
}

struct TsGemm {
  DevFactor F;
  const TsSup* sups;
  const int2* tiles;        // {wide supernode, row tile | K slice << 16} of the level
  const __nv_bfloat16* A;   // panel slices of this direction's factor
  const double* rowscale;
  double* Y;
  double* Y2;
  int ldy, ncols, fwd;
  int32_t* err;             // raised when a bounded wait gives up
};

// Destination rows of the level's wide supernodes cleared for the GEMM's
// atomics: y_s in Y2 (forward) or x_s in Y (backward), ncols columns; no one
// else reads them during this level.
__global__ void ts_clear_kernel(const TsSup* __restrict__ sups, const int32_t* __restrict__ list,
                                int fwd, double* Y, double* Y2, int ldy, int ncols) {
  const TsSup d = sups[list[blockIdx.x]];
  double* dst = fwd ? Y2 : Y;
  for (int e = threadIdx.x; e < d.w * ncols; e += blockDim.x) {
    const int k = e / ncols, q = e - k * ncols;
    dst[(int64_t)(d.f + k) * ldy + q] = 0.0;
  }
}

constexpr int kTsSliceVals = kTsSliceSteps * kTcK;  // reduction values of one CTA
constexpr int kTsBRes = kTsSliceSteps * kTcS * kTsBBytes;  // its resident B slices

// One CTA per (row tile of a wide supernode, K slice of kTsSliceSteps steps,
// 32 right-hand sides): a level's few wide supernodes become enough CTAs to
// keep the SMs busy.  The CTA first splits its own part of the right-hand
// sides: 128 reduction values x 32 columns read from Y / Y2 (thread (q, g):
// right-hand side q, 8-value groups g, g + 4, ...: a warp reads 32
// consecutive right-hand sides of one row), each column scaled by a power of
// two over this K slice, cut into nine digits straight into the resident B
// tiles in shared memory.  Then thread 0 streams the panel's slice tiles K
// step by K step into two shared-memory stages (bulk copies, completion by
// transaction count) and issues the MMAs of every slice pair p + q <= 8 into
// accumulator d = p + q (the slice's 128 values keep the sums exact); all 128
// threads drain the accumulators (warp w: tile rows 32w..32w+31), combine the
// nine integer sums exactly in 64-bit integers and add the FP64 result by
// atomics (the K slices of a tile meet there): forward y_s into Y2 and -u_R
// into the ancestors' rows of Y, backward x_s into Y (cleared by ts_clear).
__global__ void __launch_bounds__(kTsThreads, 1) ts_gemm_kernel(TsGemm g) {
  extern __shared__ __align__(1024) unsigned char ts_smem[];
  __shared__ uint32_t tbase;
  __shared__ __align__(8) uint64_t full[2], freed[2], fin;
  __shared__ int failed;
  __shared__ double cmax[kTsThreads / kTsN][kTsN];
  __shared__ double cscale[kTsN];
  const int2 tl = g.tiles[blockIdx.x];
  const TsSup d = g.sups[tl.x];
  const int mt = tl.y & 0xFFFF, kc = tl.y >> 16, nt = blockIdx.y;
  const int rows = g.fwd ? d.ld : d.w;
  const int kdim = g.fwd ? d.w : d.ld;
  const int ksteps = (kdim + kTcK - 1) / kTcK;
  const int s0 = kc * kTsSliceSteps, s1 = min(ksteps, s0 + kTsSliceSteps);
  const unsigned char* Abase = reinterpret_cast<const unsigned char*>(g.A) + (g.fwd ? d.a_f : d.a_b) +
                               (size_t)mt * ksteps * kTcS * kTsABytes;
  unsigned char* Bres = ts_smem + 2 * (size_t)kTcS * kTsABytes;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tbase)),
                 "r"(kTsTmemCols));
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
  // ---- the right-hand sides' slices of this K slice --------------------------
  {
    const int q = lane;                 // right-hand side within the tile
    const int qq = nt * kTsN + q;
    const bool qlive = qq < g.ncols;
    const int32_t* srow = g.F.sup_rows + d.rp;
    auto val = [&](int k) -> double {   // k: within the K slice
      const int kg = s0 * kTcK + k;
      if (!qlive || kg >= kdim) return 0.0;
      if (g.fwd) return g.Y[(int64_t)(d.f + kg) * g.ldy + qq];
      if (kg < d.w) return g.Y2[(int64_t)(d.f + kg) * g.ldy + qq] * g.F.dinv[d.f + kg];
      return -g.Y[(int64_t)srow[kg] * g.ldy + qq];
    };
    constexpr int NG = kTsSliceVals / 8 / (kTsThreads / kTsN);  // 8-value groups per thread
    double v[NG][8];
    double mx = 0.0;
#pragma unroll
    for (int i = 0; i < NG; ++i) {
      const int grp = warp + i * (kTsThreads / kTsN);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        v[i][u] = val(grp * 8 + u);
        mx = fmax(mx, fabs(v[i][u]));
      }
    }
    cmax[warp][q] = mx;
    __syncthreads();
    if (warp == 0) {
      double m = 0.0;
#pragma unroll
      for (int e = 0; e < kTsThreads / kTsN; ++e) m = fmax(m, cmax[e][q]);
      cscale[q] = pow2_above(m);
    }
    __syncthreads();
    const double inv = 1.0 / cscale[q];  // a power of two: exact
#pragma unroll
    for (int i = 0; i < NG; ++i) {
      const int grp = warp + i * (kTsThreads / kTsN);
      const int s = grp / (kTcK / 8), k8 = (grp % (kTcK / 8)) * 8;
      float sl[8][kTcS];
#pragma unroll
      for (int u = 0; u < 8; ++u) slice9(v[i][u] * inv, sl[u]);
      unsigned char* blk = Bres + (size_t)s * kTcS * kTsBBytes;
#pragma unroll
      for (int p = 0; p < kTcS; ++p) {
        uint4 w4;
        w4.x = pack_bf16x2(sl[0][p], sl[1][p]);
        w4.y = pack_bf16x2(sl[2][p], sl[3][p]);
        w4.z = pack_bf16x2(sl[4][p], sl[5][p]);
        w4.w = pack_bf16x2(sl[6][p], sl[7][p]);
        *reinterpret_cast<uint4*>(blk + (size_t)p * kTsBBytes + tc_off(q, k8)) = w4;
      }
    }
    // the generic-proxy stores must be visible to the tensor cores' reads
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tbase;
  const int row = mt * kTsM + 32 * warp + lane;
  const bool live = row < rows;
  const double rs = live ? g.rowscale[(g.fwd ? d.rs_f : d.rs_b) + row] : 0.0;
  // where this thread's row goes, and with which sign
  double* dst = nullptr;
  double sign = 1.0;
  if (live) {
    if (!g.fwd) {
      dst = g.Y + (int64_t)(d.f + row) * g.ldy;
    } else if (row < d.w) {
      dst = g.Y2 + (int64_t)(d.f + row) * g.ldy;
    } else {
      dst = g.Y + (int64_t)g.F.sup_rows[d.rp + row] * g.ldy;
      sign = -1.0;
    }
  }
  if (threadIdx.x == 0) {
    auto issue_copy = [&](int s, int k) {
      const int st = k & 1;
      unsigned char* a = ts_smem + (size_t)st * kTcS * kTsABytes;
      expect_tx(&full[st], kTcS * kTsABytes);
      bulk_load(a, Abase + (size_t)s * kTcS * kTsABytes, kTcS * kTsABytes, &full[st]);
    };
    bool ok = true;
    int it = 0;  // K steps issued (stage = it & 1, use = it >> 1)
    issue_copy(s0, 0);
    for (int s = s0; s < s1 && ok; ++s, ++it) {
      if (s + 1 < s1) {
        const int k = it + 1;
        // the stage was last used by step k - 2: its MMAs must be done
        if (k >= 2) ok = mbar_wait(&freed[k & 1], ((k >> 1) - 1) & 1);
        if (!ok) break;
        issue_copy(s + 1, k);
      }
      const int st = it & 1;
      if (!mbar_wait(&full[st], (it >> 1) & 1)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a = smem_addr(ts_smem + (size_t)st * kTcS * kTsABytes);
      const uint32_t b = smem_addr(Bres + (size_t)(s - s0) * kTcS * kTsBBytes);
#pragma unroll 1
      for (int p = 0; p < kTcS; ++p)
#pragma unroll 1
        for (int q = 0; q + p < kTcS; ++q)
#pragma unroll
          for (int kk = 0; kk < kTcK; kk += 16) {
            const uint64_t ad = tc_desc(a + p * kTsABytes + (kk / 8) * 128, 128, kTcSbo);
            const uint64_t bd = tc_desc(b + q * kTsBBytes + (kk / 8) * 128, 128, kTcSbo);
            const uint32_t acc = (s == s0 && p == 0 && kk == 0) ? 0u : 1u;
            tc_mma(tmem + (uint32_t)((p + q) * kTsN), ad, bd, kTsIdesc, acc);
          }
      tc_commit(&freed[st]);
    }
    if (ok) tc_commit(&fin);
    else failed = 1;
  }
  __syncthreads();
  const bool drained = !failed && mbar_wait(&fin, 0);
  if (drained) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // C_d at TMEM column d * kTsN + c of this warp's lanes
#pragma unroll 1
    for (int cb = 0; cb < kTsN; cb += 8) {
      uint32_t v[kTcS][8];
#pragma unroll
      for (int dd = 0; dd < kTcS; ++dd)
        tc_ld8(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(dd * kTsN + cb), v[dd]);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        const int q = nt * kTsN + cb + jj;
        if (!live || q >= g.ncols) continue;
        long long hi = 0, lo = 0;
#pragma unroll
        for (int dd = 0; dd < 5; ++dd)
          hi += (long long)__float2int_rz(__uint_as_float(v[dd][jj])) * (1ll << (6 * (4 - dd)));
#pragma unroll
        for (int dd = 5; dd < kTcS; ++dd)
          lo += (long long)__float2int_rz(__uint_as_float(v[dd][jj])) * (1ll << (6 * (8 - dd)));
        const double val = fma((double)lo, 0x1p-24, (double)hi) * (rs * cscale[cb + jj] * 0x1p-36);
        atomicAdd(dst + q, sign * val);
      }
    }
  } else if (threadIdx.x == 0) {
    failed = 1;
  }
  if (failed && threadIdx.x == 0) {
    atomicExch(g.err, 1);
    // let the MMAs already issued finish before the accumulators are freed
    tc_commit(&fin);
    mbar_wait(&fin, drained ? 1 : 0);  // bounded: gives up after about two seconds as well
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTsTmemCols));
  }
}

}  // namespace

// ---- host side ------------------------------------------------------------------

size_t ts_a_bytes(int rows, int kdim) {
  const size_t mt = (rows + kTsM - 1) / kTsM, ks = (kdim + kTcK - 1) / kTcK;
  return mt * ks * kTcS * kTsABytes;
}
int ts_row_tiles(int rows) { return (rows + kTsM - 1) / kTsM; }
int ts_k_slices(int kdim) { return ((kdim + kTcK - 1) / kTcK + kTsSliceSteps - 1) / kTsSliceSteps; }

constexpr int kTsSmem = 2 * kTcS * kTsABytes + kTsBRes;  // two panel stages, resident B slices

void ts_set_limits() {
  cudaFuncSetAttribute(ts_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTsSmem);
}

void ts_split_panels(const DevFactor& F, const TsSup* sups, int nsup, int max_mt, bool fwd,
                     __nv_bfloat16* A, double* rowscale, cudaStream_t st) {
  if (nsup <= 0) return;
  ts_split_a_kernel<<<dim3((unsigned)nsup, (unsigned)max_mt), kTsM, 0, st>>>(F, sups, fwd ? 1 : 0, A,
                                                                              rowscale);
}

void ts_solve_level(const DevFactor& F, const TsSup* sups, const TsLevel& L, bool fwd,
                    const __nv_bfloat16* A, const double* rowscale, double* Y, double* Y2, int ldy,
                    int ncols, int32_t* err, cudaStream_t st) {
  const int ntiles = fwd ? L.ntile_f : L.ntile_b;
  if (L.nsup <= 0 || ncols <= 0) return;
  const int nct = (ncols + kTsN - 1) / kTsN;
  ts_clear_kernel<<<(unsigned)L.nsup, 256, 0, st>>>(sups, L.list, fwd ? 1 : 0, Y, Y2, ldy, ncols);
  TsGemm g{F, sups, fwd ? L.tiles_f : L.tiles_b, A, rowscale, Y, Y2, ldy, ncols, fwd ? 1 : 0, err};
  ts_gemm_kernel<<<dim3((unsigned)ntiles, (unsigned)nct), kTsThreads, kTsSmem, st>>>(g);
}

}  // namespace matex
