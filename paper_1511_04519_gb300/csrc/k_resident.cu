// Resident rounds for small grids: one CTA runs one column's whole segment of
// a round (Alg. 2's inner loop for one group), from the input solutions of
// Eq. 5/6 through the Arnoldi process of Alg. 1 with its residual test
// (Sec. 3.3.3) to the output coefficients and the state at the segment's end.
// Only the recombination of the round's outputs (Eq. 6, summed over the
// columns) stays a launch of its own.
//
// On a grid of a few thousand nodes every batched launch of the general path
// carries almost no work, so a segment there costs its ~80 launches' latency.
// Here the right-hand side and the forward intermediate live in shared memory,
// both triangular substitutions run level by level inside the CTA (a barrier
// per tree level instead of a launch), and the Gram-Schmidt reductions are
// CTA reductions.  The columns of a round are independent until the
// recombination, so a round of K columns is K CTAs with no inter-CTA wait.
#include "kernels.h"
#include "column_steps.cuh"

namespace matex {

namespace {


// Sum over the CTA, returned to every thread.  red: 32 doubles of shared memory.
__device__ __forceinline__ double res_block_sum(double v, double* red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  __syncthreads();  // earlier readers of red are done
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  const int nw = (int)(blockDim.x >> 5);
  for (int i = 0; i < nw; ++i) s += red[i];
  return s;
}


constexpr int kResBatch = 8;  // panel loads in flight per lane (masked FMAs cost full pipe time)

// Part of sum over k < n of p[k * stride] v[k] taken by lane sub of a group
// of lpr lanes (terms sub, sub + lpr, ...), kResBatch loads in flight per
// step: the panel entries come from L2, one round trip per batch per lane.
__device__ __forceinline__ double res_dot(const double* __restrict__ p, int64_t stride,
                                          const double* __restrict__ v, int n, int sub, int lpr) {
  double a0 = 0.0, a1 = 0.0;
  for (int k = sub; k < n; k += kResBatch * lpr) {
    double q[kResBatch], x[kResBatch];
#pragma unroll
    for (int u = 0; u < kResBatch; ++u) {
      const int kk = k + u * lpr;
      const bool ok = kk < n;
      q[u] = ok ? __ldg(p + (int64_t)kk * stride) : 0.0;
      x[u] = ok ? v[kk] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kResBatch; u += 2) {
      a0 = fma(q[u], x[u], a0);
      a1 = fma(q[u + 1], x[u + 1], a1);
    }
  }
  return a0 + a1;
}

// the same over gathered entries: terms p[i * stride] v[idx[i]] (idx in
// shared memory)
__device__ __forceinline__ double res_dot_gather(const double* __restrict__ p, int64_t stride,
                                                 const int* __restrict__ idx,
                                                 const double* __restrict__ v, int n, int sub,
                                                 int lpr) {
  double a0 = 0.0, a1 = 0.0;
  for (int k = sub; k < n; k += kResBatch * lpr) {
    double q[kResBatch], x[kResBatch];
#pragma unroll
    for (int u = 0; u < kResBatch; ++u) {
      const int kk = k + u * lpr;
      const bool ok = kk < n;
      q[u] = ok ? __ldg(p + (int64_t)kk * stride) : 0.0;
      x[u] = ok ? v[idx[kk]] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kResBatch; u += 2) {
      a0 = fma(q[u], x[u], a0);
      a1 = fma(q[u + 1], x[u + 1], a1);
    }
  }
  return a0 + a1;
}

// sum over the lpr lanes of a group (lpr a power of two <= 32, groups aligned
// in the warp); every lane of the warp must call it
__device__ __forceinline__ double res_group_sum(double v, int lpr) {
  for (int off = lpr >> 1; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// The plan's sections in shared memory (see ResidentPlan).
struct ResSmem {
  const int* offs;
  const ResSup* sups;
  const uint16_t* fsup;
  const uint16_t* bsup;
  const int* tgt;
  const int* tpp;
  const int* tslot;
  const int* brows;
};

// Copy the plan blob into shared memory at pl (16-byte aligned) and point
// into it; the caller synchronises before use.
__device__ __forceinline__ ResSmem res_stage_plan(const ResidentPlan& P, unsigned char* pl) {
  const int4* src = reinterpret_cast<const int4*>(P.blob);
  int4* dst = reinterpret_cast<int4*>(pl);
  for (int e = threadIdx.x; e < P.bytes / 16; e += blockDim.x) dst[e] = __ldg(src + e);
  ResSmem m;
  m.offs = reinterpret_cast<const int*>(pl + P.o_offs);
  m.sups = reinterpret_cast<const ResSup*>(pl + P.o_sups);
  m.fsup = reinterpret_cast<const uint16_t*>(pl + P.o_fsup);
  m.bsup = reinterpret_cast<const uint16_t*>(pl + P.o_bsup);
  m.tgt = reinterpret_cast<const int*>(pl + P.o_tgt);
  m.tpp = reinterpret_cast<const int*>(pl + P.o_tpp);
  m.tslot = reinterpret_cast<const int*>(pl + P.o_tslot);
  m.brows = reinterpret_cast<const int*>(pl + P.o_brows);
  return m;
}

// x = X^{-1} b for one right-hand side with the factor L D L^T of X (its
// resident copy F).  b (in: right-hand side, out: solution), y and U
// (scratch: n and P.uslots doubles) and the plan (m) are shared memory; b
// must be complete and visible to the CTA on entry.
//   forward, leaves first: [D_s^{-1} y_s; u_R] = P'_s b_s (P'_s: P_s with
//   D_s^{-1} folded into its diagonal block) with u_R into U, then
//   b_R -= u_R, each ancestor row by one thread, its contributions in a
//   fixed order.  A level reads only b_s of its own supernodes, which no
//   supernode of the level writes (the updates go to ancestors, which sit on
//   higher levels);
//   backward, root first: x_s = P_s^T [D_s^{-1} y_s; -x_R] with x_R already
//   final, written over b_s.
// Only panel entries come from global memory.  No atomics: the result does
// not depend on the order threads run in.  Every thread runs the same number
// of loop trips (the group sums shuffle).
__device__ void res_solve(const ResFactor& F, int nlev, const ResSmem& m, double* __restrict__ b,
                          double* __restrict__ y, double* __restrict__ U) {
  const int W = nlev + 1;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int l = 0; l < nlev; ++l) {
    const int r0 = m.offs[kResOffR * W + l], nrow = m.offs[kResOffR * W + l + 1] - r0;
    const int lpr = m.offs[kResOffFL * W + l];
    const int lb = m.offs[kResOffLB * W + l];
    const int sub = tid & (lpr - 1);
    for (int u0 = 0; u0 < nrow * lpr; u0 += nt) {
      const int t = (u0 + tid) / lpr;
      const bool live = t < nrow;
      double v = 0.0;
      ResSup d{};
      int i = 0;
      if (live) {
        d = m.sups[m.fsup[r0 + t]];
        i = t - d.rb;
        v = res_dot(F.fpan + d.p + i, d.ld, b + d.f, i < d.w ? i + 1 : d.w, sub, lpr);
      }
      v = res_group_sum(v, lpr);
      if (live && sub == 0) {
        if (i < d.w) y[d.f + i] = v;
        else U[d.gb + i - d.w - lb] = v;
      }
    }
    __syncthreads();
    const int t0 = m.offs[kResOffT * W + l], t1 = m.offs[kResOffT * W + l + 1];
    if (t1 > t0) {
      for (int j = t0 + tid; j < t1; j += nt) {
        const int row = m.tgt[j];
        double acc = b[row];
        for (int e = j > 0 ? m.tpp[j - 1] : 0; e < m.tpp[j]; ++e) acc -= U[m.tslot[e]];
        b[row] = acc;
      }
      __syncthreads();
    }
  }
  for (int l = nlev - 1; l >= 0; --l) {
    const int c0 = m.offs[kResOffC * W + l], ncol = m.offs[kResOffC * W + l + 1] - c0;
    const int lpr = m.offs[kResOffBL * W + l];
    const int sub = tid & (lpr - 1);
    for (int u0 = 0; u0 < ncol * lpr; u0 += nt) {
      const int t = (u0 + tid) / lpr;
      const bool live = t < ncol;
      double v = 0.0;
      ResSup d{};
      int k = 0;
      if (live) {
        d = m.sups[m.bsup[c0 + t]];
        k = t - d.cb;
        const double* __restrict__ p = F.bpan + d.p + k;  // (i, k) at i * w + k
        v = res_dot(p + (int64_t)k * d.w, d.w, y + d.f + k, d.w - k, sub, lpr) -
            res_dot_gather(p + (int64_t)d.w * d.w, d.w, m.brows + d.gb, b, d.ld - d.w, sub, lpr);
      }
      v = res_group_sum(v, lpr);
      if (live && sub == 0) b[d.f + k] = v;
    }
    __syncthreads();
  }
}

// hsh[k] = <V_k, b> for k < nb: one warp per basis vector
__device__ __forceinline__ void res_dots(const double* __restrict__ V, int64_t n, int nb,
                                         const double* __restrict__ b, double* hsh) {
  const int lane = threadIdx.x & 31, nw = (int)(blockDim.x >> 5);
  for (int k = (int)(threadIdx.x >> 5); k < nb; k += nw) {
    const double* __restrict__ vk = V + (int64_t)k * n;
    double a0 = 0.0, a1 = 0.0;
    int64_t i = lane;
    for (; i + 32 < n; i += 64) {
      a0 = fma(vk[i], b[i], a0);
      a1 = fma(vk[i + 32], b[i + 32], a1);
    }
    if (i < n) a0 = fma(vk[i], b[i], a0);
    double s = a0 + a1;
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) hsh[k] = s;
  }
}

__host__ __device__ constexpr size_t res_small_bytes() {
  return (sizeof(SmallShared) + 15) & ~(size_t)15;
}
constexpr int kResHsh = 24;  // >= kMaxB, padded
// solve kernel: the plan (16-byte aligned), then b, y, U
size_t res_solve_smem_bytes(int64_t n, const ResidentPlan& P) {
  return sizeof(double) * (2 * (size_t)n + (size_t)P.uslots) + (size_t)P.bytes;
}
// round kernel: the small dense work, the dot products and reductions, then
// as the solve kernel
size_t res_smem_bytes(int64_t n, const ResidentPlan& P) {
  return res_small_bytes() + sizeof(double) * ((size_t)kResHsh + 32) +
         res_solve_smem_bytes(n, P);
}

// The input part of column q's segment (Eq. 5/6 with the segment's source
// slopes s_j): z' = G^{-1} B s_j into Zp, w = G^{-1} C z' into W, and w left
// in b.  Depends on the sources only, not on the state.  b, y, U, the plan
// (ms) are shared memory; every thread of the CTA calls it.
__device__ void res_inputs(const ResidentArgs& a, const ResSmem& ms, int q, double* __restrict__ b,
                           double* __restrict__ y, double* __restrict__ U, double* __restrict__ Zp,
                           double* __restrict__ W) {
  const int64_t n = a.n;
  const int tid = threadIdx.x, nt = blockDim.x;
  const RoundCols& rc = a.rc;
  for (int64_t i = tid; i < n; i += nt) b[i] = 0.0;
  __syncthreads();
  // B s_j: the slopes of the column's sources on the segment
  {
    const SourceTable& src = a.src;
    const int sg = rc.sgroup ? rc.sgroup[q] : (int)rc.group[q];
    const double l0 = rc.l0[q], L = rc.len[q], l1 = l0 + L;
    const int p0 = src.grp_ptr[sg], p1 = src.grp_ptr[sg + 1];
    auto slope = [&](int p) {
      const int s = src.grp_src[p];
      const int o = src.pwl_off[s], np = src.pwl_off[s + 1] - o;
      const double u0 = pwl_eval(src.pwl_t + o, src.pwl_v + o, np, l0);
      return (pwl_eval(src.pwl_t + o, src.pwl_v + o, np, l1) - u0) / L;
    };
    // slopes in parallel (y is free until the first solve), then added in
    // source order by one thread: sources may share a node
    if (p1 - p0 <= n) {
      for (int p = p0 + tid; p < p1; p += nt) y[p - p0] = slope(p);
      __syncthreads();
      if (tid == 0)
        for (int p = p0; p < p1; ++p) b[src.node[src.grp_src[p]]] += y[p - p0];
    } else if (tid == 0) {
      for (int p = p0; p < p1; ++p) b[src.node[src.grp_src[p]]] += slope(p);
    }
  }
  __syncthreads();
  res_solve(a.FG, a.plan.nlev, ms, b, y, U);  // z' = G^{-1} B s_j
  for (int64_t i = tid; i < n; i += nt) {
    const double zp = b[i];
    Zp[i] = zp;
    b[i] = zp * a.cperm[i];
  }
  __syncthreads();
  res_solve(a.FG, a.plan.nlev, ms, b, y, U);  // w = G^{-1} C z'
  for (int64_t i = tid; i < n; i += nt) W[i] = b[i];
}

__global__ void __launch_bounds__(kResidentThreads, 1) resident_round_kernel(ResidentArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmallShared& sh = *reinterpret_cast<SmallShared*>(smem_raw);
  double* hsh = reinterpret_cast<double*>(smem_raw + res_small_bytes());
  int* stflag = reinterpret_cast<int*>(hsh + kResHsh - 1);  // past the kMaxB dot products
  double* red = hsh + kResHsh;
  unsigned char* pl = reinterpret_cast<unsigned char*>(red + 32);  // 16-byte aligned
  const int64_t n = a.n;
  double* b = reinterpret_cast<double*>(pl + a.plan.bytes);
  double* y = b + n;
  double* U = y + n;
  const int nlev = a.plan.nlev;
  const RoundCols& rc = a.rc;
  SmallState& ss = a.ss;
  const int q = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t g = rc.group[q];
  double* __restrict__ X = a.X + g * n;
  double* __restrict__ Z = a.Z + g * n;
  double* __restrict__ Zp = a.Zp + g * n;
  double* __restrict__ W = a.W + g * n;
  double* __restrict__ V = a.Vb + (int64_t)rc.vslot[q] * a.vstride;
  // z carried over the breakpoint (z_0 = x(0), z_j = z_{j-1} + L_{j-1} z'_{j-1})
  const bool first = rc.seg[q] == 0;
  const double lp = rc.lprev[q];
  if (tid == 0) sh.cm = 0;  // no residual test has run yet
  const ResSmem ms = res_stage_plan(a.plan, pl);
  double acc = 0.0;
  if (a.zpre) {
    // z' and w of this segment computed ahead (resident_inputs): the start
    // vector v = x + F (F = w - z, Eq. 6) right away
    const double* __restrict__ zq = a.zpre + (int64_t)q * n;
    const double* __restrict__ wq = a.wpre + (int64_t)q * n;
    for (int64_t i = tid; i < n; i += nt) {
      const double z = first ? X[i] : fma(lp, Zp[i], Z[i]);
      const double wv = wq[i];
      Z[i] = z;
      Zp[i] = zq[i];
      W[i] = wv;
      const double v = X[i] + (wv - z);
      b[i] = v;
      acc = fma(v, v, acc);
    }
    __syncthreads();
  } else {
    for (int64_t i = tid; i < n; i += nt) Z[i] = first ? X[i] : fma(lp, Zp[i], Z[i]);
    res_inputs(a, ms, q, b, y, U, Zp, W);
    // start vector v = x + F (F = w - z, Eq. 6), beta = ||v||
    for (int64_t i = tid; i < n; i += nt) {
      const double v = X[i] + (b[i] - Z[i]);
      b[i] = v;
      acc = fma(v, v, acc);
    }
  }
  const double beta = sqrt(res_block_sum(acc, red));
  double* Ht = ss.Ht + (int64_t)q * kMaxB * kMaxM;
  for (int e = tid; e < kMaxB * kMaxM; e += nt) Ht[e] = 0.0;
  const bool quiet = beta <= 1e-300;
  if (tid == 0) {
    ss.beta[q] = beta;
    ss.m[q] = 0;
    ss.status[q] = quiet ? 4 : 0;
    ss.scale[q] = quiet ? 0.0 : 1.0 / beta;
  }
  if (!quiet) {
    const double sc = 1.0 / beta;
    for (int64_t i = tid; i < n; i += nt) V[i] = b[i] * sc;
    for (int j = 0; j < a.m_max; ++j) {
      // w = X1^{-1} C v_j (Alg. 1 with X2 = C)
      const double* __restrict__ vj = V + (int64_t)j * n;
      __syncthreads();
      for (int64_t i = tid; i < n; i += nt) b[i] = vj[i] * a.cperm[i];
      __syncthreads();
      res_solve(a.F1, nlev, ms, b, y, U);
      // two classical Gram-Schmidt passes against v_0..v_j
      for (int pass = 0; pass < 2; ++pass) {
        res_dots(V, n, j + 1, b, hsh);
        __syncthreads();
        if (tid <= j) Ht[tid * kMaxM + j] += hsh[tid];
        for (int64_t i = tid; i < n; i += nt) {
          double t = b[i];
          for (int k = 0; k <= j; ++k) t = fma(-hsh[k], V[(int64_t)k * n + i], t);
          b[i] = t;
        }
        __syncthreads();
      }
      double a2 = 0.0;
      for (int64_t i = tid; i < n; i += nt) a2 = fma(b[i], b[i], a2);
      const double nrm = sqrt(res_block_sum(a2, red));
      const double sc2 = nrm > 0.0 ? 1.0 / nrm : 0.0;
      if (tid == 0) {
        Ht[(j + 1) * kMaxM + j] = nrm;
        ss.scale[q] = sc2;
      }
      double* __restrict__ vn = V + (int64_t)(j + 1) * n;
      for (int64_t i = tid; i < n; i += nt) vn[i] = b[i] * sc2;
      // the residual test (small dense work) by warp 0 alone: warp barriers
      // instead of CTA barriers between its many short steps
      __syncthreads();
      if (tid < 32) {
        const int st = residual_column<WarpGroup>(ss, rc, q, j, a.gamma, a.tol, a.m_max, a.replay, sh);
        if (tid == 0) *stflag = st;
      }
      __syncthreads();
      if (*stflag != 0) break;
    }
  }
  __syncthreads();
  if (tid < 32)
    coef_column<WarpGroup>(ss, rc, q, a.gamma, a.dt_out, a.coef, a.ldo, a.yend, 0.0, nullptr, nullptr,
                           sh);
  __syncthreads();
  // state at the segment's end: x = z + L z' - w + V y(L)
  const int m = ss.m[q];
  const double L = rc.len[q];
  const double* ye = a.yend + (int64_t)q * kMaxM;
  for (int64_t i = tid; i < n; i += nt) {
    double s = Z[i] + L * Zp[i] - W[i];
    for (int k = 0; k < m; ++k) s = fma(V[(int64_t)k * n + i], ye[k], s);
    X[i] = s;
  }
  if (tid == 0) {
    a.m_rec[rc.segid[q]] = m;
    a.st_rec[rc.segid[q]] = ss.status[q];
  }
}

// The input solves of columns q (one CTA each) ahead of their rounds:
// z' and w of column q into zpre + q n and wpre + q n.
__global__ void __launch_bounds__(kResidentThreads, 1) resident_inputs_kernel(ResidentArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const ResSmem ms = res_stage_plan(a.plan, smem_raw);
  const int64_t n = a.n;
  double* b = reinterpret_cast<double*>(smem_raw + a.plan.bytes);
  double* y = b + n;
  double* U = y + n;
  const int q = blockIdx.x;
  res_inputs(a, ms, q, b, y, U, a.zpre + (int64_t)q * n, a.wpre + (int64_t)q * n);
}

// Solve pairs x_q = F^{-1} b_q, one CTA per right-hand side q.  Entry i of
// column q sits at q * ldq + r(i) * ldi, r(i) = perm[i] (perm: new -> old,
// the caller's order) or i (the factor's order).  b and x may alias.
__global__ void __launch_bounds__(kResidentThreads, 1)
resident_solve_kernel(ResFactor F, ResidentPlan P, const double* bin, double* xout, int64_t n,
                      int64_t ldi, int64_t ldq, const int32_t* __restrict__ perm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const ResSmem ms = res_stage_plan(P, smem_raw);
  double* b = reinterpret_cast<double*>(smem_raw + P.bytes);
  double* y = b + n;
  double* U = y + n;
  const double* bq = bin + (int64_t)blockIdx.x * ldq;
  double* xq = xout + (int64_t)blockIdx.x * ldq;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) b[i] = bq[(perm ? perm[i] : i) * ldi];
  __syncthreads();
  res_solve(F, P.nlev, ms, b, y, U);
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) xq[(perm ? perm[i] : i) * ldi] = b[i];
}

// Resident copy of one supernode's panel per CTA: forward rows with D^{-1}
// folded into the diagonal block, backward columns as they are.
__global__ void resident_store_kernel(DevFactor F, const ResStoreSup* __restrict__ sup,
                                      double* __restrict__ fpan, double* __restrict__ bpan) {
  const ResStoreSup d = sup[blockIdx.x];
  const int64_t cnt = (int64_t)d.ld * d.w;
  for (int64_t e = threadIdx.x; e < cnt; e += blockDim.x) {
    const int i = (int)(e % d.ld);  // column-major: e = k * ld + i
    const double sc = i < d.w ? F.dinv[d.f + i] : 1.0;
    fpan[d.fdst + e] = F.pan_cm[d.src + e] * sc;
    bpan[d.bdst + e] = F.pan_rm[d.src + e];
  }
}

}  // namespace

void resident_store(const DevFactor& F, const ResStoreSup* sup, int nsup, double* fpan, double* bpan,
                    cudaStream_t st) {
  if (nsup <= 0) return;
  resident_store_kernel<<<nsup, 256, 0, st>>>(F, sup, fpan, bpan);
}

bool resident_fits(int64_t n, const ResidentPlan& P) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return n > 0 && n <= kResidentMaxN && res_smem_bytes(n, P) <= (size_t)optin;
}

bool resident_set_limits(int64_t n, const ResidentPlan& P) {
  // the kernels' limits only grow: contexts of several sizes share them
  static size_t done = 0;
  const size_t bytes = res_smem_bytes(n, P);
  if (bytes <= done) return true;
  const bool ok =
      cudaFuncSetAttribute(resident_round_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)bytes) == cudaSuccess &&
      cudaFuncSetAttribute(resident_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)res_solve_smem_bytes(n, P)) == cudaSuccess &&
      cudaFuncSetAttribute(resident_inputs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)res_solve_smem_bytes(n, P)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return false;
  }
  done = bytes;
  return true;
}

void resident_round(const ResidentArgs& a, int K, cudaStream_t st) {
  if (K <= 0) return;
  resident_round_kernel<<<K, kResidentThreads, res_smem_bytes(a.n, a.plan), st>>>(a);
}

void resident_inputs(const ResidentArgs& a, int K, cudaStream_t st) {
  if (K <= 0) return;
  resident_inputs_kernel<<<K, kResidentThreads, res_solve_smem_bytes(a.n, a.plan), st>>>(a);
}

void resident_solve(const ResFactor& F, const ResidentPlan& P, const double* b, double* x,
                    int64_t n, int ncols, int64_t ldi, int64_t ldq, const int32_t* perm,
                    cudaStream_t st) {
  if (ncols <= 0) return;
  const size_t smem = res_solve_smem_bytes(n, P);
  resident_solve_kernel<<<ncols, kResidentThreads, smem, st>>>(F, P, b, x, n, ldi, ldq, perm);
}

float resident_time_solve(const ResFactor& F, const ResidentPlan& P, const double* b, double* x,
                          int64_t n, cudaStream_t st, int reps) {
  resident_solve(F, P, b, x, n, 1, 1, n, nullptr, st);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = -1.f;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(e0, st);
    resident_solve(F, P, b, x, n, 1, 1, n, nullptr, st);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (best < 0.f || ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cudaGetLastError() != cudaSuccess) return -1.f;
  return best;
}

}  // namespace matex
