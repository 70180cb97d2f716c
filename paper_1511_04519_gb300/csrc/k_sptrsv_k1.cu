// Single-right-hand-side level solves: the operator apply of Alg. 1 with one
// column (a segment of one group, the Krylov steps of a lone group, the
// fixed-step trapezoidal baseline).  With one column the work per tree level
// is small and each level launch is bound by its chain of dependent memory
// round trips, not by bandwidth or the FP64 pipe.  These kernels shorten that
// chain to one round trip after the previous level completes:
//   - everything that does not depend on the right-hand side (the warp's
//     work descriptor, its supernodes' sizes and offsets, the panel entries
//     of every lane's first trips, the ancestor rows of its first gathers) is loaded
//     before griddepcontrol.wait, while the previous level still runs
//     (programmatic dependent launch);
//   - after the wait a lane loads its right-hand-side entries (all in flight
//     at once), multiplies, reduces over its group of lanes by shuffles and
//     writes: no shared memory, no partial sums through global memory.
// Work: one output row (forward) or column (backward) of a supernode per
// group of G lanes (G a power of two, 16 panel entries per lane per trip);
// a warp covers 32 / G consecutive rows of the level's supernodes of one
// group size (small supernodes packed), found by a prefix sum over the rows
// of the warp's first 32 supernodes.  Forward row i of supernode s:
//   i <  w: y_i = D_i^{-1} (P_s b_s)_i  (stored, D^{-1} folded in here),
//   i >= w: b_{R(i)} -= (P_s b_s)_i     (FP64 atomic into the ancestor row);
// backward column k: x_k = sum_i P_s(i, k) v_i, v = [y_s; -x_R].
#include "kernels.h"

namespace matex {

namespace {

constexpr int kK1Threads = 32;  // one warp per CTA: a warp leaves as soon as it is done
constexpr int kK1Terms = 16;  // panel entries per lane per trip (two FMA chains)

__device__ __forceinline__ void k1_chain_wait() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Lane's row (forward) or column (backward) within the warp's supernodes:
// the supernode's record and the index i inside it.  Every lane calls it.
struct K1Lane {
  K1Sup d;
  int i;
  bool live;
  int G, sub;
};

template <bool kFwd>
__device__ __forceinline__ K1Lane k1_lane(const K1Sup* __restrict__ sups, int nsup, const K1Warp& wp,
                                          bool wvalid) {
  const int lane = threadIdx.x & 31;
  K1Lane L;
  L.G = 1 << wp.lg;
  L.sub = lane & (L.G - 1);
  const int slot = lane >> wp.lg;
  K1Sup md{};
  int cnt = 0;
  if (wvalid && wp.k0 + lane < nsup) {
    md = sups[wp.k0 + lane];
    cnt = kFwd ? md.ld : md.w;
  }
  // inclusive prefix of the rows (columns) of supernodes k0 .. k0 + lane
  int pre = cnt;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, pre, off);
    if (lane >= off) pre += v;
  }
  const int r = wp.i0 + slot;
  // m = number of the warp's supernodes whose rows end at or before r
  int m = 0;
#pragma unroll
  for (int b = 16; b > 0; b >>= 1) {
    const int pv = __shfl_sync(0xffffffffu, pre, m + b - 1);
    if (pv <= r) m += b;
  }
  const int mm = m < 32 ? m : 31;
  const int before = __shfl_sync(0xffffffffu, pre, mm > 0 ? mm - 1 : 0);
  L.d.po = __shfl_sync(0xffffffffu, md.po, mm);
  L.d.rp = __shfl_sync(0xffffffffu, md.rp, mm);
  L.d.f = __shfl_sync(0xffffffffu, md.f, mm);
  L.d.w = __shfl_sync(0xffffffffu, md.w, mm);
  L.d.ld = __shfl_sync(0xffffffffu, md.ld, mm);
  L.i = r - (mm > 0 ? before : 0);
  L.live = wvalid && slot < wp.nslot && m < 32;
  return L;
}

// sum over the G lanes of a group (G uniform across the warp)
__device__ __forceinline__ double k1_group_sum(double v, int G) {
  for (int off = G >> 1; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

__global__ void __launch_bounds__(kK1Threads)
k1_fwd_kernel(DevFactor F, const K1Sup* __restrict__ sups, int nsup,
              const K1Warp* __restrict__ warps, int nwarps, double* __restrict__ Y,
              double* __restrict__ Y2, int ldy) {
  const int wid = blockIdx.x * (kK1Threads / 32) + (threadIdx.x >> 5);
  const bool wvalid = wid < nwarps;
  const K1Warp wp = wvalid ? warps[wid] : K1Warp{0, 0, 0, 0, 0};
  const K1Lane L = k1_lane<true>(sups, nsup, wp, wvalid);
  const int i = L.i, w = L.d.w, ld = L.d.ld, G = L.G;
  const int n = L.live ? (i < w ? i + 1 : w) : 0;
  const int trips = __reduce_max_sync(0xffffffffu, (n + kK1Terms * G - 1) / (kK1Terms * G));
  const double* __restrict__ P = F.pan_cm + L.d.po + i;  // entry (i, t) at P[t * ld]
  // the first two trips' panel entries before the wait
  double q[kK1Terms], q1[kK1Terms];
#pragma unroll
  for (int u = 0; u < kK1Terms; ++u) {
    const int t = L.sub + G * u;
    q[u] = t < n ? __ldg(P + (int64_t)t * ld) : 0.0;
  }
  if (trips > 1) {
#pragma unroll
    for (int u = 0; u < kK1Terms; ++u) {
      const int t = kK1Terms * G + L.sub + G * u;
      q1[u] = t < n ? __ldg(P + (int64_t)t * ld) : 0.0;
    }
  }
  int orow = 0;
  double dinv = 0.0;
  if (L.live) {
    if (i < w) dinv = __ldg(F.dinv + L.d.f + i);
    else orow = __ldg(F.sup_rows + L.d.rp + i);
  }
  k1_chain_wait();
  if (F.abort && *F.abort) return;
  const double* __restrict__ b = Y + (int64_t)L.d.f * ldy;
  double acc = 0.0, acc2 = 0.0;
  for (int tr = 0; tr < trips; ++tr) {
    const int t0 = tr * kK1Terms * G + L.sub;
    if (tr == 1) {
#pragma unroll
      for (int u = 0; u < kK1Terms; ++u) q[u] = q1[u];
    } else if (tr > 1) {
#pragma unroll
      for (int u = 0; u < kK1Terms; ++u) {
        const int t = t0 + G * u;
        q[u] = t < n ? __ldg(P + (int64_t)t * ld) : 0.0;
      }
    }
    double x[kK1Terms];
#pragma unroll
    for (int u = 0; u < kK1Terms; ++u) {
      const int t = t0 + G * u;
      x[u] = t < n ? __ldcg(b + (int64_t)t * ldy) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kK1Terms; u += 2) {
      acc = fma(q[u], x[u], acc);
      acc2 = fma(q[u + 1], x[u + 1], acc2);
    }
  }
  acc = k1_group_sum(acc + acc2, G);
  if (L.live && L.sub == 0) {
    if (i < w) Y2[(int64_t)(L.d.f + i) * ldy] = acc * dinv;
    else atomicAdd(Y + (int64_t)orow * ldy, -acc);
  }
}

__global__ void __launch_bounds__(kK1Threads)
k1_bwd_kernel(DevFactor F, const K1Sup* __restrict__ sups, int nsup,
              const K1Warp* __restrict__ warps, int nwarps, double* __restrict__ Y,
              const double* __restrict__ Y2, int ldy) {
  const int wid = blockIdx.x * (kK1Threads / 32) + (threadIdx.x >> 5);
  const bool wvalid = wid < nwarps;
  const K1Warp wp = wvalid ? warps[wid] : K1Warp{0, 0, 0, 0, 0};
  const K1Lane L = k1_lane<false>(sups, nsup, wp, wvalid);
  const int k = L.i, w = L.d.w, G = L.G;
  const int n = L.live ? L.d.ld - k : 0;  // terms i = k .. ld - 1
  const int trips = __reduce_max_sync(0xffffffffu, (n + kK1Terms * G - 1) / (kK1Terms * G));
  const double* __restrict__ P = F.pan_rm + L.d.po + k;  // entry (i, k) at P[i * w]
  const int32_t* __restrict__ rows = F.sup_rows + L.d.rp;
  // the ancestor rows of the first three trips' gathers are loaded before
  // the wait, so after it a trip's gathers wait only for the right-hand side
  // (the later trips' panel entries load beside them)
  constexpr int kPre = 3;
  auto load_g = [&](int (&g)[kK1Terms], int tr) {
#pragma unroll
    for (int u = 0; u < kK1Terms; ++u) {
      const int t = tr * kK1Terms * G + L.sub + G * u, ii = k + t;
      g[u] = t < n && ii >= w ? __ldg(rows + ii) : -1;
    }
  };
  auto load_q = [&](double (&q)[kK1Terms], int tr) {
#pragma unroll
    for (int u = 0; u < kK1Terms; ++u) {
      const int t = tr * kK1Terms * G + L.sub + G * u, ii = k + t;
      q[u] = t < n ? __ldg(P + (int64_t)ii * w) : 0.0;
    }
  };
  double q[kK1Terms];
  int g[kPre][kK1Terms];
  load_q(q, 0);
#pragma unroll
  for (int tp = 0; tp < kPre; ++tp)
    if (tp < trips) load_g(g[tp], tp);
  k1_chain_wait();
  if (F.abort && *F.abort) return;
  const double* __restrict__ y = Y2 + (int64_t)L.d.f * ldy;
  double acc = 0.0, acc2 = 0.0;
  auto step = [&](const int (&gg)[kK1Terms], int tr) {
    double v[kK1Terms];
#pragma unroll
    for (int u = 0; u < kK1Terms; ++u) {
      const int t = tr * kK1Terms * G + L.sub + G * u, ii = k + t;
      v[u] = t >= n ? 0.0 : gg[u] < 0 ? __ldcg(y + (int64_t)ii * ldy) : -__ldcg(Y + (int64_t)gg[u] * ldy);
    }
#pragma unroll
    for (int u = 0; u < kK1Terms; u += 2) {
      acc = fma(q[u], v[u], acc);
      acc2 = fma(q[u + 1], v[u + 1], acc2);
    }
  };
#pragma unroll
  for (int tp = 0; tp < kPre; ++tp)
    if (tp < trips) {
      if (tp > 0) load_q(q, tp);
      step(g[tp], tp);
    }
  for (int tr = kPre; tr < trips; ++tr) {
    int gg[kK1Terms];
    load_g(gg, tr);
    load_q(q, tr);
    step(gg, tr);
  }
  acc = k1_group_sum(acc + acc2, G);
  if (L.live && L.sub == 0) Y[(int64_t)(L.d.f + k) * ldy] = acc;
}

}  // namespace

int solve_k1(const DevFactor& F, const K1Plan& P, double* Y, double* Y2, int ldy, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.blockDim = dim3(kK1Threads);
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const int wpc = kK1Threads / 32;
  int launches = 0;
  for (int l = 0; l < P.nlev; ++l) {
    const int nw = P.fw_off[l + 1] - P.fw_off[l];
    if (nw <= 0) continue;
    cfg.gridDim = dim3((unsigned)((nw + wpc - 1) / wpc));
    cudaLaunchKernelEx(&cfg, k1_fwd_kernel, F, (const K1Sup*)P.fsups, P.nsup,
                       (const K1Warp*)(P.fwarps + P.fw_off[l]), nw, Y, Y2, ldy);
    ++launches;
  }
  for (int l = P.nlev - 1; l >= 0; --l) {
    const int nw = P.bw_off[l + 1] - P.bw_off[l];
    if (nw <= 0) continue;
    cfg.gridDim = dim3((unsigned)((nw + wpc - 1) / wpc));
    cudaLaunchKernelEx(&cfg, k1_bwd_kernel, F, (const K1Sup*)P.bsups, P.nsup,
                       (const K1Warp*)(P.bwarps + P.bw_off[l]), nw, Y, (const double*)Y2, ldy);
    ++launches;
  }
  return launches;
}

}  // namespace matex
