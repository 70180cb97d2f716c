// Per-column small steps of one segment, executed by a thread group G (all
// threads of a CTA of any size, or one warp): the residual test of Sec. 3.3.3 after Arnoldi step j, and
// the coefficient vectors ||v|| e^{h H_m} e_1 at the segment's outputs and its
// end (Alg. 2, "snapshots" reuse the basis).  Shared by the batched kernels
// (one CTA per column of a round) and the resident round kernel (one CTA runs
// a column's whole segment).
#pragma once
#include "kernels.h"
#include "small_dense.cuh"

namespace matex {
namespace {

using ExpmWork = SmallWork<kMaxM>;
constexpr int kLd = Small<kMaxM>::kLd;
constexpr int kMat = Small<kMaxM>::kMat;

template <class G = CtaGroup>
__device__ __forceinline__ void expm_dev(const double* M, double h, double* E, int m, ExpmWork& w) {
  Small<kMaxM, G>::expm(M, h, E, m, w);
}
template <class G = CtaGroup>
__device__ __forceinline__ void rational_H(const double* Ht, int m, double gamma, double* H,
                                           ExpmWork& w, int variant) {
  Small<kMaxM, G>::rational_H(Ht, m, gamma, H, w, variant);
}

// value at x of the piecewise-linear source (t, v) with np breakpoints, held
// constant outside [t_0, t_{np-1}]
__device__ __forceinline__ double pwl_eval(const double* t, const double* v, int np, double x) {
  if (x <= t[0]) return v[0];
  if (x >= t[np - 1]) return v[np - 1];
  int j = 0;
  while (j + 1 < np && t[j + 1] <= x) ++j;
  const double slope = (v[j + 1] - v[j]) / (t[j + 1] - t[j]);
  return slope * (x - t[j]) + v[j];
}

struct SmallShared {
  ExpmWork w;
  double H[kMat];
  double E[kMat];
  double y[kMaxM], y2[kMaxM];
  int flag;
  // the last residual test's H (for Krylov dimension cm) and its two
  // exponentials e^{ch[i] H} (ce[i]); cm = 0: none.  The caller clears cm
  // where the shared memory is not that of the test's own CTA.
  int cm;
  double ch[2];
  double ce[2][kMat];
};

// Status of column q after Arnoldi step j (m = j + 1), returned to every
// thread and stored in ss.status[q]: 0 iterate on, 1 converged (or the
// replayed dimension reached), 2 happy breakdown, 3 m_max reached unconverged.
// The residual of Sec. 3.3.3, ||v|| |h_{m+1,m} e_m^T e^{hH} e_1| (h_{m+1,m}
// scaled by ss.rscale), is taken at the segment's first output and at its end.
// Ht and ss.beta[q] may have been written by any thread of the CTA before the call.
template <class G = CtaGroup>
__device__ int residual_column(SmallState ss, const RoundCols& rc, int q, int j, double gamma,
                               double tol, int m_max, const int32_t* __restrict__ replay,
                               SmallShared& sh) {
  const int m = j + 1;
  const double* Ht = ss.Ht + (int64_t)q * kMaxB * kMaxM;
  G::sync();  // Ht complete; sh.flag of an earlier call has been read
  const double hnext = Ht[m * kMaxM + (m - 1)];
  if (G::rank() == 0) {
    ss.m[q] = m;
    int st = 0;
    if (hnext <= 1e-13 * fabs(Ht[0])) st = 2;  // happy breakdown (h_11 < 0 for A itself)
    else if (replay) st = (replay[rc.segid[q]] <= m) ? 1 : 0;
    sh.flag = st;
  }
  G::sync();
  int st = sh.flag;
  if (st == 0 && !replay) {
    rational_H<G>(Ht, m, gamma, sh.H, sh.w, ss.krylov);
    const double L = rc.len[q];
    const double hc = fmin(rc.hfirst[q], L);
    double rmax = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
      double* E = sh.ce[pass];
      expm_dev<G>(sh.H, pass == 0 ? hc : L, E, m, sh.w);
      // r = ||v|| |s h_{m+1,m} e_m^T e^{hH} e_1|, s making h_{m+1,m} dimensionless
      rmax = fmax(rmax, ss.beta[q] * fabs(ss.rscale * hnext) * fabs(E[(m - 1) * kLd + 0]));
    }
    if (rmax < tol) st = 1;
    if (G::rank() == 0) {
      sh.cm = m;
      sh.ch[0] = hc;
      sh.ch[1] = L;
    }
    G::sync();
  } else if (G::rank() == 0) {
    sh.cm = 0;
  }
  if (st == 0 && m >= m_max) st = 3;
  if (G::rank() == 0) ss.status[q] = st;
  return st;
}

// Coefficients of column q at the outputs of its segment: coef row o holds
// y(h_o) = ||v|| e^{h_o H_m} e_1 (h_o = t_o - l_j) in slots 0..m-1 and h_o in
// slot kMaxM; yend[q] = y(L).  With tail_eps > 0 and pbound given, tcut[q]
// receives the tail cut (outputs up to the last one whose ||y||_2 exceeds
// tail_eps/2 keep V y; a NaN norm or bound counts as large).
template <class G = CtaGroup>
__device__ void coef_column(SmallState ss, const RoundCols& rc, int q, double gamma, double dt_out,
                            double* __restrict__ coef, int ldo, double* __restrict__ yend,
                            double tail_eps, const double* __restrict__ pbound,
                            int32_t* __restrict__ tcut, SmallShared& sh) {
  const int m = ss.m[q];
  const int no = rc.nout[q];
  double* cq = coef + (int64_t)q * ldo * kCoefLd;
  const bool cut = pbound != nullptr && tail_eps > 0.0;
  const double e2 = 0.25 * tail_eps * tail_eps;
  int last = -1;
  auto put_cut = [&]() {
    if (tcut == nullptr || G::rank() != 0) return;
    tcut[2 * q] = cut ? last + 1 : no;
    tcut[2 * q + 1] =
        cut && pbound[2 * q] + rc.len[q] * pbound[2 * q + 1] <= 0.5 * tail_eps ? 1 : 0;
  };
  auto note_norm = [&](int o) {
    if (!cut || G::rank() != 0) return;
    double s = 0.0;
    for (int k = 0; k < m; ++k) s = fma(sh.y[k], sh.y[k], s);
    if (!(s <= e2)) last = o;
  };
  // step of the -P term at every output: h = t_o - l_j with t_o = o * dt_out
  for (int o = G::rank(); o < no; o += G::size())
    cq[(int64_t)o * kCoefLd + kMaxM] = (double)(rc.obeg[q] + o) * dt_out - rc.l0[q];
  if (m <= 0 || no <= 0) {
    put_cut();
    if (m <= 0) return;
  }
  const double* Ht = ss.Ht + (int64_t)q * kMaxB * kMaxM;
  const double beta = ss.beta[q];
  // e^{hH} for h = t: from the residual test of this m when it took it
  const bool cached = sh.cm == m;
  auto expm_at = [&](double t) -> const double* {
    if (cached && sh.ch[0] == t) return sh.ce[0];
    if (cached && sh.ch[1] == t) return sh.ce[1];
    expm_dev<G>(sh.H, t, sh.E, m, sh.w);
    return sh.E;
  };
  if (!cached) rational_H<G>(Ht, m, gamma, sh.H, sh.w, ss.krylov);
  // segment end
  const double* E = expm_at(rc.len[q]);
  for (int i = G::rank(); i < m; i += G::size()) yend[(int64_t)q * kMaxM + i] = beta * E[i * kLd];
  if (no <= 0) return;
  G::sync();
  // first output, then the propagator e^{dt H} for the equally spaced rest
  E = expm_at(rc.hfirst[q]);
  for (int i = G::rank(); i < m; i += G::size()) {
    sh.y[i] = beta * E[i * kLd];
    cq[i] = sh.y[i];
  }
  G::sync();
  note_norm(0);
  if (no > 1) {
    expm_dev<G>(sh.H, dt_out, sh.E, m, sh.w);
    for (int o = 1; o < no; ++o) {
      for (int i = G::rank(); i < m; i += G::size()) {
        double s = 0.0;
        for (int k = 0; k < m; ++k) s = fma(sh.E[i * kLd + k], sh.y[k], s);
        sh.y2[i] = s;
        cq[(int64_t)o * kCoefLd + i] = s;
      }
      G::sync();
      for (int i = G::rank(); i < m; i += G::size()) sh.y[i] = sh.y2[i];
      G::sync();
      note_norm(o);
    }
  }
  put_cut();
}

}  // namespace
}  // namespace matex
