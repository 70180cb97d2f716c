// Host setup, part 2: numeric supernodal L D L^T by the multifrontal method.
// This is the one-time serial factorisation of Alg. 2 (UMFPACK's LU in the
// paper); the matrices are SPD here (C diagonal positive, G a grounded
// conductance matrix), so a symmetric factorisation without pivoting is used.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>

#include "internal.h"

namespace matex {

namespace {

// Run f(lo, hi) over [0, n) split across the host's cores (serially when
// `work` is small).
template <typename F>
void parallel_for(int64_t n, double work, F f) {
  int nt = (int)std::min<unsigned>(std::max(1u, std::thread::hardware_concurrency()), 32u);
  if (work < 4e6 || n < nt) nt = 1;
  if (nt == 1) {
    f((int64_t)0, n);
    return;
  }
  std::vector<std::thread> th;
  const int64_t chunk = (n + nt - 1) / nt;
  for (int t = 0; t < nt; ++t) {
    const int64_t lo = t * chunk, hi = std::min(n, lo + chunk);
    if (lo >= hi) break;
    th.emplace_back([=, &f] { f(lo, hi); });
  }
  for (auto& x : th) x.join();
}

constexpr int64_t kPanel = 64;

// Partial L D L^T of the first w columns of the front F (nr x nr, column-major,
// lower triangle): blocked right-looking, panels of 64 columns, the trailing
// update of each panel spread over threads (columns are independent).
// On return column j < w holds l_j (unit diagonal implied) below the diagonal
// and dinv[j] = 1/d_j; the trailing (nr-w) x (nr-w) block holds the Schur
// complement.  Returns false on a non-positive pivot.
bool partial_ldlt(double* F, int64_t nr, int64_t w, double* dinv, std::vector<double>& W) {
  for (int64_t jb = 0; jb < w; jb += kPanel) {
    const int64_t b = std::min(kPanel, w - jb);
    // unscaled copies l_i d_j of the panel's columns, kept for the trailing update
    W.assign((size_t)b * nr, 0.0);
    for (int64_t j = jb; j < jb + b; ++j) {
      double* cj = &F[j * nr];
      const double d = cj[j];
      if (!(d > 0.0) || !std::isfinite(d)) return false;
      const double di = 1.0 / d;
      dinv[j] = di;
      double* wj = &W[(j - jb) * nr];
      for (int64_t i = j + 1; i < nr; ++i) wj[i] = cj[i];
      for (int64_t i = j + 1; i < nr; ++i) cj[i] *= di;
      // update the rest of the panel
      for (int64_t k = j + 1; k < jb + b; ++k) {
        const double lk = cj[k];
        if (lk == 0.0) continue;
        double* ck = &F[k * nr];
        for (int64_t i = k; i < nr; ++i) ck[i] -= wj[i] * lk;
      }
    }
    // trailing update: F[i][k] -= sum_j W[i][j] l_k,j for k >= jb+b, i >= k;
    // columns dealt cyclically over threads (the triangle shortens with k)
    const int64_t k0 = jb + b;
    const double work = (double)b * (double)(nr - k0) * (double)(nr - k0) / 2.0;
    const int64_t nt = std::max<int64_t>(1, std::min<int64_t>(32, std::thread::hardware_concurrency()));
    parallel_for(nt, work, [&](int64_t tlo, int64_t thi) {
      for (int64_t t = tlo; t < thi; ++t)
        for (int64_t kk = t; kk < nr - k0; kk += nt) {
          const int64_t k = k0 + kk;
          double* ck = &F[k * nr];
          for (int64_t j = jb; j < jb + b; ++j) {
            const double lk = F[j * nr + k];
            if (lk == 0.0) continue;
            const double* wj = &W[(j - jb) * nr];
            for (int64_t i = k; i < nr; ++i) ck[i] -= wj[i] * lk;
          }
        }
    });
  }
  return true;
}

}  // namespace

std::string numeric_ldlt(const CsrSym& A, const double* dshift, double alpha,
                         const Symbolic& S, Numeric& F) {
  const int64_t n = S.n;
  F.dinv.assign(n, 0.0);
  F.pan_cm.assign(S.pan_off[S.nsup], 0.0);
  F.pan_rm.assign(S.pan_off[S.nsup], 0.0);
  std::vector<int32_t> pos(n, -1);
  std::vector<std::vector<double>> upd(S.nsup);
  std::vector<std::vector<int32_t>> kids(S.nsup);
  for (int32_t s = 0; s < S.nsup; ++s)
    if (S.sup_parent[s] >= 0) kids[S.sup_parent[s]].push_back(s);
  std::vector<double> front, lcol;
  for (int32_t s = 0; s < S.nsup; ++s) {
    const int32_t f = S.sup_first[s], l = S.sup_first[s + 1];
    const int64_t w = l - f;
    const int32_t* R = &S.sup_rows[S.sup_rowptr[s]];
    const int64_t nr = S.sup_rowptr[s + 1] - S.sup_rowptr[s];
    const int64_t r = nr - w;
    for (int64_t k = 0; k < nr; ++k) pos[R[k]] = (int32_t)k;
    front.assign(nr * nr, 0.0);
    // assemble the columns of diag(dshift) + alpha*A owned by this supernode
    for (int32_t j = f; j < l; ++j) {
      int32_t o = S.perm[j];
      double* colj = &front[(j - f) * nr];
      for (int64_t p = A.rowptr[o]; p < A.rowptr[o + 1]; ++p) {
        int32_t i = S.iperm[A.col[p]];
        if (i < j) continue;
        if (pos[i] < 0) return "row outside the symbolic structure";
        colj[pos[i]] += alpha * A.val[p];
      }
      if (dshift) colj[j - f] += dshift[o];
    }
    // extend-add the children's update matrices
    for (int32_t c : kids[s]) {
      const int64_t wc = S.sup_first[c + 1] - S.sup_first[c];
      const int32_t* Rc = &S.sup_rows[S.sup_rowptr[c] + wc];
      const int64_t rc = S.sup_rowptr[c + 1] - S.sup_rowptr[c] - wc;
      const std::vector<double>& U = upd[c];
      std::vector<int32_t> rel(rc);
      for (int64_t a = 0; a < rc; ++a) rel[a] = pos[Rc[a]];
      for (int64_t b = 0; b < rc; ++b) {
        double* fc = &front[(int64_t)rel[b] * nr];
        const double* uc = &U[b * rc];
        for (int64_t a = b; a < rc; ++a) fc[rel[a]] += uc[a];
      }
      std::vector<double>().swap(upd[c]);
    }
    // partial factorisation of the first w columns
    if (!partial_ldlt(front.data(), nr, w, &F.dinv[f], lcol))
      return "matrix is not symmetric positive definite";
    // solve panel P = [L_ss^{-1}; L_Rs L_ss^{-1}]: column k of L_ss^{-1} by
    // forward substitution on e_k, then column k of L_Rs L_ss^{-1}
    double* pcm = &F.pan_cm[S.pan_off[s]];
    double* prm = &F.pan_rm[S.pan_off[s]];
    const int64_t ld = w + r;
    const double pwork = (double)w * (double)w * (double)ld / 2.0;
    parallel_for(w, pwork, [&](int64_t lo, int64_t hi) {
      for (int64_t k = lo; k < hi; ++k) {
        double* x = &pcm[k * ld];  // x[0..w) = L_ss^{-1} e_k, x[w..w+r) = L_Rs x[0..w)
        x[k] = 1.0;
        for (int64_t j = k; j < w; ++j) {
          const double xj = x[j];
          if (xj == 0.0) continue;
          const double* cj = &front[j * nr];
          for (int64_t i = j + 1; i < w; ++i) x[i] -= cj[i] * xj;
          for (int64_t i = 0; i < r; ++i) x[w + i] += cj[w + i] * xj;
        }
      }
    });
    parallel_for(ld, (double)w * ld, [&](int64_t lo, int64_t hi) {
      for (int64_t i = lo; i < hi; ++i)
        for (int64_t k = 0; k < w; ++k) prm[i * w + k] = pcm[k * ld + i];
    });
    // Schur complement handed to the parent
    if (r > 0 && S.sup_parent[s] >= 0) {
      std::vector<double>& U = upd[s];
      U.assign(r * r, 0.0);
      for (int64_t b = 0; b < r; ++b)
        std::memcpy(&U[b * r + b], &front[(w + b) * nr + w + b], sizeof(double) * (r - b));
    }
    for (int64_t k = 0; k < nr; ++k) pos[R[k]] = -1;
  }
  return "";
}

}  // namespace matex
