// Host setup, part 2: numeric supernodal L D L^T by the multifrontal method.
// This is the one-time serial factorisation of Alg. 2 (UMFPACK's LU in the
// paper); the matrices are SPD here (C diagonal positive, G a grounded
// conductance matrix), so a symmetric factorisation without pivoting is used.
#include <cmath>
#include <cstring>

#include "internal.h"

namespace matex {

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
    // partial factorisation of the first w columns (right-looking)
    lcol.resize(nr);
    for (int64_t j = 0; j < w; ++j) {
      double* cj = &front[j * nr];
      const double d = cj[j];
      if (!(d > 0.0) || !std::isfinite(d)) return "matrix is not symmetric positive definite";
      const double di = 1.0 / d;
      for (int64_t k = j + 1; k < nr; ++k) lcol[k] = cj[k] * di;
      for (int64_t k = j + 1; k < nr; ++k) {
        const double lk = lcol[k];
        if (lk == 0.0) continue;
        double* ck = &front[k * nr];
        for (int64_t i = k; i < nr; ++i) ck[i] -= cj[i] * lk;
      }
      for (int64_t k = j + 1; k < nr; ++k) cj[k] = lcol[k];
      F.dinv[f + j] = di;
    }
    // solve panel P = [L_ss^{-1}; L_Rs L_ss^{-1}]: column k of L_ss^{-1} by
    // forward substitution on e_k, then column k of L_Rs L_ss^{-1}
    double* pcm = &F.pan_cm[S.pan_off[s]];
    double* prm = &F.pan_rm[S.pan_off[s]];
    const int64_t ld = w + r;
    for (int64_t k = 0; k < w; ++k) {
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
    for (int64_t k = 0; k < w; ++k)
      for (int64_t i = 0; i < ld; ++i) prm[i * w + k] = pcm[k * ld + i];
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
